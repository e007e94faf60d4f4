"""The lane layouts of the double-FP32 sweep, each against the oracle.

The double-FP32 sweep picks its lane layout per target from the bins: lane
groups (a lane per emitting point) while the lit rays carry at most 14
points on average, each ray with more than 32 points then swept by a lane
pair; lane pairs for every ray above that mean.  The scenes here put a
target into each case on purpose; the oracle's bins confirm that the scene
does what it is meant to, then the fluxes of the target and of cells near
it are compared with the oracle in all three forms.

* long ray among short ones: a row of point sources along the diagonal
  from the corner cell of a 128^3 grid, one per radial point (Eq. 4), and
  47 sources in other directions.  The corner cell sees one ray with more
  than 32 emitting points and a few rays with one or two.
* many points on every ray: emission from every cell (diffuse), so that the
  lit rays of every target carry more than 14 points on average.
"""
import numpy as np
import pytest

from helpers import KAPPA
from oracle_pool import sampled_check, uniform_neighbours
from test_gpu_parity import B, RTOL, gpu_solve  # noqa: F401
from workloads import PC_CM, Workload

pytestmark = pytest.mark.gpu

FORMS = [0, 1, 2]
GROUP_MAX, GROUP_MEAN_MAX = 32, 14


def long_ray_scene(orc, N=128):
    """Optically thin gas (n_H = 1 cm^-3, 10 pc box); sources at the radial
    points r_i along (1, 1, 1) from the centre of cell (0, 0, 0), and 47 at
    100 cells in seeded directions of the same octant."""
    box = 10.0 * PC_CM
    dx = box / N
    u = np.ones(3) / np.sqrt(3.0)
    t0 = np.full(3, 0.5)
    line = [t0 + orc.radius(i, 2) * u for i in range(1, 60)]
    line = [x for x in line if np.all(x < N - 0.5)]
    rng = np.random.default_rng(7)
    far = []
    for _ in range(47):
        v = np.abs(rng.normal(size=3))
        far.append(t0 + 100.0 * v / np.linalg.norm(v))
    xyz = np.array(line + far) * dx
    q = np.full(len(xyz), 1e46)
    return Workload("longray128", N, box, np.ones((N, N, N)), xyz, q, theta_src=0.05)


def emitting_points(orc_tree, p, target):
    eps = orc_tree.walk(p, int(target))["eps"]
    return (eps[:, 1:] > 0).sum(axis=1)


def diagonal_cells(N, k):
    return np.array([(i * N + i) * N + i for i in range(k)], dtype=np.int64)


@pytest.fixture(scope="module")
def long_ray(orc):
    w = long_ray_scene(orc)
    t, p = orc.Tree(w), orc.params_for(w)
    return w, t, p


def test_long_ray_scene_takes_groups_with_a_pair_swept_ray(long_ray):
    w, t, p = long_ray
    c = emitting_points(t, p, 0)
    lit = c[c > 0]
    assert c.max() > GROUP_MAX
    assert lit.sum() <= GROUP_MEAN_MAX * lit.size


@pytest.mark.parametrize("precision", FORMS)
def test_long_ray_against_oracle(B, long_ray, precision):
    w, t, p = long_ray
    F, e, ion = gpu_solve(B, w, precision)
    targets = diagonal_cells(w.N, 12)
    checked, worst = sampled_check(F, ion, targets, uniform_neighbours(targets, w.N),
                                   lambda c: t.solve_pass(p, targets=c), RTOL[precision], KAPPA[precision],
                                   lambda c: t.free_flux(p, targets=c))
    assert checked == targets.size                  # all lit, none at a front: thin gas


def diffuse_scene(N=128):
    """Every cell emits in proportion to n_H^2 (a log-normal field of mean
    n_H = 1 cm^-3), no point sources.  The emission, 1e52 s^-1 in all, is
    well above each cell's own recombinations, so every cell emits after
    the netting (Sec. 2.2) and every target's lit rays carry many points."""
    from workloads import lognormal_density
    box = 10.0 * PC_CM
    rho = lognormal_density(N, 2105) / 100.0
    w2 = rho * rho
    ndot = 1e52 * w2 / w2.sum()
    return Workload(f"diffuse{N}", N, box, rho, np.zeros((0, 3)), np.zeros(0), ndot_cell=ndot)


@pytest.fixture(scope="module")
def diffuse(orc):
    w = diffuse_scene()
    t, p = orc.Tree(w), orc.params_for(w)
    return w, t, p


def test_diffuse_scene_takes_pairs(diffuse):
    w, t, p = diffuse
    rng = np.random.default_rng(64)
    for target in rng.choice(w.N ** 3, 4, replace=False):
        c = emitting_points(t, p, target)
        lit = c[c > 0]
        assert lit.sum() > GROUP_MEAN_MAX * lit.size


@pytest.mark.parametrize("precision", FORMS)
def test_diffuse_against_oracle(B, diffuse, precision):
    w, t, p = diffuse
    F, e, ion = gpu_solve(B, w, precision)
    rng = np.random.default_rng(65)
    targets = rng.choice(w.N ** 3, 40, replace=False).astype(np.int64)
    checked, worst = sampled_check(F, ion, targets, uniform_neighbours(targets, w.N),
                                   lambda c: t.solve_pass(p, targets=c), RTOL[precision], KAPPA[precision],
                                   lambda c: t.free_flux(p, targets=c))
    assert checked >= 20
