"""End-to-end pins of the oracle: optically thin 1/r^2 flux, the Strömgren
radius (Eq. 17), mirror symmetry and the outer iteration (Sec. 2.6)."""
import json
import math
import os

import numpy as np
import pytest

from workloads import Workload, PC_CM, ALPHA_B, uniform_density, workload

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def test_stromgren_radius_formula():
    g = GOLD["stromgren_radius_pc"]
    i = g["inputs"]
    rs = (3 * i["Q"] / (4 * math.pi * i["n_H"] ** 2 * i["alpha_B"])) ** (1 / 3) / PC_CM
    assert rs == pytest.approx(g["value"], rel=g["rel_tol"])
    assert GOLD["alpha_B_cm3_s"]["value"] == ALPHA_B


def test_optically_thin_inverse_square(orc):
    """Negligible gas: F = Q / (4 pi d^2) exactly for every target, because the
    ray weights sum to one and W_f,3 keeps the flux at r = 0 exact (Eq. A6)."""
    N, box = 16, 4.0 * PC_CM
    dx = box / N
    src_cell = np.array([5, 9, 6])
    xyz = ((src_cell + 0.5) * dx)[None, :]
    w = Workload("thin", N, box, uniform_density(N, 1e-20), xyz, np.array([1e48]), theta_src=1e-3)
    t = orc.Tree(w)
    F, e, ion = t.solve_pass(orc.params_for(w, zeta_g=True))
    idx = np.arange(N ** 3)
    c = np.stack([idx % N, (idx // N) % N, idx // (N * N)], axis=1)
    d2 = (((c - src_cell) * dx) ** 2).sum(axis=1)
    s = np.ravel_multi_index(src_cell[::-1], (N, N, N))
    mask = idx != s
    np.testing.assert_allclose(F[mask], 1e48 / (4 * math.pi * d2[mask]), rtol=1e-9)
    assert F[s] == pytest.approx(1e48 / (4 * math.pi * (dx / 2) ** 2), rel=1e-9)
    np.testing.assert_allclose(e, F * w.hnu / 2.99792458e10, rtol=1e-15)
    assert ion.all()


@pytest.mark.slow
@pytest.mark.parametrize("zeta_g", [False, True])
def test_stromgren_front(orc, zeta_g):
    """Strömgren test (Sec. 3.1 set-up, static): the ionised volume's
    equivalent radius matches R_S (Eq. 17); with zeta_g the continuum
    prediction is R_S (1 - 2/N_side^3)^(-1/3).  The tolerance is the radial
    resolution of the rays there: half a segment of Eq. 4 at R_S (1.4 cells),
    never less than one cell."""
    w = workload("stromgren32", theta_src=1e-2)
    t = orc.Tree(w)
    F, e, ion = t.solve_pass(orc.params_for(w, zeta_g=zeta_g))
    rs0 = rs = (3 * 1e49 / (4 * math.pi * 100.0 ** 2 * ALPHA_B)) ** (1 / 3) / w.dx
    if zeta_g:
        rs *= (1 - 2 / w.nside ** 3) ** (-1 / 3)
    r_eff = (3 * ion.sum() / (4 * math.pi)) ** (1 / 3)
    i = math.sqrt(2 * w.eta_r ** 2 * rs)
    half_seg = 0.5 * (2 * i + 1) / (2 * w.eta_r ** 2)
    assert abs(r_eff - rs) < max(1.0, half_seg), (r_eff, rs, half_seg)
    # fully ionised well inside R_S, fully neutral outside 1.3 R_S.  Along
    # the axes the front is nearest: there the source sits on a corner of
    # four HEALPix pixels and is split between their rays
    N = w.N
    idx = np.arange(N ** 3)
    c = np.stack([idx % N, (idx // N) % N, idx // (N * N)], axis=1)
    r = np.sqrt(((c - 16) ** 2).sum(axis=1))
    assert ion[r < 0.6 * rs0].all()
    assert not ion[r > 1.3 * rs].any()


def test_mirror_symmetric_scene(orc):
    """Two sources placed mirror-symmetrically about the box centre in a
    mirror-symmetric medium give a mirror-symmetric field (cf. the x = y
    symmetry argument of the two-source test, Sec. 3.5)."""
    N, box = 16, 4.0 * PC_CM
    dx = box / N
    rng = np.random.default_rng(5)
    rho = 100.0 * np.exp(rng.normal(0, 0.5, (N, N, N)))
    rho = 0.5 * (rho + rho[:, :, ::-1])                 # symmetric under x -> N-1-x
    cells = np.array([[3, 7, 9], [12, 7, 9]])
    xyz = (cells + 0.5) * dx
    w = Workload("mirror", N, box, rho, xyz, np.array([3e47, 3e47]), theta_src=0.25)
    F, e, ion = orc.Tree(w).solve_pass(orc.params_for(w))
    Fc = F.reshape(N, N, N)
    np.testing.assert_allclose(Fc, Fc[:, :, ::-1], rtol=1e-9, atol=1e-12 * Fc.max())


def test_iteration_converges(orc):
    """Outer iteration (Sec. 2.6): delta_cell decreases below eps_lim within
    a few passes for a single source, where zeta_d ~ 1."""
    N, box = 16, 3.0 * PC_CM
    dx = box / N
    xyz = np.array([[8.5 * dx, 8.5 * dx, 8.5 * dx]])
    w = Workload("iter", N, box, uniform_density(N, 30.0), xyz, np.array([2e47]), theta_src=1e-2)
    p = orc.params_for(w)
    F1, e1, ion1, it1, d1 = orc.solve(w, p, max_iter=1)
    F, e, ion, iters, delta = orc.solve(w, p, max_iter=10, eps_lim=1e-2)
    assert it1 == 1 and math.isinf(d1)
    assert iters <= 10 and delta < 1e-2
    assert 0 < ion.sum() < N ** 3
    # delta_cell of a field against itself is zero; against zero it is infinite
    assert orc.delta(e, e) == 0.0
    assert math.isinf(orc.delta(e, np.zeros_like(e)))
    assert orc.delta(e * 1.5, e, mode=1) == pytest.approx(0.4)


@pytest.mark.parametrize("kernel_eps", [1, 2, 3])
def test_optically_thin_flux_kernels_agree(orc, kernel_eps):
    """In negligible gas every flux-conserving eps kernel (W_f,1, W_f,2,
    generalised W_f,3) delivers at the target exactly the flux of a point
    source at the node's mass centre (App. A.3), so all reproduce the W_f,3
    field cell by cell; with theta_src = inf the source is seen inside large
    nodes, where the generalised kernel spans many points."""
    N, box = 16, 4.0 * PC_CM
    dx = box / N
    src_cell = np.array([5, 9, 6])
    xyz = ((src_cell + 0.5) * dx)[None, :]
    w = Workload("thin", N, box, uniform_density(N, 1e-20), xyz, np.array([1e48]))
    t = orc.Tree(w)
    F, e, ion = t.solve_pass(orc.params_for(w, zeta_g=True, kernel_eps=kernel_eps))
    F_ref, _, _ = t.solve_pass(orc.params_for(w, zeta_g=True, kernel_eps=0))
    np.testing.assert_allclose(F, F_ref, rtol=1e-9)
    s = np.ravel_multi_index(src_cell[::-1], (N, N, N))
    assert F[s] == pytest.approx(1e48 / (4 * math.pi * (dx / 2) ** 2), rel=1e-9)


def test_stromgren_iteration_converges_to_rs(orc):
    """Outer iteration from a cold start (Sec. 2.6): a single source in a
    uniform 16^3 medium converges (delta_cell < 1e-2) in fewer than 10
    passes, with the ionised volume's equivalent radius at R_S (Eq. 17,
    zeta_g off) within the radial resolution of the rays there."""
    N, box = 16, 4.0 * PC_CM
    dx = box / N
    n, Q = 100.0, 3.3e47
    w = Workload("s16", N, box, uniform_density(N, n), np.array([[8.5 * dx] * 3]), np.array([Q]), theta_src=1e-2)
    F, e, ion, iters, delta = orc.solve(w, orc.params_for(w, zeta_g=False), max_iter=10, eps_lim=1e-2)
    assert iters < 10 and delta < 1e-2
    rs = (3 * Q / (4 * math.pi * n ** 2 * ALPHA_B)) ** (1 / 3) / dx
    r_eff = (3 * ion.sum() / (4 * math.pi)) ** (1 / 3)
    i = math.sqrt(2 * w.eta_r ** 2 * rs)
    half_seg = 0.5 * (2 * i + 1) / (2 * w.eta_r ** 2)
    assert abs(r_eff - rs) < max(1.0, half_seg), (r_eff, rs)
