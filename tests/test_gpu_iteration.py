"""The outer iteration (Sec. 2.6, Eq. 19-21) on the GPU against the oracle."""
import math

import numpy as np
import pytest

from helpers import KAPPA, flux_misses, interior_mask
from workloads import Workload, PC_CM, lognormal_density, uniform_density, uniform_sources

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    import torch
    import paper_2105_09644_gb300 as pkg
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    pkg.build()
    from paper_2105_09644_gb300 import binding
    binding.load()
    return binding


def dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("mode", [0, 1])
def test_delta_matches_oracle(B, orc, mode):
    rng = np.random.default_rng(5)
    for n in (1, 2, 7, 1000, 4097):
        old = rng.uniform(0, 1e-9, n) * (rng.random(n) < 0.6)
        new = old * rng.uniform(0.5, 1.5, n) + 1e-12 * (rng.random(n) < 0.1)
        want = orc.delta(new, old, mode)
        got = B.tr_delta(dev(new), dev(old), mode)
        assert got == pytest.approx(want, rel=1e-12, abs=0) or (math.isinf(got) and math.isinf(want))
    z = np.zeros(10)
    assert B.tr_delta(dev(z), dev(z), mode) == 0.0
    if mode == 0:
        assert math.isinf(B.tr_delta(dev(z + 1e-12), dev(z), mode))


def small(N=16, seed=21, **kw):
    box = 3.0 * PC_CM
    rho = lognormal_density(N, seed, sigma_ln=0.8, mean_nH=30.0)
    xyz, q = uniform_sources(3, box, seed + 1, 46.5, 47.5)
    return Workload(f"iter{N}", N, box, rho, xyz, q, seed=seed, theta_src=0.3, theta_if=0.3)


def gpu_iterate(B, w, precision, max_iter, eps_lim, e_init=None):
    import torch
    F, e, ion, it, dl = B.solve(dev(w.n_H), w.dx, dev(w.src_xyz), dev(w.src_Q),
                                e_prev=None if e_init is None else dev(e_init.reshape(w.N, w.N, w.N)),
                                theta_src=w.theta_src, theta_if=w.theta_if, precision=precision,
                                max_iter=max_iter, eps_lim=eps_lim)
    torch.cuda.synchronize()
    return F.cpu().numpy().ravel(), e.cpu().numpy().ravel(), ion.cpu().numpy().ravel(), it, dl


@pytest.mark.parametrize("precision,rtol", [(0, 1e-5), (1, 1e-3), (2, 1e-3)])
def test_fixed_passes_match_oracle(B, orc, precision, rtol):
    """Four passes (eps_lim = 0 never stops early): IF MAC and zeta_d are live
    from the second pass on.  Every cell away from the front meets the bar
    (the FP32 forms decide the IF MAC on the FP64 masses)."""
    w = small()
    F, e, ion, it, dl = gpu_iterate(B, w, precision, 4, 0.0)
    Fo, eo, iono, ito, dlo = orc.solve(w, orc.params_for(w), max_iter=4, eps_lim=0.0)
    assert it == ito == 4
    inner = interior_mask(iono.reshape(w.N, w.N, w.N)).ravel()
    assert np.array_equal(ion[inner], iono[inner])
    lit = np.nonzero(inner & (Fo > 0))[0]

    def free(k):                     # the last pass's tree: built with the third pass's e
        e3 = orc.solve(w, orc.params_for(w), max_iter=3, eps_lim=0.0)[1]
        return orc.Tree(w, e_prev=e3).free_flux(orc.params_for(w), targets=lit[k])
    miss = flux_misses(F[lit], Fo[lit], rtol, KAPPA[precision], free)
    assert miss.size == 0, np.sort(np.abs(F[lit] - Fo[lit]) / Fo[lit])[-5:]
    assert np.all(F[inner & (Fo == 0)] == 0.0)
    assert dl == pytest.approx(dlo, rel=1e-3 if precision else 1e-6)


def test_converges_like_oracle(B, orc):
    """A single source in a uniform medium converges (zeta_d ~ 1) within a
    few passes, the same number on both sides."""
    N, box = 16, 3.0 * PC_CM
    dx = box / N
    w = Workload("conv", N, box, uniform_density(N, 30.0), np.array([[8.5 * dx] * 3]), np.array([2e47]),
                 theta_src=1e-2)
    F, e, ion, it, dl = gpu_iterate(B, w, 0, 10, 1e-2)
    Fo, eo, iono, ito, dlo = orc.solve(w, orc.params_for(w), max_iter=10, eps_lim=1e-2)
    assert it == ito and dl < 1e-2 and dlo < 1e-2
    np.testing.assert_allclose(e[iono > 0], eo[iono > 0], rtol=1e-5)


def test_warm_start_one_pass_reports_delta(B, orc):
    w = small()
    Fo, eo, iono, _, _ = orc.solve(w, orc.params_for(w), max_iter=1)
    F, e, ion, it, dl = gpu_iterate(B, w, 0, 1, 1e-2, e_init=eo)
    F2, e2, ion2 = orc.Tree(w, e_prev=eo).solve_pass(orc.params_for(w))
    assert it == 1
    assert dl == pytest.approx(orc.delta(e2, eo), rel=1e-6)
