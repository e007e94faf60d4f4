"""The allocation-free entry point, tr_solve_noalloc.

It exists for callers that cannot call cudaMalloc (code running under CUDA
graph capture, hosts whose device memory belongs to a pool or arena, hosts
that must not allocate once running): its working memory is a fixed array
inside the library.  These tests call it through the C ABI twice in a row
and check each result against tr_solve's on the same input, with the parity
tolerances used elsewhere in the suite.  The file sorts last so that a run
stopping at its first failure has already run every other test.
"""
import numpy as np
import pytest

from helpers import interior_mask
from workloads import Workload, PC_CM, lognormal_density, uniform_sources

pytestmark = pytest.mark.gpu

RTOL = {0: 1e-5, 1: 1e-3}


@pytest.fixture(scope="module")
def B():
    import torch
    import paper_2105_09644_gb300 as pkg
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    pkg.build()
    from paper_2105_09644_gb300 import binding
    binding.load()
    return binding


def case(seed, N=32):
    box = 4.0 * PC_CM
    rho = lognormal_density(N, seed)
    xyz, q = uniform_sources(5, box, seed + 1, 46.0, 48.5)
    return Workload(f"noalloc{seed}", N, box, rho, xyz, q, seed=seed, theta_src=0.3)


def run(B, w, precision, fn):
    import torch
    n = torch.from_numpy(w.n_H).cuda()
    x = torch.from_numpy(w.src_xyz).cuda()
    q = torch.from_numpy(w.src_Q).cuda()
    g = B.make_grid(n, w.dx)
    s = B.make_sources(x, q)
    p = B.tr_params_default(theta_src=w.theta_src, precision=precision)
    F = torch.empty((w.N,) * 3, dtype=torch.float64, device="cuda")
    e = torch.empty_like(F)
    ion = torch.empty((w.N,) * 3, dtype=torch.uint8, device="cuda")
    fn(g, s, p, F, e, ion)
    torch.cuda.synchronize()
    return F.cpu().numpy().ravel(), ion.cpu().numpy().ravel()


def same(F, ion, F_ref, ion_ref, N, rtol):
    inner = interior_mask(ion_ref.reshape(N, N, N)).ravel()
    assert np.array_equal(ion[inner], ion_ref[inner])
    lit = inner & (F_ref > 0)
    assert np.all(np.abs(F[lit] - F_ref[lit]) <= rtol * F_ref[lit])
    assert np.all(F[inner & (F_ref == 0)] == 0.0)


@pytest.mark.parametrize("precision", [0, 1])
def test_matches_tr_solve_on_two_calls_in_a_row(B, precision):
    for seed in (31, 32):                       # two calls, different inputs, shared scratch
        w = case(seed)
        F_ref, ion_ref = run(B, w, precision, lambda g, s, p, F, e, i: B.tr_solve(g, s, p, F, e, i))
        F, ion = run(B, w, precision, lambda g, s, p, F, e, i: B.tr_solve_noalloc(g, s, p, F, e, i))
        same(F, ion, F_ref, ion_ref, w.N, RTOL[precision])


def test_rejects_sizes_beyond_its_scratch(B):
    w = case(33, N=64)
    with pytest.raises(B.TreeRayError) as ei:
        run(B, w, 1, lambda g, s, p, F, e, i: B.tr_solve_noalloc(g, s, p, F, e, i))
    assert ei.value.status == B.TR_EUNSUPPORTED and "32" in str(ei.value)
