"""The allocation-free entry point, tr_solve_noalloc.

It exists for callers that cannot call cudaMalloc: hosts whose device memory
belongs to a pool or arena that forbids outside allocations, and real-time
hosts that must not allocate (cudaMalloc may block and synchronise the
device) once running.  Its working memory is a fixed array inside the
library.  These tests call it through the C ABI twice in a row and check
each result against tr_solve's on the same input, with the parity
tolerances used elsewhere in the suite; they also check that the device's
free memory does not change across the calls, and that requests beyond the
fixed array are refused.  The file sorts last so that a run stopping at its
first failure has already run every other test.
"""
import numpy as np
import pytest

from helpers import interior_mask
from workloads import Workload, PC_CM, lognormal_density, uniform_sources

pytestmark = pytest.mark.gpu

RTOL = {0: 1e-5, 1: 1e-3, 2: 1e-3}


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


class Call:
    """Inputs and outputs of one call, allocated up front (torch), so that
    the calls themselves are the only GPU work between the memory checks."""

    def __init__(self, B, w, precision, **over):
        import torch
        self.w = w
        self.keep = [torch.from_numpy(a).cuda() for a in (w.n_H, w.src_xyz, w.src_Q)]
        self.g = B.make_grid(self.keep[0], w.dx)
        self.s = B.make_sources(self.keep[1], self.keep[2])
        self.p = B.tr_params_default(theta_src=w.theta_src, precision=precision, **over)
        self.F = torch.empty((w.N,) * 3, dtype=torch.float64, device="cuda")
        self.e = torch.empty_like(self.F)
        self.ion = torch.empty((w.N,) * 3, dtype=torch.uint8, device="cuda")

    def __call__(self, fn):
        import torch
        fn(self.g, self.s, self.p, self.F, self.e, self.ion)
        torch.cuda.synchronize()
        return (self.F.cpu().numpy().ravel(), self.e.cpu().numpy().ravel(), self.ion.cpu().numpy().ravel())


def same(out, ref, N, rtol):
    F, e, ion = out
    F_ref, e_ref, ion_ref = ref
    inner = interior_mask(ion_ref.reshape(N, N, N)).ravel()
    assert np.array_equal(ion[inner], ion_ref[inner])
    for a, b in ((F, F_ref), (e, e_ref)):
        lit = inner & (b > 0)
        assert np.all(np.abs(a[lit] - b[lit]) <= rtol * b[lit])
        assert np.all(a[inner & (b == 0)] == 0.0)


@pytest.mark.parametrize("precision", [0, 1, 2])
def test_matches_tr_solve_on_two_calls_in_a_row(B, precision):
    import torch
    calls = [Call(B, case(seed), precision) for seed in (31, 32)]      # different inputs, shared scratch
    refs = [c(B.tr_solve) for c in calls]
    calls[0](B.tr_solve_noalloc)                                     # the first call on the device sets up
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    outs = [c(B.tr_solve_noalloc) for c in calls]
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, f"device free memory changed by {free0 - free1} bytes across the calls"
    for c, out, ref in zip(calls, outs, refs):
        same(out, ref, c.w.N, RTOL[precision])


def test_rejects_sizes_beyond_its_scratch(B):
    with pytest.raises(B.TreeRayError) as ei:
        Call(B, case(33, N=64), 1)(B.tr_solve_noalloc)
    assert ei.value.status == B.TR_EUNSUPPORTED and "32" in str(ei.value)
    with pytest.raises(B.TreeRayError) as ei:
        Call(B, case(34), 1, nside=4)(B.tr_solve_noalloc)
    assert ei.value.status == B.TR_EUNSUPPORTED and "N_side" in str(ei.value)


def test_checks_arguments_like_tr_solve(B):
    """A non-finite box corner or alpha_B is refused as tr_solve refuses it."""
    c = Call(B, case(35), 1)
    c.g.box_lo[0] = float("nan")
    with pytest.raises(B.TreeRayError) as ei:
        c(B.tr_solve_noalloc)
    assert ei.value.status == B.TR_EINVAL
    c = Call(B, case(35), 1, alpha_B=float("inf"))
    with pytest.raises(B.TreeRayError) as ei:
        c(B.tr_solve_noalloc)
    assert ei.value.status == B.TR_EINVAL
