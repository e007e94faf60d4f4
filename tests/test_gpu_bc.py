"""Parity of the walk's boundary conditions (Sec. 2.8) between the CUDA
path and the oracle: periodic (nearest copy) and corner of symmetry (the
original and its 7 mirror images), on uniform and AMR grids.  Bars as for
isolated boundaries: accepted-node lists bit-exact and bins within 1e-12
in FP64; flux within 1e-5 (FP64) / 1e-3 (FP32 form) away from the front."""
import numpy as np
import pytest

from test_gpu_amr import compare_amr, gpu_amr_solve, small_amr
from helpers import KAPPA
from test_gpu_parity import B, RTOL, compare_fields, dev, gpu_solve, gpu_tree, small_turbulent  # noqa: F401

pytestmark = pytest.mark.gpu

BCS = [1, 2]          # TR_BC_PERIODIC, TR_BC_CORNER


@pytest.mark.parametrize("bc", BCS)
def test_bc_walk_lists_and_bins_fp64(B, orc, bc):
    import torch
    w = small_turbulent(N=16, n_src=5, theta_src=0.4)
    t = gpu_tree(B, w, 0, bc=bc)
    rng = np.random.default_rng(31)
    targets = np.unique(np.concatenate([rng.integers(0, w.N ** 3, 24), [0, w.N ** 3 - 1]])).astype(np.int64)
    r = B.tr_walk_map(t, dev(targets))
    info = r.info()
    nt, npix, nr, cap = info["n_targets"], info["npix"], info["nr"], info["acc_cap"]
    a = torch.empty((nt, npix, nr), dtype=torch.float64, device="cuda")
    e = torch.empty_like(a)
    ids = torch.empty((nt, cap), dtype=torch.int64, device="cuda")
    counts = torch.empty(nt, dtype=torch.int32, device="cuda")
    B.tr_rays_export(r, a, e, None, ids, counts)
    torch.cuda.synchronize()
    a, e, ids, counts = a.cpu().numpy(), e.cpu().numpy(), ids.cpu().numpy(), counts.cpu().numpy()
    ot = orc.Tree(w)
    p = orc.params_for(w, bc=bc)
    for k, tgt in enumerate(targets):
        res = ot.walk(p, int(tgt))
        assert counts[k] == res["n_accepted"]
        assert np.array_equal(np.sort(ids[k, :counts[k]]), np.sort(res["accepted"]))
        np.testing.assert_allclose(a[k], res["alpha"], rtol=1e-12, atol=1e-12 * max(res["alpha"].max(), 1e-300))
        np.testing.assert_allclose(e[k], res["eps"], rtol=1e-12, atol=1e-12 * max(res["eps"].max(), 1e-300))


@pytest.mark.parametrize("precision", [0, 1, 2])
@pytest.mark.parametrize("bc", BCS)
def test_bc_solve(B, orc, bc, precision):
    w = small_turbulent(N=32, theta_src=0.4)
    F, e, ion = gpu_solve(B, w, precision, bc=bc)
    ot, p = orc.Tree(w), orc.params_for(w, bc=bc)
    F_orc, _, ion_orc = ot.solve_pass(p)
    compare_fields(F, ion, F_orc, ion_orc, w.N, RTOL[precision], KAPPA[precision],
                   lambda c: ot.free_flux(p, targets=c))


@pytest.mark.parametrize("bc", BCS)
def test_bc_amr(B, orc, bc):
    g = small_amr()
    F, e, ion = gpu_amr_solve(B, g, 0, bc=bc)
    F_orc, _, ion_orc = orc.AmrTree(g).solve_pass(orc.params_for(g, bc=bc))
    compare_amr(g, F, ion, F_orc, ion_orc, RTOL[0])


def test_bc_is_checked(B):
    import torch
    n = torch.ones((16, 16, 16), dtype=torch.float64, device="cuda")
    with pytest.raises(B.TreeRayError) as ei:
        B.solve(n, 1e18, bc=3)
    assert ei.value.status == B.TR_EINVAL
