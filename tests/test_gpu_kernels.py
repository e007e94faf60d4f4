"""Parity of the radial kernel choices (App. A) between the CUDA path and
the oracle: W_p / W_g for alpha and e; W_f,3, W_f,1, W_f,2, generalised
W_f,3, W_p, W_g for eps.  Same bars as the default kernels: ray bins within
1e-12 in FP64, cell flux within 1e-5 (FP64) / 1e-3 (FP32 forms) away from
the ionisation front."""
import numpy as np
import pytest

from helpers import KAPPA
from test_gpu_parity import B, RTOL, compare_fields, dev, gpu_solve, gpu_tree, small_turbulent  # noqa: F401

pytestmark = pytest.mark.gpu

COMBOS = [(0, 1), (0, 2), (0, 3), (0, 4), (0, 5), (1, 0), (1, 3)]


@pytest.mark.parametrize("kernel_alpha,kernel_eps", COMBOS)
def test_kernel_bins_fp64(B, orc, kernel_alpha, kernel_eps):
    import torch
    w = small_turbulent(N=16, n_src=6, theta_src=0.6)
    kw = dict(kernel_alpha=kernel_alpha, kernel_eps=kernel_eps)
    t = gpu_tree(B, w, 0, **kw)
    rng = np.random.default_rng(21)
    targets = np.unique(rng.integers(0, w.N ** 3, 24)).astype(np.int64)
    r = B.tr_walk_map(t, dev(targets))
    info = r.info()
    nt, npix, nr = info["n_targets"], info["npix"], info["nr"]
    a = torch.empty((nt, npix, nr), dtype=torch.float64, device="cuda")
    e = torch.empty_like(a)
    B.tr_rays_export(r, a, e)
    torch.cuda.synchronize()
    a, e = a.cpu().numpy(), e.cpu().numpy()
    ot = orc.Tree(w)
    p = orc.params_for(w, **kw)
    for k, tgt in enumerate(targets):
        res = ot.walk(p, int(tgt))
        np.testing.assert_allclose(a[k], res["alpha"], rtol=1e-12, atol=1e-12 * max(res["alpha"].max(), 1e-300))
        np.testing.assert_allclose(e[k], res["eps"], rtol=1e-12, atol=1e-12 * max(res["eps"].max(), 1e-300))


@pytest.mark.parametrize("precision", [0, 1, 2])
@pytest.mark.parametrize("kernel_alpha,kernel_eps", COMBOS)
def test_kernel_solve(B, orc, precision, kernel_alpha, kernel_eps):
    """Every kernel choice in every form against the oracle, no cell exempt
    but the front band: the FP32 forms take their opening decisions, and the
    choices of the radial spreading that jump with the distance, in FP64
    where FP32 cannot settle them."""
    w = small_turbulent(N=32, theta_src=0.6)
    kw = dict(kernel_alpha=kernel_alpha, kernel_eps=kernel_eps)
    F, e, ion = gpu_solve(B, w, precision, **kw)
    ot, p = orc.Tree(w), orc.params_for(w, **kw)
    F_orc, _, ion_orc = ot.solve_pass(p)
    compare_fields(F, ion, F_orc, ion_orc, w.N, RTOL[precision], KAPPA[precision],
                   lambda c: ot.free_flux(p, targets=c))


def test_kernel_choice_is_checked(B):
    import torch
    n = torch.ones((16, 16, 16), dtype=torch.float64, device="cuda")
    for bad in (dict(kernel_alpha=2), dict(kernel_eps=6), dict(kernel_eps=-1)):
        with pytest.raises(B.TreeRayError) as ei:
            B.solve(n, 1e18, **bad)
        assert ei.value.status == B.TR_EINVAL
