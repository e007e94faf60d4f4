"""Parity of the column-density maps (cdMaps) between the CUDA path and the
oracle: within 1e-12 in FP64 and 1e-5 in the FP32 form (FP32 node moments
and distances), on uniform and AMR grids, with every boundary."""
import numpy as np
import pytest

from test_gpu_amr import gpu_amr_tree, small_amr
from test_gpu_parity import B, dev, gpu_tree, small_turbulent  # noqa: F401

pytestmark = pytest.mark.gpu

RTOL_CD = {0: 1e-12, 1: 1e-5}


def gpu_cd(B, tree, targets=None, n=None):
    import torch
    npix = tree.info()["npix"]
    rows = n if targets is None else len(targets)
    out = torch.empty((rows, npix), dtype=torch.float64, device="cuda")
    B.tr_column_density(tree, out, None if targets is None else dev(np.asarray(targets, dtype=np.int64)))
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("nside,bc", [(2, 0), (1, 0), (4, 0), (2, 1), (2, 2)])
def test_cd_uniform(B, orc, precision, nside, bc):
    w = small_turbulent(N=32, theta_lim=0.5)
    w.nside = nside
    t = gpu_tree(B, w, precision, bc=bc)
    rng = np.random.default_rng(61)
    targets = np.unique(np.concatenate([rng.integers(0, w.N ** 3, 40), [0, w.N ** 3 - 1]]))
    cd = gpu_cd(B, t, targets)
    ot = orc.Tree(w)
    p = orc.params_for(w, bc=bc)
    for k, tgt in enumerate(targets):
        want = ot.column_density(p, int(tgt))
        np.testing.assert_allclose(cd[k], want, rtol=RTOL_CD[precision], atol=RTOL_CD[precision] * want.max())


def test_cd_all_cells_rows(B, orc):
    """targets = NULL: row c is cell c."""
    w = small_turbulent(N=16)
    t = gpu_tree(B, w, 0)
    cd = gpu_cd(B, t, None, n=w.N ** 3)
    ot = orc.Tree(w)
    p = orc.params_for(w)
    for tgt in (0, 1234, w.N ** 3 - 1):
        np.testing.assert_allclose(cd[tgt], ot.column_density(p, tgt), rtol=1e-12)


@pytest.mark.parametrize("precision", [0, 1])
def test_cd_amr(B, orc, precision):
    g = small_amr()
    t = gpu_amr_tree(B, g, precision)
    rng = np.random.default_rng(62)
    targets = np.unique(rng.integers(0, g.n_leaves, 30))
    cd = gpu_cd(B, t, targets)
    ot = orc.AmrTree(g)
    p = orc.params_for(g)
    for k, tgt in enumerate(targets):
        want = ot.column_density(p, int(tgt))
        np.testing.assert_allclose(cd[k], want, rtol=RTOL_CD[precision], atol=RTOL_CD[precision] * want.max())
