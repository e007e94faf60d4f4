"""Host-side argument checks of the C ABI, run without a GPU: every call
below is rejected before the library touches a device, so the placeholder
pointers it is given are never dereferenced (on a GPU machine as well)."""
import ctypes as C

import numpy as np
import pytest

FAKE = 0x1000                    # a non-NULL device address that is never used


@pytest.fixture(scope="module")
def B():
    import paper_2105_09644_gb300 as pkg
    from paper_2105_09644_gb300 import binding
    pkg.build()
    binding.load()
    return binding


def build_status(B, grid, params):
    tree = C.c_void_p()
    rc = B.load().tr_build_tree(C.byref(grid), C.byref(B.Sources(0, None, None)), C.byref(params), C.byref(tree), None)
    return rc, B.load().tr_last_error().decode()


def test_defaults_include_kernels_and_boundaries(B):
    p = B.tr_params_default()
    assert p.kernel_alpha == B.TR_KERNEL_WP and p.kernel_eps == B.TR_EPS_WF3 and p.bc == B.TR_BC_ISOLATED
    assert p.precision == B.TR_FP64 and p.zeta_g == 1 and p.delta_mode == 0


@pytest.mark.parametrize("field,value,word", [("nside", 3, "nside"), ("eta_r", 3, "eta_r"), ("precision", 3, "precision"),
                                              ("kernel_alpha", 2, "kernel_alpha"), ("kernel_eps", 6, "kernel_eps"),
                                              ("bc", 3, "bc"), ("theta_lim", 0.0, "opening"), ("max_iter", 0, "max_iter"),
                                              ("alpha_B", -1.0, "alpha_B")])
def test_bad_parameters_are_rejected(B, field, value, word):
    p = B.tr_params_default()
    setattr(p, field, value)
    g = B.Grid(16, (C.c_double * 3)(0, 0, 0), 1e18, FAKE, None, None)
    rc, msg = build_status(B, g, p)
    assert rc == B.TR_EINVAL and word in msg


@pytest.mark.parametrize("N,dx,nH,word", [(12, 1e18, FAKE, "power of two"), (1024, 1e18, FAKE, "power of two"),
                                          (16, 0.0, FAKE, "dx"), (16, 1e18, None, "n_H")])
def test_bad_grids_are_rejected(B, N, dx, nH, word):
    g = B.Grid(N, (C.c_double * 3)(0, 0, 0), dx, nH, None, None)
    rc, msg = build_status(B, g, B.tr_params_default())
    assert rc == B.TR_EINVAL and word in msg


def amr_status(B, N_base, max_level, lev, pos):
    lev = np.ascontiguousarray(lev, dtype=np.int32)
    pos = np.ascontiguousarray(pos, dtype=np.int32).reshape(-1)
    g = B.AmrGrid(N_base, max_level, int(lev.shape[0]), lev.ctypes.data, pos.ctypes.data,
                  (C.c_double * 3)(0, 0, 0), 1e18, FAKE, None, None)
    tree = C.c_void_p()
    rc = B.load().tr_build_tree_amr(C.byref(g), C.byref(B.Sources(0, None, None)), C.byref(B.tr_params_default()),
                                    C.byref(tree), None)
    return rc, B.load().tr_last_error().decode()


def refined_layout():
    """base 16^3 (2^3 blocks), block (0,0,0) refined once: 7 + 8 blocks"""
    lev, pos = [], []
    for z in range(2):
        for y in range(2):
            for x in range(2):
                if (x, y, z) == (0, 0, 0):
                    continue
                lev.append(0); pos.append((x, y, z))
    for c in range(8):
        lev.append(1); pos.append((c & 1, (c >> 1) & 1, c >> 2))
    return np.array(lev), np.array(pos)


def test_amr_layout_checks(B):
    lev, pos = refined_layout()
    # (the valid layout itself is not built here: that would read the fake n_H)
    rc, msg = amr_status(B, 16, 1, lev[1:], pos[1:])                  # a gap
    assert rc == B.TR_EINVAL and "fill" in msg
    rc, msg = amr_status(B, 16, 1, np.append(lev, 0), np.vstack([pos, [0, 0, 0]]))   # a block over refined ones
    assert rc == B.TR_EINVAL and ("inside" in msg or "repeats" in msg)
    rc, msg = amr_status(B, 16, 1, np.append(lev[:-1], 1), np.vstack([pos[:-1], pos[-2]]))  # a repeated block
    assert rc == B.TR_EINVAL and "repeats" in msg
    bad = pos.copy(); bad[0] = (5, 0, 0)
    rc, msg = amr_status(B, 16, 1, lev, bad)                            # out of the box
    assert rc == B.TR_EINVAL and "position" in msg
    rc, msg = amr_status(B, 12, 1, lev, pos)                            # base not a power of two
    assert rc == B.TR_EINVAL and "N_base" in msg


def test_null_handles_are_rejected(B):
    L = B.load()
    assert L.tr_walk_sweep(None, None, None, None, None) == B.TR_EINVAL
    assert L.tr_column_density(None, None, 0, None, None) == B.TR_EINVAL
    assert L.tr_tree_cells(None, None) == B.TR_EINVAL
    out = C.c_double()
    assert L.tr_delta(None, None, 0, 0, C.byref(out), None) == B.TR_EINVAL
