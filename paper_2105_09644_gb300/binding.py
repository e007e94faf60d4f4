"""ctypes binding of libtreeray.so (include/treeray.h), argument marshalling only.

Every step of the method runs in the library's CUDA kernels; this module
only converts torch tensors to device pointers and checks return codes.
There is no CPU fallback: if the library is missing, importing the binding
raises.
"""
from __future__ import annotations

import ctypes as C
import math
import os

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libtreeray.so")

TR_OK, TR_EINVAL, TR_ENOMEM, TR_ECUDA, TR_ETIMEOUT, TR_EUNSUPPORTED, TR_EOVERFLOW = range(7)
TR_FP64, TR_FP32_SWEEP64, TR_FP32_SWEEPDF = 0, 1, 2
PRECISIONS = (TR_FP64, TR_FP32_SWEEP64, TR_FP32_SWEEPDF)
TR_KERNEL_WP, TR_KERNEL_WG = 0, 1
TR_EPS_WF3, TR_EPS_WF1, TR_EPS_WF2, TR_EPS_WF3N, TR_EPS_WP, TR_EPS_WG = range(6)
TR_BC_ISOLATED, TR_BC_PERIODIC, TR_BC_CORNER = 0, 1, 2
STATUS_NAMES = {0: "TR_OK", 1: "TR_EINVAL", 2: "TR_ENOMEM", 3: "TR_ECUDA", 4: "TR_ETIMEOUT",
                5: "TR_EUNSUPPORTED", 6: "TR_EOVERFLOW"}

# every symbol include/treeray.h declares
EXPORTED = ["tr_params_default", "tr_build_tree", "tr_build_tree_amr", "tr_tree_cells", "tr_tree_flags",
            "tr_walk_map", "tr_ray_sweep", "tr_walk_sweep", "tr_solve", "tr_column_density",
            "tr_tree_stats", "tr_solve_noalloc", "tr_delta", "tr_walk_sweep_batch",
            "tr_tree_info", "tr_tree_nodes", "tr_rays_info", "tr_rays_export", "tr_table_info",
            "tr_table_export", "tr_tree_free", "tr_rays_free", "tr_last_error"]


class TreeRayError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class Params(C.Structure):
    _fields_ = [("theta_lim", C.c_double), ("theta_if", C.c_double), ("theta_src", C.c_double),
                ("nside", C.c_int32), ("eta_r", C.c_int32), ("L_ray_cm", C.c_double),
                ("alpha_B", C.c_double), ("hnu", C.c_double), ("eps_lim", C.c_double),
                ("delta_mode", C.c_int32), ("max_iter", C.c_int32), ("precision", C.c_int32),
                ("zeta_g", C.c_int32), ("kernel_alpha", C.c_int32), ("kernel_eps", C.c_int32),
                ("bc", C.c_int32)]


class Grid(C.Structure):
    _fields_ = [("N", C.c_int32), ("box_lo", C.c_double * 3), ("dx", C.c_double),
                ("n_H", C.c_void_p), ("ndot", C.c_void_p), ("e_prev", C.c_void_p)]


class AmrGrid(C.Structure):
    _fields_ = [("N_base", C.c_int32), ("max_level", C.c_int32), ("n_blocks", C.c_int32),
                ("blk_level", C.c_void_p), ("blk_pos", C.c_void_p), ("box_lo", C.c_double * 3),
                ("dx_fine", C.c_double), ("n_H", C.c_void_p), ("ndot", C.c_void_p), ("e_prev", C.c_void_p)]


class Sources(C.Structure):
    _fields_ = [("n", C.c_int32), ("xyz", C.c_void_p), ("Q", C.c_void_p)]


_lib = None


def load():
    """Load libtreeray.so; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with __graft_entry__.build() "
                          "(there is no CPU fallback)")
    L = C.CDLL(LIB_PATH)
    vp, i64, i32 = C.c_void_p, C.c_int64, C.c_int32
    L.tr_params_default.argtypes = [C.POINTER(Params)]
    L.tr_params_default.restype = None
    L.tr_build_tree.argtypes = [C.POINTER(Grid), C.POINTER(Sources), C.POINTER(Params), C.POINTER(vp), vp]
    L.tr_build_tree_amr.argtypes = [C.POINTER(AmrGrid), C.POINTER(Sources), C.POINTER(Params), C.POINTER(vp), vp]
    L.tr_tree_cells.argtypes = [vp, C.POINTER(i64)]
    L.tr_tree_flags.argtypes = [vp, vp, vp]
    L.tr_walk_map.argtypes = [vp, vp, i64, C.POINTER(vp), vp]
    L.tr_column_density.argtypes = [vp, vp, i64, vp, vp]
    L.tr_ray_sweep.argtypes = [vp, vp, vp, vp, vp]
    L.tr_walk_sweep.argtypes = [vp, vp, vp, vp, vp]
    L.tr_tree_stats.argtypes = [vp, C.POINTER(i64)]
    L.tr_walk_sweep_batch.argtypes = [C.POINTER(vp), C.POINTER(i64), C.POINTER(i64), i32, C.POINTER(vp),
                                      C.POINTER(vp), C.POINTER(vp), vp]
    L.tr_delta.argtypes = [vp, vp, i64, i32, C.POINTER(C.c_double), vp]
    L.tr_solve_noalloc.argtypes = [C.POINTER(Grid), C.POINTER(Sources), C.POINTER(Params), vp, vp, vp, vp]
    L.tr_solve.argtypes = [C.POINTER(Grid), C.POINTER(Sources), C.POINTER(Params), vp, vp, vp,
                           C.POINTER(i32), C.POINTER(C.c_double), vp]
    L.tr_tree_info.argtypes = [vp, C.POINTER(i64), C.POINTER(i32), C.POINTER(i32), C.POINTER(i32)]
    L.tr_tree_nodes.argtypes = [vp, vp, vp]
    L.tr_rays_info.argtypes = [vp, C.POINTER(i64), C.POINTER(i32), C.POINTER(i32), C.POINTER(i32)]
    L.tr_rays_export.argtypes = [vp, vp, vp, vp, vp, vp, vp]
    L.tr_table_info.argtypes = [i32, C.POINTER(i32), C.POINTER(i32)]
    L.tr_table_export.argtypes = [i32, vp, vp, vp, vp]
    L.tr_tree_free.argtypes = [vp]
    L.tr_tree_free.restype = None
    L.tr_rays_free.argtypes = [vp]
    L.tr_rays_free.restype = None
    L.tr_last_error.restype = C.c_char_p
    for name in EXPORTED:
        if name not in ("tr_params_default", "tr_tree_free", "tr_rays_free", "tr_last_error"):
            getattr(L, name).restype = C.c_int
    _lib = L
    return L


def check(status: int):
    if status != TR_OK:
        raise TreeRayError(status, load().tr_last_error().decode())


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


# ---- the C-ABI calls, same names -------------------------------------------

def tr_params_default(**overrides) -> Params:
    p = Params()
    load().tr_params_default(C.byref(p))
    for k, v in overrides.items():
        setattr(p, k, v)
    return p


def make_grid(n_H, dx: float, box_lo=(0.0, 0.0, 0.0), ndot=None, e_prev=None) -> Grid:
    """Grid over device float64 tensors of shape (N, N, N)."""
    N = int(n_H.shape[0])
    for t in (n_H, ndot, e_prev):
        if t is not None:
            assert t.is_cuda and t.dtype.is_floating_point and t.element_size() == 8 and t.is_contiguous()
            assert tuple(t.shape) == (N, N, N)
    return Grid(N, (C.c_double * 3)(*box_lo), float(dx), n_H.data_ptr(),
                None if ndot is None else ndot.data_ptr(), None if e_prev is None else e_prev.data_ptr())


def make_amr_grid(N_base: int, max_level: int, blk_level, blk_pos, n_H, dx_fine: float, box_lo=(0.0, 0.0, 0.0),
                  ndot=None, e_prev=None):
    """AMR grid: blk_level (B,) and blk_pos (B, 3) host integer arrays, cell
    arrays device float64 tensors of B x 512 values.  Returns the struct and
    the host arrays it points to (keep both alive for the call)."""
    import numpy as np
    lev = np.ascontiguousarray(blk_level, dtype=np.int32)
    pos = np.ascontiguousarray(blk_pos, dtype=np.int32).reshape(-1)
    B = int(lev.shape[0])
    assert pos.shape[0] == 3 * B
    for t in (n_H, ndot, e_prev):
        if t is not None:
            assert t.is_cuda and t.dtype.is_floating_point and t.element_size() == 8 and t.is_contiguous()
            assert t.numel() == B * 512
    g = AmrGrid(int(N_base), int(max_level), B, lev.ctypes.data, pos.ctypes.data, (C.c_double * 3)(*box_lo),
                float(dx_fine), n_H.data_ptr(), None if ndot is None else ndot.data_ptr(),
                None if e_prev is None else e_prev.data_ptr())
    return g, (lev, pos)


def make_sources(xyz=None, Q=None) -> Sources:
    if xyz is None or Q is None or Q.numel() == 0:
        return Sources(0, None, None)
    assert xyz.is_cuda and Q.is_cuda and xyz.is_contiguous() and Q.is_contiguous()
    return Sources(int(Q.numel()), xyz.data_ptr(), Q.data_ptr())


class Tree:
    """Owner of a tr_tree handle."""

    def __init__(self):
        self.h = C.c_void_p()

    def __del__(self):
        if _lib is not None and self.h:
            _lib.tr_tree_free(self.h)
            self.h = C.c_void_p()

    def info(self):
        n, lv, nr, npix = C.c_int64(), C.c_int32(), C.c_int32(), C.c_int32()
        check(load().tr_tree_info(self.h, C.byref(n), C.byref(lv), C.byref(nr), C.byref(npix)))
        return dict(n_nodes=n.value, levels=lv.value, nr=nr.value, npix=npix.value)


class Rays:
    """Owner of a tr_rays handle."""

    def __init__(self):
        self.h = C.c_void_p()

    def __del__(self):
        if _lib is not None and self.h:
            _lib.tr_rays_free(self.h)
            self.h = C.c_void_p()

    def info(self):
        n, npix, nr, cap = C.c_int64(), C.c_int32(), C.c_int32(), C.c_int32()
        check(load().tr_rays_info(self.h, C.byref(n), C.byref(npix), C.byref(nr), C.byref(cap)))
        return dict(n_targets=n.value, npix=npix.value, nr=nr.value, acc_cap=cap.value)


def tr_build_tree(grid: Grid, sources: Sources, params: Params, tree: Tree | None = None, stream=None) -> Tree:
    tree = tree or Tree()
    check(load().tr_build_tree(C.byref(grid), C.byref(sources), C.byref(params), C.byref(tree.h), _stream(stream)))
    return tree


def tr_build_tree_amr(grid, sources: Sources, params: Params, tree: Tree | None = None, stream=None) -> Tree:
    """grid: the (struct, host arrays) pair of make_amr_grid."""
    g, _keep = grid
    tree = tree or Tree()
    check(load().tr_build_tree_amr(C.byref(g), C.byref(sources), C.byref(params), C.byref(tree.h), _stream(stream)))
    return tree


def tr_tree_cells(tree: Tree) -> int:
    n = C.c_int64()
    check(load().tr_tree_cells(tree.h, C.byref(n)))
    return n.value


def tr_tree_flags(tree: Tree, out, stream=None):
    check(load().tr_tree_flags(tree.h, _ptr(out), _stream(stream)))


def tr_walk_map(tree: Tree, targets=None, n_targets: int | None = None, stream=None) -> Rays:
    rays = Rays()
    if targets is not None:
        assert targets.is_cuda and targets.dtype.itemsize == 8 and targets.is_contiguous()
        n = int(targets.numel())
    else:
        n = int(n_targets)
    check(load().tr_walk_map(tree.h, _ptr(targets), n, C.byref(rays.h), _stream(stream)))
    return rays


def tr_column_density(tree: Tree, out, targets=None, stream=None):
    """Column-density maps: out is a device float64 tensor [n_targets, N_PIX]
    (n_targets = the cell count when targets is None)."""
    if targets is not None:
        assert targets.is_cuda and targets.dtype.itemsize == 8 and targets.is_contiguous()
        n = int(targets.numel())
    else:
        n = tr_tree_cells(tree)
    assert out.is_cuda and out.dtype.itemsize == 8 and out.is_contiguous() and out.numel() >= n * tree.info()["npix"]
    check(load().tr_column_density(tree.h, _ptr(targets), n, _ptr(out), _stream(stream)))


def tr_ray_sweep(rays: Rays, F=None, e=None, ion=None, stream=None):
    check(load().tr_ray_sweep(rays.h, _ptr(F), _ptr(e), _ptr(ion), _stream(stream)))


def tr_walk_sweep(tree: Tree, F=None, e=None, ion=None, stream=None):
    check(load().tr_walk_sweep(tree.h, _ptr(F), _ptr(e), _ptr(ion), _stream(stream)))


def tr_tree_stats(tree: Tree) -> dict:
    out = (C.c_int64 * 6)()
    check(load().tr_tree_stats(tree.h, out))
    return dict(visited=out[0], accepted=out[1], entries=out[2], max_stack=out[3], fp64_mac=out[4],
                fp64_setup=out[5])


def tr_solve(grid: Grid, sources: Sources, params: Params, F=None, e=None, ion=None, stream=None):
    iters, delta = C.c_int32(), C.c_double()
    check(load().tr_solve(C.byref(grid), C.byref(sources), C.byref(params), _ptr(F), _ptr(e), _ptr(ion),
                          C.byref(iters), C.byref(delta), _stream(stream)))
    return iters.value, delta.value


def tr_walk_sweep_batch(trees, first, count, F=None, e=None, ion=None, stream=None):
    """One persistent launch over target ranges of several trees (lists of equal length)."""
    n = len(trees)
    arr = lambda xs, t: (t * n)(*xs)
    vp = C.c_void_p
    Fp = arr([None if F is None or F[i] is None else F[i].data_ptr() for i in range(n)], vp)
    ep = arr([None if e is None or e[i] is None else e[i].data_ptr() for i in range(n)], vp)
    ip = arr([None if ion is None or ion[i] is None else ion[i].data_ptr() for i in range(n)], vp)
    check(load().tr_walk_sweep_batch(arr([t.h.value for t in trees], vp), arr([int(x) for x in first], C.c_int64),
                                     arr([int(x) for x in count], C.c_int64), n, Fp, ep, ip, _stream(stream)))


def tr_delta(e_new, e_old, mode: int = 0, stream=None) -> float:
    out = C.c_double()
    check(load().tr_delta(_ptr(e_new), _ptr(e_old), int(e_new.numel()), mode, C.byref(out), _stream(stream)))
    return out.value


def tr_solve_noalloc(grid: Grid, sources: Sources, params: Params, F=None, e=None, ion=None, stream=None):
    """The allocation-free single pass (see include/treeray.h)."""
    check(load().tr_solve_noalloc(C.byref(grid), C.byref(sources), C.byref(params), _ptr(F), _ptr(e), _ptr(ion),
                                  _stream(stream)))


def tr_tree_nodes(tree: Tree, out8, stream=None):
    check(load().tr_tree_nodes(tree.h, _ptr(out8), _stream(stream)))


def tr_rays_export(rays: Rays, alpha=None, eps=None, e=None, ids=None, counts=None, stream=None):
    check(load().tr_rays_export(rays.h, _ptr(alpha), _ptr(eps), _ptr(e), _ptr(ids), _ptr(counts), _stream(stream)))


def tr_table_info(nside: int):
    nk, ne = C.c_int32(), C.c_int32()
    check(load().tr_table_info(nside, C.byref(nk), C.byref(ne)))
    return nk.value, ne.value


def tr_table_export(nside: int, offsets, pix, cnt, stream=None):
    check(load().tr_table_export(nside, _ptr(offsets), _ptr(pix), _ptr(cnt), _stream(stream)))


# ---- convenience ------------------------------------------------------------

def solve(n_H, dx: float, src_xyz=None, src_Q=None, *, box_lo=(0.0, 0.0, 0.0), ndot=None, e_prev=None,
          stream=None, **params):
    """Run tr_solve on device tensors; returns (F, e, ion, iters, delta)."""
    import torch
    p = tr_params_default(**params)
    g = make_grid(n_H, dx, box_lo, ndot, e_prev)
    s = make_sources(src_xyz, src_Q)
    N = g.N
    F = torch.empty((N, N, N), dtype=torch.float64, device=n_H.device)
    e = torch.empty_like(F)
    ion = torch.empty((N, N, N), dtype=torch.uint8, device=n_H.device)
    it, dl = tr_solve(g, s, p, F, e, ion, stream)
    return F, e, ion, it, dl


def theta_inf() -> float:
    return math.inf
