"""Python front end of the plain FP64 CPU oracle (``treeray_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by ``__graft_entry__.smoke``
and by the CPU-baseline leg of ``bench.py``; the CUDA library never calls it.
The C source is the oracle; this module compiles it with gcc and marshals
numpy arrays through ctypes.  Nothing here computes any part of the method.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "treeray_oracle.c")
_HDR = os.path.join(_HERE, "treeray_oracle.h")
_LIB = os.path.join(_HERE, "libtreeray_oracle.so")
_lock = threading.Lock()
_lib = None

TQH, TQ, TB, TM = 16, 33, 40, 8
TW = 2 * TM ** 3                       # weight denominator of a table entry's counts
NFACEKEYS, NEDGEKEYS, NCORNERKEYS = 6 * TQ * TQ * TB, 12 * TQ * TB, 8 * TB
NKEYS = NFACEKEYS + NEDGEKEYS + NCORNERKEYS


def build(force: bool = False) -> str:
    """Compile the oracle into a shared library next to its source."""
    stale = (not os.path.exists(_LIB)
             or os.path.getmtime(_LIB) < max(os.path.getmtime(_SRC), os.path.getmtime(_HDR)))
    if force or stale:
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
               "-shared", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


class Params(C.Structure):
    _fields_ = [("N", C.c_int32), ("dx_cm", C.c_double), ("nside", C.c_int32),
                ("eta_r", C.c_int32), ("theta_lim", C.c_double), ("theta_if", C.c_double),
                ("theta_src", C.c_double), ("lray_cells", C.c_double),
                ("alpha_B", C.c_double), ("hnu", C.c_double), ("zeta_g", C.c_int32),
                ("kernel_alpha", C.c_int32), ("kernel_eps", C.c_int32), ("bc", C.c_int32)]


# kernel choices (App. A): kernel_alpha for alpha and e, kernel_eps for eps
K_WP, K_WG = 0, 1
KE_WF3, KE_WF1, KE_WF2, KE_WF3N, KE_WP, KE_WG = range(6)
# boundary conditions of the walk (Sec. 2.8)
BC_ISOLATED, BC_PERIODIC, BC_CORNER = 0, 1, 2


_D = C.POINTER(C.c_double)
_I32 = C.POINTER(C.c_int32)
_I64 = C.POINTER(C.c_int64)
_U8 = C.POINTER(C.c_uint8)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            L.orc_ang2pix.restype = C.c_int64
            L.orc_ang2pix.argtypes = [C.c_int32, C.c_double, C.c_double, C.c_double]
            L.orc_pix2vec.argtypes = [C.c_int32, C.c_int64, _D]
            L.orc_num_points.restype = C.c_int32
            L.orc_num_points.argtypes = [C.c_int32, C.c_double]
            L.orc_radius.restype = C.c_double
            L.orc_radius.argtypes = [C.c_int32, C.c_int32]
            L.orc_wp.restype = C.c_double
            L.orc_wp.argtypes = [C.c_double]
            L.orc_wf3_split.argtypes = [C.c_double, C.c_int32, C.c_int32, _D]
            L.orc_wf1_split.argtypes = [C.c_double, C.c_int32, C.c_int32, _D]
            L.orc_wf2_split.argtypes = [C.c_double, C.c_int32, C.c_int32, _D]
            L.orc_wg.restype = C.c_double
            L.orc_wg.argtypes = [C.c_double]
            L.orc_wg_weights.argtypes = [C.c_double, C.c_double, C.c_int32, C.c_int32, _D]
            L.orc_wf3n_weights.argtypes = [C.c_double, C.c_double, C.c_int32, C.c_int32, _D]
            L.orc_eps_weights.argtypes = [C.c_int32, C.c_double, C.c_double, C.c_int32, C.c_int32, _D]
            L.orc_wp_weights.argtypes = [C.c_double, C.c_double, C.c_int32, C.c_int32, _D]
            L.orc_table_key.restype = C.c_int32
            L.orc_table_key.argtypes = [C.c_int64] * 4
            L.orc_table_entry.restype = C.c_int32
            L.orc_table_entry.argtypes = [C.c_int32, C.c_int32, _I32, _I32, C.c_int32]
            L.orc_sweep_ray.restype = C.c_double
            L.orc_sweep_ray.argtypes = [C.c_int32, C.c_int32, C.c_int32, C.c_int32, _D, _D, _D,
                                        C.c_double, _D, _D]
            L.orc_tree_build.restype = C.c_void_p
            L.orc_tree_build.argtypes = [C.c_int32, C.c_double, C.c_double, _D, _D, _D,
                                         C.c_int32, _D, _D, _D]
            L.orc_tree_build_amr.restype = C.c_void_p
            L.orc_tree_build_amr.argtypes = [C.c_int32, C.c_int32, C.c_double, C.c_double, _D, C.c_int32,
                                             _I32, _I32, _D, _D, C.c_int32, _D, _D, _D]
            L.orc_tree_n_leaves.restype = C.c_int64
            L.orc_tree_n_leaves.argtypes = [C.c_void_p]
            L.orc_tree_flag.restype = C.c_int32
            L.orc_tree_flag.argtypes = [C.c_void_p, C.c_int32, C.c_int64, C.c_int64, C.c_int64]
            L.orc_tree_free.argtypes = [C.c_void_p]
            L.orc_tree_levels.restype = C.c_int32
            L.orc_tree_levels.argtypes = [C.c_void_p]
            L.orc_tree_node.argtypes = [C.c_void_p, C.c_int32, C.c_int64, C.c_int64, C.c_int64, _D]
            L.orc_cell_quantities.argtypes = [C.c_void_p, _D, _D, _D]
            L.orc_walk_target.restype = C.c_int64
            L.orc_walk_target.argtypes = [C.c_void_p, C.POINTER(Params), C.c_int64, _D, _D, _D,
                                          _I64, C.c_int64, _I64]
            L.orc_column_density.argtypes = [C.c_void_p, C.POINTER(Params), C.c_int64, _D]
            L.orc_solve_pass.restype = C.c_int32
            L.orc_solve_pass.argtypes = [C.c_void_p, C.POINTER(Params), _I64, C.c_int64, _D, _D, _U8]
            L.orc_free_flux.restype = C.c_int32
            L.orc_free_flux.argtypes = [C.c_void_p, C.POINTER(Params), _I64, C.c_int64, _D]
            L.orc_solve.restype = C.c_int32
            L.orc_solve.argtypes = [C.POINTER(Params), _D, _D, _D, C.c_int32, _D, _D, _D,
                                    C.c_int32, C.c_double, C.c_int32, _D, _D, _U8, _I32, _D]
            L.orc_delta.restype = C.c_double
            L.orc_delta.argtypes = [C.c_int64, _D, _D, C.c_int32]
            _lib = L
    return _lib


def _p(a, ctype=_D):
    if a is None:
        return None
    return a.ctypes.data_as(ctype)


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


def ang2pix(nside: int, v) -> int:
    return int(lib().orc_ang2pix(nside, float(v[0]), float(v[1]), float(v[2])))


def pix2vec(nside: int, pix: int) -> np.ndarray:
    out = np.zeros(3)
    lib().orc_pix2vec(nside, pix, _p(out))
    return out


def num_points(eta_r: int, lray_cells: float) -> int:
    return int(lib().orc_num_points(eta_r, lray_cells))


def radius(i: int, eta_r: int) -> float:
    return float(lib().orc_radius(i, eta_r))


def wp(x: float) -> float:
    return float(lib().orc_wp(x))


def wp_weights(d: float, h: float, nr: int, eta_r: int) -> np.ndarray:
    out = np.zeros(nr)
    lib().orc_wp_weights(d, h, nr, eta_r, _p(out))
    return out


def wf3_split(d: float, nr: int, eta_r: int) -> np.ndarray:
    out = np.zeros(nr)
    lib().orc_wf3_split(d, nr, eta_r, _p(out))
    return out


def wg(x: float) -> float:
    return float(lib().orc_wg(x))


def wg_weights(d: float, h: float, nr: int, eta_r: int) -> np.ndarray:
    out = np.zeros(nr)
    lib().orc_wg_weights(d, h, nr, eta_r, _p(out))
    return out


def wf1_split(d: float, nr: int, eta_r: int) -> np.ndarray:
    out = np.zeros(nr)
    lib().orc_wf1_split(d, nr, eta_r, _p(out))
    return out


def wf2_split(d: float, nr: int, eta_r: int) -> np.ndarray:
    out = np.zeros(nr)
    lib().orc_wf2_split(d, nr, eta_r, _p(out))
    return out


def wf3n_weights(d: float, h: float, nr: int, eta_r: int) -> np.ndarray:
    out = np.zeros(nr)
    lib().orc_wf3n_weights(d, h, nr, eta_r, _p(out))
    return out


def eps_weights(kind: int, d: float, h: float, nr: int, eta_r: int) -> np.ndarray:
    out = np.zeros(nr)
    lib().orc_eps_weights(kind, d, h, nr, eta_r, _p(out))
    return out


def table_key(o, s: int) -> int:
    return int(lib().orc_table_key(int(o[0]), int(o[1]), int(o[2]), int(s)))


def table_entry(nside: int, key: int, cap: int = 4096):
    pix = np.zeros(cap, dtype=np.int32)
    cnt = np.zeros(cap, dtype=np.int32)
    n = lib().orc_table_entry(nside, key, _p(pix, _I32), _p(cnt, _I32), cap)
    return pix[:n].copy(), cnt[:n].copy()


def sweep_ray(alpha_vol, eps, e_vol=None, *, eta_r=2, nside=2, zeta_g=True, kd=0.0):
    a = _f64(alpha_vol)
    e = _f64(eps)
    ev = _f64(e_vol)
    nr = a.shape[0]
    phi0 = np.zeros(nr)
    loss = np.zeros(nr)
    F0 = lib().orc_sweep_ray(nr, eta_r, nside, int(zeta_g), _p(a), _p(e), _p(ev), kd,
                             _p(phi0), _p(loss))
    return float(F0), phi0, loss


def params_for(w, *, zeta_g: bool = True, lray_cells: float = 0.0, **over) -> Params:
    """Oracle parameters for a :class:`workloads.Workload` or an AMR grid
    (lengths in finest cells there; overrides by keyword)."""
    N, dx = (w.N_fine, w.dx_fine) if hasattr(w, "N_fine") else (w.N, w.dx)
    d = dict(N=N, dx_cm=dx, nside=w.nside, eta_r=w.eta_r, theta_lim=w.theta_lim,
             theta_if=w.theta_if, theta_src=w.theta_src, lray_cells=lray_cells,
             alpha_B=w.alpha_B, hnu=w.hnu, zeta_g=int(zeta_g))
    d.update(over)
    return Params(**d)


class Tree:
    """Oracle octree over a uniform N^3 grid (Sec. 2.1)."""

    def __init__(self, w, e_prev=None, box_lo=(0.0, 0.0, 0.0)):
        if w.N < 2 or w.N & (w.N - 1):
            raise ValueError(f"the octree needs a power-of-two grid (got N = {w.N})")
        self.N = w.N
        self._keep = [_f64(w.n_H).ravel(), _f64(w.ndot_cell).ravel() if w.ndot_cell is not None else None,
                      _f64(w.src_xyz).reshape(-1), _f64(w.src_Q), _f64(e_prev).ravel() if e_prev is not None else None,
                      np.asarray(box_lo, dtype=np.float64)]
        nH, nd, xyz, q, ep, lo = self._keep
        self.h = lib().orc_tree_build(w.N, w.dx, w.alpha_B, _p(lo), _p(nH), _p(nd),
                                      int(q.shape[0]), _p(xyz), _p(q), _p(ep))
        self.use_e = e_prev is not None
        self.n_leaf = w.N ** 3

    def __del__(self):
        if getattr(self, "h", None):
            lib().orc_tree_free(self.h)
            self.h = None

    @property
    def levels(self) -> int:
        return int(lib().orc_tree_levels(self.h))

    def flag(self, level, ix, iy, iz) -> int:
        """1 leaf (a cell), 2 parent, 0 inside a cell."""
        return int(lib().orc_tree_flag(self.h, level, ix, iy, iz))

    def node(self, level, ix, iy, iz) -> np.ndarray:
        out = np.zeros(8)
        lib().orc_tree_node(self.h, level, ix, iy, iz, _p(out))
        return out

    def cell_quantities(self):
        nc = self.n_leaf
        nd, a, e = np.zeros(nc), np.zeros(nc), np.zeros(nc)
        lib().orc_cell_quantities(self.h, _p(nd), _p(a), _p(e))
        return nd, a, e

    def walk(self, p: Params, target: int, cap: int = 1 << 16):
        diag = (2.0 if p.bc == BC_CORNER else 1.0) * p.N * math.sqrt(3.0)
        nr = num_points(p.eta_r, p.lray_cells if p.lray_cells > 0 else diag)
        npix = 12 * p.nside * p.nside
        ba, be = np.zeros(npix * nr), np.zeros(npix * nr)
        bee = np.zeros(npix * nr) if self.use_e else None
        acc = np.zeros(cap, dtype=np.int64)
        nacc = np.zeros(1, dtype=np.int64)
        visited = lib().orc_walk_target(self.h, C.byref(p), int(target), _p(ba), _p(be), _p(bee),
                                        _p(acc, _I64), cap, _p(nacc, _I64))
        n = int(nacc[0])
        return dict(visited=int(visited), accepted=acc[:min(n, cap)].copy(), n_accepted=n,
                    alpha=ba.reshape(npix, nr), eps=be.reshape(npix, nr),
                    e=None if bee is None else bee.reshape(npix, nr))

    def column_density(self, p: Params, target: int) -> np.ndarray:
        """cdMaps of one target: N_PIX column densities in cm^-2."""
        out = np.zeros(12 * p.nside * p.nside)
        lib().orc_column_density(self.h, C.byref(p), int(target), _p(out))
        return out

    def solve_pass(self, p: Params, targets=None):
        if targets is None:
            n = self.n_leaf
            tp = None
        else:
            targets = np.ascontiguousarray(targets, dtype=np.int64)
            n = targets.shape[0]
            tp = _p(targets, _I64)
        F, e, ion = np.zeros(n), np.zeros(n), np.zeros(n, dtype=np.uint8)
        lib().orc_solve_pass(self.h, C.byref(p), tp, n, _p(F), _p(e), _p(ion, _U8))
        return F, e, ion

    def free_flux(self, p: Params, targets=None):
        """Flux each target would get with no recombination losses."""
        if targets is None:
            n, tp = self.n_leaf, None
        else:
            targets = np.ascontiguousarray(targets, dtype=np.int64)
            n, tp = targets.shape[0], _p(targets, _I64)
        F = np.zeros(n)
        lib().orc_free_flux(self.h, C.byref(p), tp, n, _p(F))
        return F


class AmrTree(Tree):
    """Oracle octree over an AMR grid of 8^3-cell blocks (Sec. 2.1): targets
    and per-cell arrays are indexed b * 512 + c, c = (iz * 8 + iy) * 8 + ix."""

    def __init__(self, g, e_prev=None, box_lo=(0.0, 0.0, 0.0), ndot_cell=None):
        self.N = g.N_fine
        lev = np.ascontiguousarray(g.blk_level, dtype=np.int32)
        pos = np.ascontiguousarray(g.blk_pos, dtype=np.int32).reshape(-1)
        self._keep = [lev, pos, _f64(g.n_H).ravel(), _f64(ndot_cell).ravel() if ndot_cell is not None else None,
                      _f64(g.src_xyz).reshape(-1), _f64(g.src_Q),
                      _f64(e_prev).ravel() if e_prev is not None else None, np.asarray(box_lo, dtype=np.float64)]
        lev, pos, nH, nd, xyz, q, ep, lo = self._keep
        self.h = lib().orc_tree_build_amr(g.N_base, g.max_level, g.dx_fine, g.alpha_B, _p(lo), int(lev.shape[0]),
                                          _p(lev, _I32), _p(pos, _I32), _p(nH), _p(nd), int(q.shape[0]),
                                          _p(xyz), _p(q), _p(ep))
        self.use_e = e_prev is not None
        self.n_leaf = int(lib().orc_tree_n_leaves(self.h))


def solve(w, p: Params, *, e_init=None, max_iter: int = 1, eps_lim: float = 1e-2,
          delta_mode: int = 0, box_lo=(0.0, 0.0, 0.0)):
    """Full oracle solve with the outer iteration (Sec. 2.6)."""
    nc = w.N ** 3
    nH = _f64(w.n_H).ravel()
    nd = _f64(w.ndot_cell).ravel() if w.ndot_cell is not None else None
    xyz = _f64(w.src_xyz).reshape(-1)
    q = _f64(w.src_Q)
    ei = _f64(e_init).ravel() if e_init is not None else None
    lo = np.asarray(box_lo, dtype=np.float64)
    F, e, ion = np.zeros(nc), np.zeros(nc), np.zeros(nc, dtype=np.uint8)
    iters = np.zeros(1, dtype=np.int32)
    delta = np.zeros(1)
    lib().orc_solve(C.byref(p), _p(lo), _p(nH), _p(nd), int(q.shape[0]), _p(xyz), _p(q), _p(ei),
                    max_iter, eps_lim, delta_mode, _p(F), _p(e), _p(ion, _U8),
                    _p(iters, _I32), _p(delta))
    return F, e, ion, int(iters[0]), float(delta[0])


def delta(e_new, e_old, mode: int = 0) -> float:
    a, b = _f64(e_new).ravel(), _f64(e_old).ravel()
    return float(lib().orc_delta(a.shape[0], _p(a), _p(b), mode))
