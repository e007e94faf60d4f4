"""Geometry of the paper's two static test scenes, laid out on a cubic grid.

Only layout: which cells hold which of two gas densities, and where the
sources sit.  None of the method's arithmetic is here.

* rabbit hole (Sec. 3.2, the rabbit-hole test): dense cold gas with a
  straight square channel of warm rarefied gas (side l_w) from one face of
  the box to the other along one axis, the source at the channel's entrance
  on the axis.  The paper's box is 6 x 2 x 2 pc; here the box is a 6 pc cube
  whose extra volume is dense wall gas, which the radiation does not enter.
* two sources and an opaque cloud (Sec. 3.4, Table 3): a uniform cloud of
  radius 0.5 pc (rho = 2.6e-21 g cm^-3, 20 solar masses) in rarefied gas
  (1e-24 g cm^-3), lit by two equal sources 2 pc from its centre along -x
  and -y.  The paper's box [-2, 4] x [-2, 4] x [-3, 3] pc is shifted to
  [0, 6]^3 pc, so the cloud sits at (2, 2, 3) pc and the sources at
  (0, 2, 3) and (2, 0, 3) pc: the scene is symmetric under x <-> y.

Densities are hydrogen number densities n_H = rho / m_H (hydrogen gas).
"""
from __future__ import annotations

import numpy as np

from .fields import PC_CM, Workload

M_H = 1.67262192e-24           # g (proton mass)


def nh_of_rho(rho_g_cm3: float) -> float:
    return rho_g_cm3 / M_H


def rabbit_hole(N: int = 64, width_cells: int = 4, axis: int = 0, box_pc: float = 6.0,
                q: float = 1e49, rho_cold: float = 1e-18, rho_warm: float = 1e-24, **kw) -> Workload:
    """Channel of width_cells x width_cells cells (even) centred on the box's
    mid-line along `axis` (0 = x, 2 = z), from one face to the other; the
    source at the channel's entrance (coordinate 0 along the axis, the box
    centre across it)."""
    assert width_cells % 2 == 0 and 0 < width_cells < N
    box = box_pc * PC_CM
    n = np.full((N, N, N), nh_of_rho(rho_cold), dtype=np.float64)     # [iz, iy, ix]
    lo, hi = N // 2 - width_cells // 2, N // 2 + width_cells // 2
    if axis == 0:
        n[lo:hi, lo:hi, :] = nh_of_rho(rho_warm)
        src = np.array([[0.0, 0.5 * box, 0.5 * box]])
    elif axis == 2:
        n[:, lo:hi, lo:hi] = nh_of_rho(rho_warm)
        src = np.array([[0.5 * box, 0.5 * box, 0.0]])
    else:
        raise ValueError("axis must be 0 (x) or 2 (z)")
    w = Workload(f"rabbit{N}_w{width_cells}_{'xz'[axis // 2]}", N, box, n, src, np.array([q]), **kw)
    w.channel = (lo, hi, axis)
    return w


def channel_cells(w: Workload) -> np.ndarray:
    """C-order indices of the channel's cells, ordered by depth (distance
    along the channel from the source's face), shape (N, width^2)."""
    lo, hi, axis = w.channel
    N = w.N
    a = np.arange(lo, hi)
    out = []
    for depth in range(N):
        if axis == 0:
            iz, iy = np.meshgrid(a, a, indexing="ij")
            ix = np.full_like(iz, depth)
        else:
            iy, ix = np.meshgrid(a, a, indexing="ij")
            iz = np.full_like(iy, depth)
        out.append(((iz * N + iy) * N + ix).ravel())
    return np.array(out)


def two_sources_cloud(N: int = 64, box_pc: float = 6.0, q: float = 3.2e48, radius_pc: float = 0.5,
                      rho_cloud: float = 2.6e-21, rho_out: float = 1e-24, **kw) -> Workload:
    """The cloud at (2, 2, 3) pc (cells whose centre lies inside the sphere),
    the sources at (0, 2, 3) and (2, 0, 3) pc."""
    box = box_pc * PC_CM
    dx = box / N
    c = (np.arange(N) + 0.5) * dx
    z, y, x = np.meshgrid(c, c, c, indexing="ij")
    cx, cy, cz = 2.0 * PC_CM, 2.0 * PC_CM, 3.0 * PC_CM
    inside = (x - cx) ** 2 + (y - cy) ** 2 + (z - cz) ** 2 < (radius_pc * PC_CM) ** 2
    n = np.where(inside, nh_of_rho(rho_cloud), nh_of_rho(rho_out)).astype(np.float64)
    src = np.array([[0.0, cy, cz], [cx, 0.0, cz]])
    return Workload(f"twosrc{N}", N, box, n, src, np.array([q, q]), **kw)


def mirror_xy(field: np.ndarray) -> np.ndarray:
    """A cell field [iz, iy, ix] mirrored through the plane x = y."""
    return np.swapaxes(field, 1, 2)
