"""Seeded AMR workload: blocks of 8^3 cells at up to three refinement levels.

Recipe (the AMR cluster set-up): one log-normal k^-4 realisation on the
finest lattice (base 64^3 refined twice -> 256^3 finest cells, box 10 pc),
block-averaged to each level; a block is refined into 8 child blocks when
its largest cell density exceeds the threshold (300 cm^-3), twice.  Leaves
are the cells of the resulting blocks.  Sources: power law dN/dQ ~ Q^-2.

Layout of an AmrGrid: block b has refinement level blk_level[b] (cell edge
N_fine / (N_base * 2^level) finest cells) and corner blk_pos[b] in units of
its own edge (8 cells); its cells' densities are n_H[b] as an (8, 8, 8)
array [iz][iy][ix].  Random numbers and layout only: no method arithmetic.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

from .fields import PC_CM, ALPHA_B, HNU_EUV, SEED_BASE, lognormal_density, powerlaw_sources


@dataclasses.dataclass
class AmrGrid:
    name: str
    N_base: int                      # base cells per axis
    max_level: int                   # finest refinement level
    box_cm: float
    blk_level: np.ndarray            # (B,) int32
    blk_pos: np.ndarray              # (B, 3) int32, [x, y, z] in units of the block edge
    n_H: np.ndarray                  # (B, 8, 8, 8) float64
    src_xyz: np.ndarray              # (S, 3) cm
    src_Q: np.ndarray                # (S,) s^-1
    nside: int = 4
    theta_lim: float = 0.5
    theta_if: float = 0.5
    theta_src: float = 0.5
    eta_r: int = 2
    alpha_B: float = ALPHA_B
    hnu: float = HNU_EUV

    @property
    def N_fine(self) -> int:
        return self.N_base << self.max_level

    @property
    def dx_fine(self) -> float:
        return self.box_cm / self.N_fine

    @property
    def n_blocks(self) -> int:
        return int(self.blk_level.shape[0])

    @property
    def n_leaves(self) -> int:
        return self.n_blocks * 512

    def cell_size(self, b: int) -> int:
        """Edge of block b's cells in finest cells."""
        return self.N_fine // (self.N_base << int(self.blk_level[b]))


def _block_average(fine: np.ndarray, f: int) -> np.ndarray:
    n = fine.shape[0] // f
    return fine.reshape(n, f, n, f, n, f).mean(axis=(1, 3, 5))


def refine_blocks(fine: np.ndarray, N_base: int, max_level: int, threshold: float):
    """Blocks of the refined grid: refine a block when its max density > threshold."""
    N_fine = fine.shape[0]
    levels = [_block_average(fine, N_fine // (N_base << l)) for l in range(max_level + 1)]
    out_lev, out_pos, out_val = [], [], []
    stack = [(0, x, y, z) for z in range(N_base // 8) for y in range(N_base // 8) for x in range(N_base // 8)]
    while stack:
        l, x, y, z = stack.pop()
        vals = levels[l][8 * z:8 * z + 8, 8 * y:8 * y + 8, 8 * x:8 * x + 8]
        if l < max_level and vals.max() > threshold:
            for c in range(8):
                stack.append((l + 1, 2 * x + (c & 1), 2 * y + ((c >> 1) & 1), 2 * z + ((c >> 2) & 1)))
        else:
            out_lev.append(l)
            out_pos.append((x, y, z))
            out_val.append(vals)
    order = np.lexsort((np.array([p[0] for p in out_pos]), np.array([p[1] for p in out_pos]),
                        np.array([p[2] for p in out_pos]), np.array(out_lev)))
    lev = np.array(out_lev, dtype=np.int32)[order]
    pos = np.array(out_pos, dtype=np.int32)[order]
    val = np.stack(out_val)[order]
    return lev, pos, val


def amr_cluster(N_base: int = 64, max_level: int = 2, threshold: float = 300.0, n_src: int = 100,
                seed: int = SEED_BASE + 2, box_pc: float = 10.0, **kw) -> AmrGrid:
    N_fine = N_base << max_level
    fine = lognormal_density(N_fine, seed)
    lev, pos, val = refine_blocks(fine, N_base, max_level, threshold)
    box = box_pc * PC_CM
    xyz, q = powerlaw_sources(n_src, box, seed + 5, 1e46, 1e50)
    return AmrGrid(f"amr{N_base}x{max_level}", N_base, max_level, box, lev, pos, val, xyz, q, **kw)
