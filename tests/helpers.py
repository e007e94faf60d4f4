"""Shared helpers of the tests (no method arithmetic)."""
import numpy as np


def interior_mask(ion):
    """Cells whose six face neighbours share their ionised/neutral class,
    i.e. cells that are not within one cell of an ionisation front."""
    ion = np.asarray(ion)
    m = np.ones(ion.shape, dtype=bool)
    for ax in range(3):
        for sh in (1, -1):
            nb = np.roll(ion, sh, axis=ax)
            edge = [slice(None)] * 3
            edge[ax] = 0 if sh == 1 else -1
            same = nb == ion
            same[tuple(edge)] = True
            m &= same
    return m


def near_front(ion_a, ion_b):
    """Cells where two classifications differ must lie within one cell of
    the front of the reference classification."""
    return ~interior_mask(ion_a)


def decode_id(cid):
    level, off = 0, 0
    while cid >= off + 8 ** level:
        off += 8 ** level
        level += 1
    m = cid - off
    ix = iy = iz = 0
    for b in range(level):
        ix |= ((m >> (3 * b)) & 1) << b
        iy |= ((m >> (3 * b + 1)) & 1) << b
        iz |= ((m >> (3 * b + 2)) & 1) << b
    return level, ix, iy, iz


def amr_cells(g):
    """Corner (finest cells, [x, y, z]) and edge of every cell of an AMR grid,
    indexed b * 512 + (iz * 8 + iy) * 8 + ix: the layout of its blocks only."""
    size = np.array([g.cell_size(b) for b in range(g.n_blocks)], dtype=np.int64)
    c = np.arange(512)
    local = np.stack([c & 7, (c >> 3) & 7, c >> 6], axis=1)               # [x, y, z]
    corner = (8 * g.blk_pos.astype(np.int64)[:, None, :] + local[None, :, :]) * size[:, None, None]
    return corner.reshape(-1, 3), np.repeat(size, 512)



def amr_paint(g, values):
    """Cell values of an AMR grid painted onto its finest lattice [z, y, x]."""
    N = g.N_fine
    out = np.empty((N, N, N), dtype=np.asarray(values).dtype)
    v = np.asarray(values).reshape(g.n_blocks, 8, 8, 8)
    for b in range(g.n_blocks):
        s = g.cell_size(b)
        x0, y0, z0 = 8 * s * g.blk_pos[b]
        blk = np.repeat(np.repeat(np.repeat(v[b], s, 0), s, 1), s, 2)
        out[z0:z0 + 8 * s, y0:y0 + 8 * s, x0:x0 + 8 * s] = blk
    return out


def amr_interior_mask(g, ion):
    """AMR cells whose neighbourhood (the cell grown by one finest cell on
    every side) holds one ionised/neutral class: cells not at a front."""
    from scipy import ndimage
    fine = amr_paint(g, np.asarray(ion).astype(np.int8))
    uniform = ndimage.minimum_filter(fine, size=3, mode="nearest") == ndimage.maximum_filter(fine, size=3, mode="nearest")
    out = np.empty((g.n_blocks, 8, 8, 8), dtype=bool)
    for b in range(g.n_blocks):
        s = g.cell_size(b)
        x0, y0, z0 = 8 * s * g.blk_pos[b]
        sub = uniform[z0:z0 + 8 * s, y0:y0 + 8 * s, x0:x0 + 8 * s]
        out[b] = sub.reshape(8, s, 8, s, 8, s).all(axis=(1, 3, 5))
    return out.ravel()


# FP32 forms: a cell's flux is a difference of FP32-derived terms (emitted
# photons less recombinations), so its rounding error is at most a few FP32
# unit roundoffs times the flux the recombinations removed on the way to the
# cell (measured: <= 6e-7 of it, about 10 roundoffs; 30 allowed).  Cells
# where one beam is all but extinguished are ill-conditioned in this sense
# (the removed flux can exceed the arriving one 1e5-fold): they are held to
# rtol F + KAPPA (F_free - F) with F_free the oracle's unattenuated flux.
KAPPA = {0: 0.0, 1: 2e-6, 2: 2e-6}


def flux_misses(F, F_orc, rtol, kappa=0.0, free_fn=None):
    """Positions (in the given arrays, all lit in the oracle) where the flux
    misses the bar |F - F_orc| <= rtol F_orc, or, with kappa > 0, the bar
    rtol F_orc + kappa (F_free - F_orc); free_fn(positions) gives F_free."""
    err = np.abs(F - F_orc)
    miss = np.nonzero(err > rtol * F_orc)[0]
    if miss.size and kappa > 0.0 and free_fn is not None:
        Ff = np.asarray(free_fn(miss))
        assert np.all(Ff >= F_orc[miss] * (1.0 - 1e-12))
        miss = miss[err[miss] > rtol * F_orc[miss] + kappa * (Ff - F_orc[miss])]
    return miss
