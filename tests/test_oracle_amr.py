"""Pins for the oracle on AMR grids of 8^3-cell blocks (Sec. 2.1: the tree's
leaves are the grid cells, each block a subtree; cells may differ in size)."""
import math

import numpy as np
import pytest

from workloads import PC_CM, Workload, lognormal_density, uniform_density, uniform_sources
from workloads.amr import AmrGrid, amr_cluster, refine_blocks

from helpers import amr_cells, decode_id


def uniform_as_amr(w, N_base, max_level):
    """The cells of uniform workload w regrouped into blocks, all at max_level."""
    lev, pos, val = refine_blocks(w.n_H, N_base, max_level, threshold=-1.0)
    assert (lev == max_level).all()
    return AmrGrid("u", N_base, max_level, w.box_cm, lev, pos, val, w.src_xyz, w.src_Q, nside=w.nside,
                   theta_lim=w.theta_lim, theta_if=w.theta_if, theta_src=w.theta_src, eta_r=w.eta_r)


def uniform_index(g):
    corner, size = amr_cells(g)
    assert (size == 1).all()
    N = g.N_fine
    return (corner[:, 2] * N + corner[:, 1]) * N + corner[:, 0]


def small_amr(**kw):
    """base 8^3, refined twice: 4 blocks of level 1 and 32 of level 2 (32^3 finest)"""
    return amr_cluster(N_base=8, max_level=2, threshold=1000.0, n_src=8, box_pc=4.0, **kw)


def mid_amr(**kw):
    """base 16^3, refined twice: blocks at all three levels (64^3 finest)"""
    return amr_cluster(N_base=16, max_level=2, n_src=8, box_pc=4.0, **kw)


@pytest.mark.parametrize("N_base,max_level", [(16, 0), (8, 1)])
def test_single_level_amr_is_the_uniform_grid(orc, N_base, max_level):
    """Blocks all at one level are the uniform grid: same cells, same sources,
    the same fluxes cell by cell (a special case that reduces to the pinned
    uniform oracle, so it checks the block and cell indexing)."""
    box = 2.0 * PC_CM
    rho = lognormal_density(16, 31)
    xyz, q = uniform_sources(4, box, 32, 45.0, 47.0)
    w = Workload("u16", 16, box, rho, xyz, q, theta_lim=0.5, theta_src=0.4)
    g = uniform_as_amr(w, N_base, max_level)
    idx = uniform_index(g)
    Fu, eu, iu = orc.Tree(w).solve_pass(orc.params_for(w))
    ta = orc.AmrTree(g)
    Fa, ea, ia = ta.solve_pass(orc.params_for(g))
    np.testing.assert_array_equal(Fa, Fu[idx])
    np.testing.assert_array_equal(ia, iu[idx])
    nd, a, e = ta.cell_quantities()
    ndu, au, euu = orc.Tree(w).cell_quantities()
    np.testing.assert_array_equal(nd, ndu[idx])
    np.testing.assert_array_equal(a, au[idx])


def test_amr_nodes_equal_direct_sums(orc):
    """Every node present in the tree is the sum over the cells inside it:
    mass n_H s^3, centre of mass, alpha, eps, e = e_prev s^3 and ionised mass."""
    g = mid_amr()
    rng = np.random.default_rng(3)
    ep = rng.uniform(0, 1, g.n_leaves) * (rng.random(g.n_leaves) < 0.3)
    t = orc.AmrTree(g, e_prev=ep)
    nd, a, e = t.cell_quantities()
    corner, size = amr_cells(g)
    vol = size.astype(np.float64) ** 3
    m = g.n_H.ravel() * vol
    cen = corner + 0.5 * size[:, None]
    N = g.N_fine
    checked = 0
    for level in range(t.levels):
        n = 2 ** level
        s = N // n
        for _ in range(40):
            ix, iy, iz = rng.integers(0, n, 3)
            lo = np.array([ix, iy, iz]) * s
            inside = np.all((corner >= lo) & (corner < lo + s), axis=1)
            covered = (vol[inside].sum() == s ** 3)
            got = t.node(level, ix, iy, iz)
            if not covered:            # a node inside a leaf: not part of the tree
                continue
            M = m[inside].sum()
            want = [M, *((m[inside, None] * cen[inside]).sum(axis=0) / M), a[inside].sum(), e[inside].sum(),
                    (ep * vol)[inside].sum(), m[inside & (ep > 0)].sum()]
            np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-300)
            checked += 1
    assert checked > 100


@pytest.mark.parametrize("theta", [0.3, 0.5])
def test_amr_accepted_nodes_partition_domain(orc, theta):
    """The accepted nodes tile the domain minus the target cell exactly once,
    none lies inside a cell, and alpha and eps are conserved on the rays."""
    g = small_amr(theta_lim=theta, theta_src=0.4)
    t = orc.AmrTree(g)
    p = orc.params_for(g)
    nd, a, e = t.cell_quantities()
    corner, size = amr_cells(g)
    N = g.N_fine
    rng = np.random.default_rng(4)
    # targets of every cell size
    picks = [int(rng.choice(np.flatnonzero(size == s))) for s in np.unique(size)] + list(rng.integers(0, g.n_leaves, 4))
    for tgt in picks:
        res = t.walk(p, tgt)
        cover = np.zeros((N, N, N), dtype=np.int32)
        for cid in res["accepted"]:
            level, ix, iy, iz = decode_id(int(cid))
            s = N >> level
            assert s >= size[np.all((corner >= np.array([ix, iy, iz]) * s) &
                                    (corner < np.array([ix, iy, iz]) * s + s), axis=1)].max()
            cover[iz * s:iz * s + s, iy * s:iy * s + s, ix * s:ix * s + s] += 1
        x, y, z = corner[tgt]
        s = size[tgt]
        assert (cover[z:z + s, y:y + s, x:x + s] == 0).all()
        cover[z:z + s, y:y + s, x:x + s] = 1
        assert (cover == 1).all()
        assert res["alpha"].sum() == pytest.approx(a.sum() - a[tgt], rel=1e-12)
        assert res["eps"].sum() == pytest.approx(e.sum() - e[tgt], rel=1e-12, abs=1e-300)


def test_amr_mac_invariants(orc):
    """Accepted nodes that are not cells satisfy the MACs measured from the
    target cell's centre (Sec. 2.4)."""
    g = mid_amr(theta_lim=0.5, theta_src=0.3)
    t = orc.AmrTree(g)
    p = orc.params_for(g)
    corner, size = amr_cells(g)
    cells = {}
    for q in range(g.n_leaves):
        s = int(size[q])
        L = int(math.log2(g.N_fine // s))
        cells[(L, *(corner[q] // s))] = q
    for tgt in (0, g.n_leaves // 2, g.n_leaves - 1):
        c = corner[tgt] + 0.5 * size[tgt]
        for cid in t.walk(p, tgt)["accepted"]:
            level, ix, iy, iz = decode_id(int(cid))
            if (level, ix, iy, iz) in cells:
                continue
            node = t.node(level, ix, iy, iz)
            d = math.dist(c, node[1:4])
            h = g.N_fine >> level
            assert h < 0.5 * d
            if node[5] > 0:
                assert h < 0.3 * d


def test_amr_optically_thin_inverse_square(orc):
    """Negligible gas on an AMR grid: F = Q / (4 pi d^2) with d from the
    source cell's centre to the target cell's centre, and the source's own
    cell gets Q / (4 pi (s dx / 2)^2) for its edge s."""
    g = small_amr(theta_src=1e-3)
    g.n_H = np.full_like(g.n_H, 1e-20)
    corner, size = amr_cells(g)
    src = int(np.flatnonzero(size == size.max())[100])        # a coarse cell
    cen = (corner + 0.5 * size[:, None]) * g.dx_fine
    g.src_xyz = cen[src][None, :].copy()
    g.src_Q = np.array([1e48])
    rng = np.random.default_rng(6)
    tg = np.concatenate([[src], rng.choice(g.n_leaves, 3000, replace=False)])
    F, e, ion = orc.AmrTree(g).solve_pass(orc.params_for(g), targets=tg)
    d2 = ((cen[tg] - cen[src]) ** 2).sum(axis=1)
    mask = tg != src
    np.testing.assert_allclose(F[mask], 1e48 / (4 * math.pi * d2[mask]), rtol=1e-9)
    assert F[0] == pytest.approx(1e48 / (4 * math.pi * (size[src] * g.dx_fine / 2) ** 2), rel=1e-9)
    assert ion.all()
