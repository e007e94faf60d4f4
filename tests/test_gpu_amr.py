"""Parity of the CUDA path with the oracle on AMR grids (blocks of 8^3 cells
at up to three refinement levels, Sec. 2.1; N_PIX = 192 with the IF and Src
refinements of the MAC, Sec. 2.4).

Bars: bit-exact node topology and FP64 node masses and centres; accepted
node lists bit-exact in every form; cell flux within 1e-5 (FP64) and 1e-3
(both FP32 forms) away from the ionisation front; classification identical
except next to the front (cells whose neighbourhood holds both classes).
No fraction of the cells is exempt.
"""
import math

import numpy as np
import pytest

from helpers import KAPPA, amr_cells, amr_interior_mask, decode_id, flux_misses
from oracle_pool import amr_neighbours, oracle_free, oracle_pass, sampled_check
from workloads.amr import amr_cluster

pytestmark = pytest.mark.gpu

RTOL = {0: 1e-5, 1: 1e-3, 2: 1e-3}


@pytest.fixture(scope="module")
def B():
    import torch
    import paper_2105_09644_gb300 as pkg
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    pkg.build()
    from paper_2105_09644_gb300 import binding
    binding.load()
    return binding


def dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def small_amr(**kw):
    """base 8^3 refined twice: blocks of levels 1 and 2, 32^3 finest cells"""
    return amr_cluster(N_base=8, max_level=2, threshold=1000.0, n_src=8, box_pc=4.0, **kw)


def mid_amr(**kw):
    """base 16^3 refined twice: blocks of all three levels, 64^3 finest cells"""
    return amr_cluster(N_base=16, max_level=2, n_src=8, box_pc=4.0, **kw)


def gpu_params(B, g, precision=0, zeta_g=True, **kw):
    d = dict(theta_lim=g.theta_lim, theta_if=g.theta_if, theta_src=g.theta_src, nside=g.nside,
             eta_r=g.eta_r, alpha_B=g.alpha_B, hnu=g.hnu, precision=precision, zeta_g=int(zeta_g))
    d.update(kw)
    return B.tr_params_default(**d)


def gpu_amr_tree(B, g, precision=0, e_prev=None, **kw):
    import torch
    keep = [dev(g.n_H.ravel()), dev(g.src_xyz), dev(g.src_Q)]
    ep = dev(e_prev) if e_prev is not None else None
    grid = B.make_amr_grid(g.N_base, g.max_level, g.blk_level, g.blk_pos, keep[0], g.dx_fine, e_prev=ep)
    t = B.tr_build_tree_amr(grid, B.make_sources(keep[1], keep[2]), gpu_params(B, g, precision, **kw))
    torch.cuda.synchronize()
    t._keep = keep + [ep, grid]
    return t


def gpu_amr_solve(B, g, precision=0, e_prev=None, **kw):
    import torch
    t = gpu_amr_tree(B, g, precision, e_prev, **kw)
    n = B.tr_tree_cells(t)
    assert n == g.n_leaves
    F = torch.empty(n, dtype=torch.float64, device="cuda")
    e = torch.empty_like(F)
    ion = torch.empty(n, dtype=torch.uint8, device="cuda")
    B.tr_walk_sweep(t, F, e, ion)
    torch.cuda.synchronize()
    return F.cpu().numpy(), e.cpu().numpy(), ion.cpu().numpy()


def compare_amr(g, F, ion, F_orc, ion_orc, rtol, kappa=0.0, free_fn=None):
    inner = amr_interior_mask(g, ion_orc)
    assert not np.any((ion != ion_orc) & inner), "cells away from the front change class"
    lit = np.nonzero(inner & (F_orc > 0))[0]
    if lit.size:
        err = np.abs(F[lit] - F_orc[lit]) / F_orc[lit]
        miss = flux_misses(F[lit], F_orc[lit], rtol, kappa, None if free_fn is None else (lambda k: free_fn(lit[k])))
        assert miss.size == 0, f"{miss.size} cells miss; max rel flux error {err.max():.3e} > {rtol} (median {np.median(err):.2e})"
    dark = inner & (F_orc == 0)
    assert np.all(F[dark] == 0.0)


def morton_positions(level):
    m = np.arange(8 ** level, dtype=np.int64)
    ix = np.zeros_like(m); iy = np.zeros_like(m); iz = np.zeros_like(m)
    for b in range(level):
        ix |= ((m >> (3 * b)) & 1) << b
        iy |= ((m >> (3 * b + 1)) & 1) << b
        iz |= ((m >> (3 * b + 2)) & 1) << b
    return ix, iy, iz


# --------------------------------------------------------------------------

@pytest.mark.parametrize("make", [small_amr, mid_amr])
@pytest.mark.parametrize("precision", [0, 1])
def test_amr_topology_and_nodes(B, orc, make, precision):
    """Node flags bit-exact; FP64 masses and centres bit-exact, other
    moments to rounding; FP32 moments within their compensated-sum error."""
    import torch
    g = make()
    rng = np.random.default_rng(3)
    e_prev = rng.uniform(0, 1e-9, g.n_leaves) * (rng.random(g.n_leaves) < 0.4)
    t = gpu_amr_tree(B, g, precision, e_prev=e_prev)
    info = t.info()
    flags = torch.empty(info["n_nodes"], dtype=torch.uint8, device="cuda")
    nodes = torch.empty((info["n_nodes"], 8), dtype=torch.float64, device="cuda")
    B.tr_tree_flags(t, flags)
    B.tr_tree_nodes(t, nodes)
    torch.cuda.synchronize()
    flags, nodes = flags.cpu().numpy(), nodes.cpu().numpy()
    ot = orc.AmrTree(g, e_prev=e_prev)
    L = info["levels"] - 1
    assert 2 ** L == g.N_fine
    off = 0
    for level in range(L + 1):
        ix, iy, iz = morton_positions(level)
        want_f = np.array([ot.flag(level, x, y, z) for x, y, z in zip(ix, iy, iz)], dtype=np.uint8)
        got_f = flags[off:off + 8 ** level]
        assert np.array_equal(got_f, want_f), (level, np.flatnonzero(got_f != want_f)[:5])
        present = np.flatnonzero(want_f > 0)
        pick = present if present.size <= 3000 else rng.choice(present, 3000, replace=False)
        for m in pick:
            want = ot.node(level, ix[m], iy[m], iz[m])
            got = nodes[off + m]
            if precision == 0:
                assert np.array_equal(got[:4], want[:4]), (level, m, got[:4], want[:4])
                np.testing.assert_allclose(got[4:], want[4:], rtol=1e-13, atol=1e-300)
            else:
                np.testing.assert_allclose(got[:4], want[:4], rtol=2e-6)
                np.testing.assert_allclose(got[4:], want[4:], rtol=2e-6, atol=1e-30 + 1e-6 * np.abs(want[4:]).max())
        off += 8 ** level


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("theta,theta_src", [(0.5, 0.5), (0.3, 0.2)])
def test_amr_walk_lists_and_bins(B, orc, theta, theta_src, precision):
    """Accepted-node lists bit-exact in both walks and ray bins to rounding
    (FP64) or 2e-5 (FP32), for targets of every cell size (cell indices
    b * 512 + c)."""
    import torch
    g = mid_amr(theta_lim=theta, theta_src=theta_src)
    t = gpu_amr_tree(B, g, precision)
    corner, size = amr_cells(g)
    rng = np.random.default_rng(11)
    targets = np.unique(np.concatenate([rng.choice(np.flatnonzero(size == s), 8) for s in np.unique(size)]
                                       + [rng.integers(0, g.n_leaves, 16), [0, g.n_leaves - 1]]))
    r = B.tr_walk_map(t, dev(targets.astype(np.int64)))
    info = r.info()
    nt, npix, nr, cap = info["n_targets"], info["npix"], info["nr"], info["acc_cap"]
    assert npix == 192
    a = torch.empty((nt, npix, nr), dtype=torch.float64, device="cuda")
    e = torch.empty_like(a)
    ids = torch.empty((nt, cap), dtype=torch.int64, device="cuda")
    counts = torch.empty(nt, dtype=torch.int32, device="cuda")
    B.tr_rays_export(r, a, e, None, ids, counts)
    torch.cuda.synchronize()
    a, e, ids, counts = a.cpu().numpy(), e.cpu().numpy(), ids.cpu().numpy(), counts.cpu().numpy()
    ot = orc.AmrTree(g)
    p = orc.params_for(g)
    tol = 1e-12 if precision == 0 else 2e-5
    for k, tgt in enumerate(targets):
        res = ot.walk(p, int(tgt))
        assert counts[k] == res["n_accepted"]
        assert np.array_equal(np.sort(ids[k, :counts[k]]), np.sort(res["accepted"]))
        scale = max(res["alpha"].max(), 1e-300)
        np.testing.assert_allclose(a[k], res["alpha"], rtol=tol, atol=tol * scale)
        escale = max(res["eps"].max(), 1e-300)
        np.testing.assert_allclose(e[k], res["eps"], rtol=tol, atol=tol * escale)


@pytest.mark.parametrize("precision", [0, 1, 2])
def test_amr_solve_matches_oracle(B, orc, precision):
    """Every cell of the small AMR grid (18,432 cells, N_PIX = 192)."""
    g = small_amr()
    F, e, ion = gpu_amr_solve(B, g, precision)
    ot, p = orc.AmrTree(g), orc.params_for(g)
    F_orc, e_orc, ion_orc = ot.solve_pass(p)
    compare_amr(g, F, ion, F_orc, ion_orc, RTOL[precision], KAPPA[precision], lambda c: ot.free_flux(p, targets=c))
    np.testing.assert_allclose(e, F * g.hnu / 2.99792458e10, rtol=1e-14)


@pytest.mark.parametrize("precision", [0, 1, 2])
def test_amr_mid_sampled(B, orc, precision):
    """The 64^3-finest grid with cells of three sizes: sampled targets and
    their face neighbours against the oracle, every sampled cell away from
    the oracle's front held to the bar."""
    g = mid_amr()
    F, e, ion = gpu_amr_solve(B, g, precision)
    rng = np.random.default_rng(5)
    targets = rng.choice(g.n_leaves, 300, replace=False)
    ot = orc.AmrTree(g)
    p = orc.params_for(g)
    checked, worst = sampled_check(F, ion, targets, amr_neighbours(g, targets),
                                   lambda c: ot.solve_pass(p, targets=c), RTOL[precision], KAPPA[precision],
                                   lambda c: ot.free_flux(p, targets=c))
    assert checked >= 150


def test_amr_if_mac_with_previous_pass(B, orc):
    """A second pass with the first pass's energy density: the IF MAC
    (ionised mass, Sec. 2.4) and zeta_d (Eq. 17) on an AMR grid."""
    g = small_amr(theta_if=0.25)
    F0, e0, _ = orc.AmrTree(g).solve_pass(orc.params_for(g))
    F, e, ion = gpu_amr_solve(B, g, 0, e_prev=e0)
    F_orc, _, ion_orc = orc.AmrTree(g, e_prev=e0).solve_pass(orc.params_for(g))
    compare_amr(g, F, ion, F_orc, ion_orc, RTOL[0])


@pytest.mark.parametrize("precision", [0, 1, 2])
def test_amr_unfused_equals_fused(B, precision):
    import torch
    g = small_amr(theta_src=0.3)
    F, e, ion = gpu_amr_solve(B, g, precision)
    t = gpu_amr_tree(B, g, precision)
    r = B.tr_walk_map(t, None, n_targets=g.n_leaves)
    F2 = torch.empty(g.n_leaves, dtype=torch.float64, device="cuda")
    ion2 = torch.empty(g.n_leaves, dtype=torch.uint8, device="cuda")
    B.tr_ray_sweep(r, F2, None, ion2)
    torch.cuda.synchronize()
    compare_amr(g, F2.cpu().numpy(), ion2.cpu().numpy(), F, ion, 1e-12 if precision == 0 else 1e-6)


def test_amr_batched_with_uniform(B):
    """An AMR tree and a uniform tree in one batched launch, each cut into
    ranges, give what each gives alone."""
    import torch
    from workloads import workload
    g = small_amr()
    w = workload("turbulent32", nside=4, theta_lim=0.5)
    F_a, _, ion_a = gpu_amr_solve(B, g, 1)
    ta = gpu_amr_tree(B, g, 1)
    tu_keep = [dev(w.n_H), dev(w.src_xyz), dev(w.src_Q)]
    tu = B.tr_build_tree(B.make_grid(tu_keep[0], w.dx), B.make_sources(tu_keep[1], tu_keep[2]),
                         gpu_params(B, w, 1))
    Fu_alone = torch.empty((w.N,) * 3, dtype=torch.float64, device="cuda")
    B.tr_walk_sweep(tu, Fu_alone)
    Fa = torch.empty(g.n_leaves, dtype=torch.float64, device="cuda")
    Fu = torch.empty((w.N,) * 3, dtype=torch.float64, device="cuda")
    na, nu = g.n_leaves, w.N ** 3
    B.tr_walk_sweep_batch([ta, tu, ta, tu], [0, 0, na // 3, nu // 2], [na // 3, nu // 2, na - na // 3, nu - nu // 2],
                          F=[Fa, Fu, Fa, Fu])
    torch.cuda.synchronize()
    np.testing.assert_allclose(Fa.cpu().numpy(), F_a, rtol=1e-6, atol=1e-30)
    np.testing.assert_allclose(Fu.cpu().numpy(), Fu_alone.cpu().numpy(), rtol=1e-6, atol=1e-30)


def test_amr_layout_errors(B):
    import torch
    g = small_amr()
    nH = dev(g.n_H.ravel())
    p = gpu_params(B, g)
    s = B.make_sources()
    # a level-2 block dropped: the blocks no longer fill the box
    lev, pos = g.blk_level[1:], g.blk_pos[1:]
    with pytest.raises(B.TreeRayError) as ei:
        B.tr_build_tree_amr(B.make_amr_grid(g.N_base, g.max_level, lev, pos, nH[512:].contiguous(), g.dx_fine), s, p)
    assert ei.value.status == B.TR_EINVAL and "fill" in str(ei.value)
    # a coarse block laid over refined ones
    lev = np.concatenate([g.blk_level, [1]]).astype(np.int32)
    k = int(np.flatnonzero(g.blk_level == 2)[0])
    pos = np.concatenate([g.blk_pos, g.blk_pos[k:k + 1] // 2]).astype(np.int32)
    nH2 = torch.cat([nH, nH[:512]])
    with pytest.raises(B.TreeRayError) as ei:
        B.tr_build_tree_amr(B.make_amr_grid(g.N_base, g.max_level, lev, pos, nH2, g.dx_fine), s, p)
    assert ei.value.status == B.TR_EINVAL and "inside" in str(ei.value)
    # a target index past the last cell (the walk kernel checks each one)
    t = gpu_amr_tree(B, g, 0)
    with pytest.raises(B.TreeRayError) as ei:
        B.tr_walk_map(t, dev(np.array([0, g.n_leaves], dtype=np.int64)))
    assert ei.value.status == B.TR_EINVAL and "outside" in str(ei.value)
    # position out of range
    pos = g.blk_pos.copy()
    pos[0, 0] = 99
    with pytest.raises(B.TreeRayError) as ei:
        B.tr_build_tree_amr(B.make_amr_grid(g.N_base, g.max_level, g.blk_level, pos, nH, g.dx_fine), s, p)
    assert ei.value.status == B.TR_EINVAL


@pytest.mark.slow
@pytest.mark.parametrize("precision", [1, 2, 0])
def test_full_size_amr_cluster_sampled(B, precision):
    """The AMR cluster at full size (base 64^3 refined twice, 5.9M cells,
    N_PIX = 192, N_R = 59, theta_IF = theta_src = 0.5): sampled targets and
    their face neighbours against the oracle; every sampled cell away from
    the oracle's front meets the bar."""
    g = amr_cluster()
    F, e, ion = gpu_amr_solve(B, g, precision)
    assert np.all(np.isfinite(F))
    rng = np.random.default_rng(2105)
    targets = rng.choice(g.n_leaves, 40, replace=False).astype(np.int64)
    checked, worst = sampled_check(F, ion, targets, amr_neighbours(g, targets),
                                   lambda c: oracle_pass("amr", {}, c, nproc=8), RTOL[precision], KAPPA[precision],
                                   lambda c: oracle_free("amr", {}, c, nproc=8))
    assert checked >= 20
