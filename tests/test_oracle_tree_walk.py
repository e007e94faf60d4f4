"""Pins for the oracle's tree build (Sec. 2.1, Eq. 1-3) and walk (Sec. 2.3-2.4)."""
import math

import numpy as np
import pytest

from workloads import lognormal_density, uniform_sources, Workload, PC_CM, ALPHA_B


def small_workload(N=16, n_src=5, seed=99, **kw):
    box = 2.0 * PC_CM
    rho = lognormal_density(N, seed)
    xyz, q = uniform_sources(n_src, box, seed + 1, 44.0, 47.0)
    return Workload(f"t{N}", N, box, rho, xyz, q, seed=seed, **kw)


def decode(cid):
    """level and (ix, iy, iz) of a canonical level-order Morton id."""
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


def test_cell_netting_and_sources(orc):
    w = small_workload()
    t = orc.Tree(w)
    nd, a, e = t.cell_quantities()
    assert nd.sum() == pytest.approx(w.src_Q.sum(), rel=1e-14)
    rec = w.alpha_B * w.n_H.ravel() ** 2 * w.dx ** 3
    # Eq. 1-2 per cell: one of the two is zero, and their difference is net emission
    assert np.all((a == 0) | (e == 0)) and np.all(a >= 0) and np.all(e >= 0)
    np.testing.assert_allclose(e - a, nd - rec, rtol=1e-12, atol=1e-12 * rec.max())
    assert (e > 0).sum() >= 1


def test_nodes_equal_direct_sums(orc):
    w = small_workload()
    rng = np.random.default_rng(0)
    ep = rng.uniform(0, 1, w.N ** 3) * (rng.random(w.N ** 3) < 0.3)
    t = orc.Tree(w, e_prev=ep)
    nd, a, e = t.cell_quantities()
    N = w.N
    shape = (N, N, N)
    m = w.n_H
    ion = (ep.reshape(shape) > 0) * m
    zz, yy, xx = np.meshgrid(np.arange(N) + 0.5, np.arange(N) + 0.5, np.arange(N) + 0.5, indexing="ij")
    for level in range(t.levels):
        n = 2 ** level
        s = N // n
        for _ in range(6):
            ix, iy, iz = rng.integers(0, n, 3)
            sl = (slice(iz * s, iz * s + s), slice(iy * s, iy * s + s), slice(ix * s, ix * s + s))
            got = t.node(level, ix, iy, iz)
            M = m[sl].sum()
            want = [M, (m * xx)[sl].sum() / M, (m * yy)[sl].sum() / M, (m * zz)[sl].sum() / M,
                    a.reshape(shape)[sl].sum(), e.reshape(shape)[sl].sum(),
                    ep.reshape(shape)[sl].sum(), ion[sl].sum()]
            np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-300)


@pytest.mark.parametrize("theta", [0.3, 0.5, 1.0])
def test_accepted_nodes_partition_domain(orc, theta):
    """The accepted nodes tile the domain minus the target exactly once, and
    every mapped quantity is conserved: sum of the bins = sum over cells != target."""
    w = small_workload(theta_lim=theta, theta_src=0.4)
    t = orc.Tree(w)
    p = orc.params_for(w)
    nd, a, e = t.cell_quantities()
    N = w.N
    rng = np.random.default_rng(1)
    for tgt in rng.integers(0, N ** 3, 12):
        res = t.walk(p, int(tgt))
        cover = np.zeros(N ** 3, dtype=np.int32).reshape(N, N, N)
        for cid in res["accepted"]:
            level, ix, iy, iz = decode(int(cid))
            s = N >> level
            cover[iz * s:iz * s + s, iy * s:iy * s + s, ix * s:ix * s + s] += 1
        flat = cover.ravel()
        assert flat[tgt] == 0
        assert np.all(np.delete(flat, tgt) == 1)
        assert res["alpha"].sum() == pytest.approx(a.sum() - a[tgt], rel=1e-12)
        assert res["eps"].sum() == pytest.approx(e.sum() - e[tgt], rel=1e-12, abs=1e-300)


def test_mac_invariants(orc):
    """Accepted non-leaf nodes satisfy the BH and Src MACs; their parents fail
    a MAC or contain the target (Sec. 2.4)."""
    w = small_workload(theta_lim=0.5, theta_src=0.3)
    t = orc.Tree(w)
    p = orc.params_for(w)
    N = w.N
    L = t.levels - 1
    tgt = 1234
    tx, ty, tz = tgt % N, (tgt // N) % N, tgt // (N * N)
    res = t.walk(p, tgt)
    for cid in res["accepted"]:
        level, ix, iy, iz = decode(int(cid))
        node = t.node(level, ix, iy, iz)
        d = math.dist((tx + 0.5, ty + 0.5, tz + 0.5), node[1:4])
        h = N >> level
        if level < L:
            assert h < 0.5 * d
            if node[5] > 0:
                assert h < 0.3 * d
        if level > 0:
            pl, px, py, pz = level - 1, ix // 2, iy // 2, iz // 2
            par = t.node(pl, px, py, pz)
            hp = N >> pl
            contains = (px * hp <= tx < px * hp + hp) and (py * hp <= ty < py * hp + hp) and (pz * hp <= tz < pz * hp + hp)
            dp = math.dist((tx + 0.5, ty + 0.5, tz + 0.5), par[1:4])
            assert contains or hp >= 0.5 * dp or (par[5] > 0 and hp >= 0.3 * dp)


def test_theta_zero_opens_everything(orc):
    w = small_workload(N=8, theta_lim=1e-9)
    t = orc.Tree(w)
    res = t.walk(orc.params_for(w), 100)
    assert res["n_accepted"] == 8 ** 3 - 1
    assert all(decode(int(c))[0] == 3 for c in res["accepted"])


def test_cost_independent_of_source_count(orc):
    """With theta_src = theta_lim the visited nodes do not depend on the sources (Sec. 5.2)."""
    base = small_workload(N=16, n_src=1, theta_lim=0.5, theta_src=0.5)
    many = small_workload(N=16, n_src=100, theta_lim=0.5, theta_src=0.5)
    many.n_H = base.n_H
    t1, t2 = orc.Tree(base), orc.Tree(many)
    for tgt in (0, 777, 4095):
        assert t1.walk(orc.params_for(base), tgt)["visited"] == t2.walk(orc.params_for(many), tgt)["visited"]
