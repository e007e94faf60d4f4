"""The seeded inputs follow their stated recipes (no method arithmetic here):
log-normal k^-4 fields, source distributions, the source-count workloads
and the AMR refinement."""
import math

import numpy as np
import pytest

from workloads import lognormal_density, powerlaw_sources, uniform_sources, workload
from workloads.amr import amr_cluster, _block_average


def test_lognormal_field_statistics():
    n = lognormal_density(64, 123, sigma_ln=1.5, mean_nH=100.0)
    ln = np.log(n)
    assert ln.std() == pytest.approx(1.5, rel=1e-9)                # sigma_ln by construction
    assert ln.mean() == pytest.approx(math.log(100.0) - 0.5 * 1.5 ** 2, rel=1e-9)
    assert n.mean() == pytest.approx(100.0, rel=0.35)              # exp(g - s^2/2) has mean 1 (heavy tail)
    # power spectrum of g: P(k) ~ k^-4, fitted over shells 2 <= k < 20
    g = ln - ln.mean()
    P = np.abs(np.fft.fftn(g)) ** 2
    k = np.sqrt(sum(np.meshgrid(*(np.fft.fftfreq(64) * 64,) * 3, indexing="ij")[a] ** 2 for a in range(3)))
    shells = np.arange(2, 20)
    Pk = np.array([P[(k >= s) & (k < s + 1)].mean() for s in shells])
    slope = np.polyfit(np.log(shells + 0.5), np.log(Pk), 1)[0]
    assert slope == pytest.approx(-4.0, abs=0.3)


def test_fields_and_sources_are_seeded():
    assert np.array_equal(lognormal_density(16, 5), lognormal_density(16, 5))
    assert not np.array_equal(lognormal_density(16, 5), lognormal_density(16, 6))
    a = uniform_sources(10, 1.0, 3, 47.0, 50.0)
    b = uniform_sources(10, 1.0, 3, 47.0, 50.0)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_uniform_sources_ranges():
    xyz, q = uniform_sources(20000, 7.0, 9, 47.0, 50.0)
    assert xyz.min() >= 0.0 and xyz.max() < 7.0
    lq = np.log10(q)
    assert lq.min() >= 47.0 and lq.max() <= 50.0
    assert abs(lq.mean() - 48.5) < 0.03


def test_powerlaw_sources_follow_q_minus_two():
    """dN/dQ ~ Q^-2 on [q_lo, q_hi]: the CDF is (1/q_lo - 1/Q) / (1/q_lo - 1/q_hi)."""
    from scipy import stats
    lo, hi = 1e46, 1e50
    _, q = powerlaw_sources(20000, 1.0, 4, lo, hi)
    assert q.min() >= lo and q.max() <= hi
    cdf = lambda x: (1 / lo - 1 / np.asarray(x)) / (1 / lo - 1 / hi)
    assert stats.kstest(q, cdf).pvalue > 0.01


def test_sourcecount_workloads():
    for name, S in (("sourcecount256_s1", 1), ("sourcecount256_s100", 100)):
        w = workload(name)
        assert w.N == 256 and w.src_Q.shape == (S,)
        assert w.src_Q.sum() == pytest.approx(1e51, rel=1e-12)
        assert w.box_cm == pytest.approx(30 * 3.0856775814913673e18)
    d = workload("diffuse256")
    assert d.src_Q.size == 0 and d.ndot_cell.sum() == pytest.approx(1e51, rel=1e-12)
    ratio = d.ndot_cell / d.n_H ** 2
    assert np.allclose(ratio, ratio.flat[0], rtol=1e-12)


def test_amr_refinement_follows_the_threshold():
    """Small cluster grid: blocks tile the box; a block at a level below
    the maximum has all cell densities <= threshold at its level (it was
    not refined), and each refined block's parent region exceeded it."""
    g = amr_cluster(N_base=16, max_level=2, threshold=300.0, n_src=3)
    fine = lognormal_density(g.N_fine, 2105_09644 + 2)      # the cluster's default seed
    vol = sum((8 * g.cell_size(b)) ** 3 for b in range(g.n_blocks))
    assert vol == g.N_fine ** 3
    for b in range(g.n_blocks):
        s = g.cell_size(b)
        lev = int(g.blk_level[b])
        x0, y0, z0 = 8 * s * g.blk_pos[b]
        region = fine[z0:z0 + 8 * s, y0:y0 + 8 * s, x0:x0 + 8 * s]
        np.testing.assert_allclose(g.n_H[b], _block_average(region, s), rtol=1e-12)
        if lev < g.max_level:
            assert g.n_H[b].max() <= 300.0
        if lev > 0:                                   # its parent block was refined
            ps = 2 * s
            px, py, pz = (g.blk_pos[b] // 2) * 8 * ps
            parent = _block_average(fine[pz:pz + 8 * ps, py:py + 8 * ps, px:px + 8 * ps], ps)
            assert parent.max() > 300.0
