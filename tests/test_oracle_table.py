"""Pins for the node->ray table (Sec. 2.3 first mapping step)."""
import math
from fractions import Fraction

import numpy as np
import pytest


def ref_key(o, s, TQH=16, TQ=33, TB=40):
    """Key from exact rational arithmetic (independent of the C integer code)."""
    ab = [abs(x) for x in o]
    a = max(range(3), key=lambda i: (ab[i], -i))
    b, c = [i for i in range(3) if i != a]
    A = ab[a]
    face = 2 * a + (1 if o[a] < 0 else 0)

    def fb(x):
        if x == 0:
            return TQH
        q = min(TQH - 1, math.floor(Fraction(TQH * abs(x), A)))
        return TQH + 1 + q if x > 0 else TQH - 1 - q
    # psi = 2s/|o|, bin = floor(32 psi) = floor(64 s / |o|), exactly
    o2 = sum(x * x for x in o)
    pb = 0
    while Fraction((pb + 1) ** 2) * o2 <= (64 * s) ** 2:
        pb += 1
    pb = min(pb, TB - 1)
    return ((face * TQ + fb(o[b])) * TQ + fb(o[c])) * TB + pb


def test_key_matches_exact_rational(orc):
    rng = np.random.default_rng(11)
    for _ in range(3000):
        s = int(2 ** rng.integers(0, 7))
        o = rng.integers(-400, 401, 3)
        if not o.any():
            continue
        assert orc.table_key(o, s) == ref_key([int(x) for x in o], s)
    # ties between axes go to the lowest axis; centre bins for zero offsets
    assert orc.table_key([4, 4, 4], 1) == ref_key([4, 4, 4], 1)
    assert orc.table_key([0, 0, -6], 2) == ref_key([0, 0, -6], 2)


def _mirror_key(orc, o, s, m):
    return orc.table_key(np.array(o) * np.array(m), s)


@pytest.mark.parametrize("nside", [1, 2, 4])
def test_entries_sum_and_order(orc, nside):
    rng = np.random.default_rng(12 + nside)
    keys = rng.integers(0, orc.NKEYS, 300)
    for k in keys:
        pix, cnt = orc.table_entry(nside, int(k))
        assert cnt.sum() == orc.TM ** 3            # weights sum to one
        assert np.all(np.diff(pix) > 0)            # sorted, unique
        assert np.all((pix >= 0) & (pix < 12 * nside * nside))
        assert np.all(cnt > 0)


@pytest.mark.parametrize("nside", [2, 4])
def test_small_nodes_land_in_their_pixel(orc, nside):
    """A node much smaller than a pixel maps to the pixel of its direction
    (up to the direction binning, which moves it by less than a bin)."""
    rng = np.random.default_rng(21)
    hits = total = 0
    for _ in range(400):
        o = rng.integers(-500, 501, 3)
        if np.abs(o).max() < 100:
            continue
        k = orc.table_key(o, 1)
        assert k % orc.TB == 0                     # psi bin 0 for a far leaf
        pix, cnt = orc.table_entry(nside, k)
        assert len(pix) <= 4
        total += 1
        hits += int(orc.ang2pix(nside, o.astype(float)) in set(pix.tolist()))
    assert hits >= 0.9 * total


@pytest.mark.parametrize("nside", [2, 4])
def test_mirror_symmetry(orc, nside):
    """Mirroring the node offset mirrors the pixel weights exactly."""
    rng = np.random.default_rng(31)
    for _ in range(200):
        s = int(2 ** rng.integers(0, 5))
        o = rng.integers(-60, 61, 3) * 2 + (s > 1)
        if not o.any():
            continue
        pix, cnt = orc.table_entry(nside, orc.table_key(o, s))
        for m in ([-1, 1, 1], [1, -1, 1], [1, 1, -1]):
            mpix, mcnt = orc.table_entry(nside, _mirror_key(orc, o, s, m))
            mapped = {orc.ang2pix(nside, orc.pix2vec(nside, int(p)) * np.array(m)): int(c)
                      for p, c in zip(pix, cnt)}
            assert mapped == {int(p): int(c) for p, c in zip(mpix, mcnt)}
