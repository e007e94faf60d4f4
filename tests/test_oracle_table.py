"""Pins for the node->ray table (Sec. 2.3 first mapping step)."""
import math
from fractions import Fraction

import numpy as np
import pytest


def ref_key(o, s, TQH=16, TQ=33, TB=40):
    """Key from exact rational arithmetic (independent of the C integer code):
    a face key when one axis dominates, an edge key for a two-axis tie, a
    corner key for a three-axis tie."""
    NF, NE = 6 * TQ * TQ * TB, 12 * TQ * TB
    ab = [abs(x) for x in o]
    A = max(ab)
    tied = [i for i in range(3) if ab[i] == A]

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
    if len(tied) == 1:
        a = tied[0]
        b, c = [i for i in range(3) if i != a]
        face = 2 * a + (1 if o[a] < 0 else 0)
        return ((face * TQ + fb(o[b])) * TQ + fb(o[c])) * TB + pb
    if len(tied) == 2:
        a, b = tied
        c = 3 - a - b
        pair = {(0, 1): 0, (0, 2): 1, (1, 2): 2}[(a, b)]
        edge = 4 * pair + 2 * (o[a] < 0) + (o[b] < 0)
        return NF + (edge * TQ + fb(o[c])) * TB + pb
    corner = (o[0] < 0) + 2 * (o[1] < 0) + 4 * (o[2] < 0)
    return NF + NE + corner * TB + pb


def test_key_matches_exact_rational(orc):
    rng = np.random.default_rng(11)
    for _ in range(3000):
        s = int(2 ** rng.integers(0, 7))
        o = rng.integers(-400, 401, 3)
        if not o.any():
            continue
        assert orc.table_key(o, s) == ref_key([int(x) for x in o], s)
    # ties between axes give edge and corner keys; centre bins for zero offsets
    for o in ([4, 4, 4], [-4, 4, -4], [6, -6, 1], [0, 3, -3], [5, 2, 5], [0, 0, -6]):
        assert orc.table_key(o, 1) == ref_key(o, 1)
    assert orc.table_key([4, 4, 1], 1) >= orc.NFACEKEYS
    assert orc.table_key([4, 4, 4], 1) >= orc.NFACEKEYS + orc.NEDGEKEYS


def _mirror_key(orc, o, s, m):
    return orc.table_key(np.array(o) * np.array(m), s)


@pytest.mark.parametrize("nside", [1, 2, 4])
def test_entries_sum_and_order(orc, nside):
    rng = np.random.default_rng(12 + nside)
    keys = rng.integers(0, orc.NKEYS, 300)
    for k in keys:
        pix, cnt = orc.table_entry(nside, int(k))
        assert cnt.sum() == orc.TW                 # weights sum to one
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


@pytest.mark.parametrize("nside", [1, 2, 4])
def test_diagonal_mirror_symmetry(orc, nside):
    """The reflections through the planes x = y and x = -y are symmetries of
    the HEALPix pixels; mirroring a node offset through them mirrors its
    pixel weights exactly -- for ordinary offsets and for the ties (nodes on
    the diagonal planes, whose edge and corner keys split each sample
    between a pixel and its mirror).  Without this, a scene symmetric about
    x = y (Sec. 3.4) would not give a symmetric field."""
    rng = np.random.default_rng(41)
    offsets = []
    for _ in range(150):
        s = int(2 ** rng.integers(0, 5))
        o = rng.integers(-60, 61, 3) * 2 + (s > 1)
        offsets.append((o, s))
        t = rng.integers(-60, 61) * 2 + (s > 1)
        offsets.append((np.array([t, t * rng.choice([-1, 1]), rng.integers(-abs(t), abs(t) + 1)]), s))
        offsets.append((np.array([t, t * rng.choice([-1, 1]), t * rng.choice([-1, 1])]), s))
    for o, s in offsets:
        if not o.any():
            continue
        pix, cnt = orc.table_entry(nside, orc.table_key(o, s))
        for tsgn in (1, -1):
            mo = np.array([tsgn * o[1], tsgn * o[0], o[2]])
            mpix, mcnt = orc.table_entry(nside, orc.table_key(mo, s))
            mapped = {}
            for p_, c_ in zip(pix, cnt):
                v = orc.pix2vec(nside, int(p_))
                k = orc.ang2pix(nside, np.array([tsgn * v[1], tsgn * v[0], v[2]]))
                mapped[k] = mapped.get(k, 0) + int(c_)
            assert mapped == {int(p_): int(c_) for p_, c_ in zip(mpix, mcnt)}, (o, s, tsgn)
