"""Pins for the oracle's HEALPix ring scheme (Sec. 2.2; Gorski et al. 2005)."""
import json
import math
import os

import numpy as np
import pytest

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


@pytest.mark.parametrize("nside", [1, 2, 4, 8])
def test_roundtrip_centres(orc, nside):
    npix = 12 * nside * nside
    assert GOLD["npix_for_nside"]["value"].get(str(nside), npix) == npix
    for p in range(npix):
        v = orc.pix2vec(nside, p)
        assert abs(np.linalg.norm(v) - 1.0) < 1e-12
        assert orc.ang2pix(nside, v) == p
        # a small perturbation of the centre stays in the pixel
        rng = np.random.default_rng(p)
        for _ in range(4):
            q = v + 1e-3 / nside * rng.standard_normal(3)
            assert orc.ang2pix(nside, q) == p


def test_base_pixels_golden(orc):
    zs = [orc.pix2vec(1, p)[2] for p in range(12)]
    np.testing.assert_allclose(zs, GOLD["healpix_nside1_centre_z"]["value"], atol=1e-12)
    phis = [(math.atan2(orc.pix2vec(1, p)[1], orc.pix2vec(1, p)[0]) / math.pi) % 2.0 for p in range(12)]
    phis = [0.0 if abs(x - 2.0) < 1e-9 else x for x in phis]
    np.testing.assert_allclose(phis, GOLD["healpix_nside1_centre_phi_over_pi"]["value"], atol=1e-9)


@pytest.mark.parametrize("nside", [1, 2, 4])
def test_equal_area(orc, nside):
    """Equal solid angle per pixel: uniform directions fill pixels evenly."""
    npix = 12 * nside * nside
    rng = np.random.default_rng(1234 + nside)
    n = 60000 if nside < 4 else 120000
    v = rng.standard_normal((n, 3))
    counts = np.zeros(npix)
    for x in v:
        counts[orc.ang2pix(nside, x)] += 1
    mean = n / npix
    sigma = math.sqrt(mean * (1 - 1 / npix))
    assert np.all(np.abs(counts - mean) < 5.0 * sigma), (counts.min(), counts.max(), mean)


@pytest.mark.parametrize("nside", [1, 2, 4, 8])
def test_centres_sum_to_zero_and_caps(orc, nside):
    npix = 12 * nside * nside
    V = np.array([orc.pix2vec(nside, p) for p in range(npix)])
    np.testing.assert_allclose(V.sum(axis=0), 0.0, atol=1e-9)
    # north polar cap (rings 1..N_side-1) holds 2 N_side (N_side - 1) pixels
    assert int(np.sum(V[:, 2] > 2.0 / 3.0 + 1e-12)) == 2 * nside * (nside - 1)


@pytest.mark.parametrize("nside", [2, 4])
def test_mirror_symmetries(orc, nside):
    """HEALPix is invariant under x->-x, y->-y and z->-z."""
    rng = np.random.default_rng(7)
    for v in rng.standard_normal((2000, 3)):
        p = orc.ang2pix(nside, v)
        for m in (np.array([-1, 1, 1]), np.array([1, -1, 1]), np.array([1, 1, -1])):
            pm = orc.ang2pix(nside, v * m)
            cm = orc.pix2vec(nside, p) * m
            assert orc.ang2pix(nside, cm) == pm
