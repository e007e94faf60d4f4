"""Pins for evaluation points (Eq. 4-5) and radial kernels (App. A)."""
import json
import math
import os

import numpy as np
import pytest

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))
S3H = math.sqrt(3.0) / 2.0


def test_num_points_configs(orc):
    # Eq. 5 for the three uniform workloads (box diagonal in cells = N sqrt 3)
    assert orc.num_points(2, 32 * math.sqrt(3)) == GOLD["stromgren32_segments"]["value"] + 1
    assert orc.num_points(2, 128 * math.sqrt(3)) == 43
    assert orc.num_points(2, 256 * math.sqrt(3)) == 59
    assert orc.num_points(1, 128 * math.sqrt(3)) == 22
    assert orc.num_points(8, 32 * math.sqrt(3)) == 81


def test_radii(orc):
    # Eq. 4 with dx = 1 cell; r_20 = 12.5 pc for the 8 pc / 32^3 Strömgren box
    assert orc.radius(0, 2) == 0.0
    assert orc.radius(20, 2) * 0.25 == 12.5
    r = np.array([orc.radius(i, 2) for i in range(60)])
    seg = np.diff(r)
    assert np.all(seg > 0)
    # segment length grows linearly: (2i+1) dx / (2 eta^2)
    np.testing.assert_allclose(seg, (2 * np.arange(59) + 1) / 8.0)


def test_wp_constraints(orc):
    c = GOLD["wp_constants"]["value"]
    h = 1e-6
    assert orc.wp(0.0) == pytest.approx(c["M"], abs=1e-15)
    assert (orc.wp(h) - orc.wp(0.0)) / h == pytest.approx(0.0, abs=1e-4)      # W'(0) = 0
    assert orc.wp(0.5 - 1e-12) == pytest.approx(c["A"], abs=1e-9)            # continuity at 1/2
    assert orc.wp(0.5) == pytest.approx(c["A"], abs=1e-12)
    assert orc.wp(S3H) == 0.0
    assert orc.wp(S3H - 1e-9) == pytest.approx(0.0, abs=1e-12)               # zero at the edge
    slopes = [(orc.wp(S3H - e) - orc.wp(S3H - 2 * e)) / e for e in (1e-3, 1e-4, 1e-5)]
    assert abs(slopes[2]) < 1e-3 and abs(slopes[1]) < 0.11 * abs(slopes[0])   # slope -> 0 at the edge
    assert orc.wp(0.9) == 0.0 and orc.wp(2.0) == 0.0
    xs = np.linspace(0, 0.86, 50)
    assert all(orc.wp(x) == orc.wp(-x) for x in xs)
    assert all(orc.wp(x) > 0 for x in xs)
    # cubic leading coefficients as printed: a1 (inner) and a2 (outer branch)
    def lead(x0, x1):
        xs = np.linspace(x0, x1, 7)
        return np.polyfit(xs, [orc.wp(x) for x in xs], 3)[0]
    assert lead(0.05, 0.45) == pytest.approx(c["a1"], rel=1e-6)
    assert lead(0.55, 0.85) == pytest.approx(c["a2"], rel=1e-6)


def test_wp_weights_normalised(orc):
    rng = np.random.default_rng(3)
    nr = 43
    rlast = orc.radius(nr - 1, 2)
    for _ in range(200):
        d = rng.uniform(0.5, rlast * 1.05)
        h = 2.0 ** rng.integers(0, 6)
        w = orc.wp_weights(d, h, nr, 2)
        assert w.sum() == pytest.approx(1.0, abs=1e-13)
        assert np.all(w >= 0)
        if d >= rlast:
            assert w[-1] == 1.0
            continue
        r = np.array([orc.radius(i, 2) for i in range(nr)])
        inside = np.abs(r - d) / h < S3H
        if inside.any():
            assert np.all(w[~inside] == 0.0)
        else:   # linear split between the two bracketing points
            i = np.searchsorted(r, d, side="right") - 1
            assert w[i] + w[i + 1] == pytest.approx(1.0)
            assert w[i] * r[i] + w[i + 1] * r[i + 1] == pytest.approx(d)


def test_wf3_flux_exact(orc):
    """W_f,3: two points, sum = 1, flux at r = 0 exact (Eq. A3 with Eq. A6)."""
    rng = np.random.default_rng(4)
    nr = 43
    r = np.array([orc.radius(i, 2) for i in range(nr)])
    for d in rng.uniform(0.5, r[-1] * 0.999, 500):
        w = orc.wf3_split(d, nr, 2)
        nz = np.nonzero(w)[0]
        assert len(nz) <= 2
        assert w.sum() == pytest.approx(1.0, abs=1e-14)
        assert np.sum(w[1:] / r[1:] ** 2) == pytest.approx(1.0 / d ** 2, rel=1e-13)
        assert r[nz.min()] <= d <= r[nz.max()]
    # source exactly on an evaluation point goes there whole
    w = orc.wf3_split(r[10], nr, 2)
    assert w[10] == pytest.approx(1.0) and abs(w[11]) < 1e-15


def test_wf3_error_histogram_shape(orc):
    """App. A, Fig. A3 set-up: 10^4 source positions on a ray with 10 points.
    W_f,3 is exact at r = 0 and its flux error at the other points stays
    moderate (the paper finds it acceptable, second best after W_f,2)."""
    nr = 10
    r = np.array([orc.radius(i, 2) for i in range(nr)])
    rng = np.random.default_rng(5)
    errs = []
    for d in rng.uniform(r[2], r[-1] * 0.999, 10000):
        w = orc.wf3_split(d, nr, 2)
        for j in range(nr):
            if r[j] >= d:
                break
            if j == 0:
                continue
            # flux at r_j from the two mapped points (beyond r_j) vs the true source
            nz = np.nonzero(w)[0]
            if r[nz.min()] <= r[j]:
                continue
            approx = np.sum(w[nz] / (r[nz] - r[j]) ** 2)
            errs.append(abs(approx - 1.0 / (d - r[j]) ** 2) * (d - r[j]) ** 2)
    errs = np.array(errs)
    assert np.median(errs) < 0.1
