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


def _radii(orc, nr, eta=2):
    return np.array([orc.radius(i, eta) for i in range(nr)])


def test_wg_is_a_normal_density(orc):
    """W_g (Eq. A1) normalised over the points inside its support is the
    normal density with variance 1/2 (scipy), renormalised there."""
    from scipy.stats import norm
    nr = 43
    r = _radii(orc, nr)
    rng = np.random.default_rng(7)
    assert orc.wg(0.0) == 1.0 and orc.wg(S3H) == 0.0 and orc.wg(-0.3) == orc.wg(0.3)
    for _ in range(200):
        d = rng.uniform(0.5, r[-1] * 0.999)
        h = 2.0 ** rng.integers(0, 6)
        w = orc.wg_weights(d, h, nr, 2)
        assert w.sum() == pytest.approx(1.0, abs=1e-13)
        x = (r - d) / h
        inside = np.abs(x) < S3H
        if not inside.any():
            continue
        want = norm.pdf(x[inside], scale=1 / math.sqrt(2.0))
        np.testing.assert_allclose(w[inside], want / want.sum(), rtol=1e-12)
        assert np.all(w[~inside] == 0.0)


def test_wf1_conditions(orc):
    """W_f,1 (App. A.3): flux at r = 0 exact, eps_{i+1}/eps_i = (d - r_i)/(r_{i+1} - d)."""
    nr = 43
    r = _radii(orc, nr)
    for d in np.random.default_rng(8).uniform(r[1], r[-1] * 0.999, 400):
        w = orc.wf1_split(d, nr, 2)
        i = np.searchsorted(r, d, side="right") - 1
        assert np.all(np.delete(w, [i, i + 1]) == 0.0) and np.all(w >= 0)
        assert np.sum(w[1:] / r[1:] ** 2) == pytest.approx(1.0 / d ** 2, rel=1e-12)
        assert w[i + 1] * (r[i + 1] - d) == pytest.approx(w[i] * (d - r[i]), rel=1e-12, abs=1e-15)


def test_wf2_flux_exact_at_target_and_previous_point(orc):
    """W_f,2 (App. A.3): the flux of the two mapped points equals that of
    the true source at r = 0 and at r_{i-1}; next to the target (i < 2)
    the two conditions coincide and W_f,3 is used."""
    nr = 43
    r = _radii(orc, nr)
    for d in np.random.default_rng(9).uniform(r[1], r[-1] * 0.999, 400):
        w = orc.wf2_split(d, nr, 2)
        i = np.searchsorted(r, d, side="right") - 1
        if i < 2:
            np.testing.assert_array_equal(w, orc.wf3_split(d, nr, 2))
            continue
        nz = np.nonzero(w)[0]
        assert set(nz) <= {i, i + 1} and np.all(w >= 0)
        assert np.sum(w[nz] / r[nz] ** 2) == pytest.approx(1.0 / d ** 2, rel=1e-11)
        rm = r[i - 1]
        assert np.sum(w[nz] / (r[nz] - rm) ** 2) == pytest.approx(1.0 / (d - rm) ** 2, rel=1e-11)


def test_wf3_general_linear_and_conserving(orc):
    """Generalised W_f,3 (Eq. A8-A10): the points in the node's support
    carry weights linear in their index, summing to one, with the flux at
    r = 0 exact; otherwise (too few points, a negative weight) the two-point
    W_f,3."""
    nr = 59
    r = _radii(orc, nr)
    rng = np.random.default_rng(10)
    n_general = 0
    for _ in range(600):
        d = rng.uniform(1.0, r[-1] * 0.999)
        h = 2.0 ** rng.integers(0, 7)
        w = orc.wf3n_weights(d, h, nr, 2)
        nz = np.nonzero(w)[0]
        assert np.all(w >= 0)
        assert w.sum() == pytest.approx(1.0, abs=1e-12)
        assert np.sum(w[1:] / r[1:] ** 2) == pytest.approx(1.0 / d ** 2, rel=1e-10)
        support = [i for i in range(1, nr) if abs(r[i] - d) < S3H * h]
        if len(nz) > 2:
            n_general += 1
            assert list(nz) == support
            np.testing.assert_allclose(np.diff(w[nz], 2), 0.0, atol=1e-13)
        else:
            np.testing.assert_array_equal(w, orc.wf3_split(d, nr, 2))
    assert n_general > 100


def test_flux_kernels_error_ranking(orc):
    """App. A, Fig. A3 set-up (sources on a ray with 10 points): W_f,2 gives
    the smallest flux errors at the other points, W_f,3 stays acceptable,
    and the smoothing kernel W_p (here h = d/2) is far worse than all the
    flux kernels."""
    nr = 10
    r = _radii(orc, nr)
    rng = np.random.default_rng(5)
    ds = rng.uniform(r[2], r[-1] * 0.999, 3000)
    med = {}
    for name, f in [("wf1", lambda d: orc.wf1_split(d, nr, 2)), ("wf2", lambda d: orc.wf2_split(d, nr, 2)),
                    ("wf3", lambda d: orc.wf3_split(d, nr, 2)), ("wp", lambda d: orc.wp_weights(d, 0.5 * d, nr, 2))]:
        errs = []
        for d in ds:
            w = f(d)
            nz = np.nonzero(w)[0]
            for j in range(1, nr):
                if r[j] >= d:
                    break
                if r[nz.min()] <= r[j]:
                    continue
                approx = np.sum(w[nz] / (r[nz] - r[j]) ** 2)
                errs.append(abs(approx - 1.0 / (d - r[j]) ** 2) * (d - r[j]) ** 2)
        med[name] = float(np.median(errs))
    assert med["wf2"] < min(med["wf1"], med["wf3"])
    assert med["wf3"] < 0.1
    assert med["wp"] > 5 * max(med["wf1"], med["wf2"], med["wf3"])
