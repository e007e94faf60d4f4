"""Pins for the column-density maps (cdMaps, Sec. 2.2): the same walk, each
accepted node adding w_k m / (Omega d^2) to direction k."""
import math

import numpy as np
import pytest

from workloads import PC_CM, Workload, lognormal_density, uniform_density
from workloads.amr import amr_cluster

from helpers import amr_cells


def test_cd_brute_force_when_every_cell_is_a_leaf(orc):
    """theta -> 0: every other cell is accepted, so sum_k Omega N_k equals
    the brute-force sum over cells of m_c / d_c^2 (times dx)."""
    N, box = 8, 2.0 * PC_CM
    dx = box / N
    rho = lognormal_density(N, 51, sigma_ln=1.0)
    w = Workload("cd", N, box, rho, np.zeros((0, 3)), np.zeros(0), theta_lim=1e-9)
    t = orc.Tree(w)
    for nside in (1, 2):
        p = orc.params_for(w, nside=nside)
        omega = 4 * math.pi / (12 * nside ** 2)
        z, y, x = np.meshgrid(np.arange(N), np.arange(N), np.arange(N), indexing="ij")
        for tgt in (0, 100, 511):
            cd = t.column_density(p, tgt)
            tx, ty, tz = tgt % N, (tgt // N) % N, tgt // (N * N)
            d2 = (x - tx) ** 2 + (y - ty) ** 2 + (z - tz) ** 2
            m = rho.copy()
            m[tz, ty, tx] = 0.0
            d2[tz, ty, tx] = 1
            want = np.sum(m / d2) * dx
            assert np.sum(cd) * omega == pytest.approx(want, rel=1e-12)
            assert np.all(cd >= 0)


def test_cd_uniform_box_is_density_times_path(orc):
    """Uniform gas: the column in each direction is n times the mean
    distance to the box wall over that pixel's cone (Monte Carlo over
    directions binned by HEALPix), less the target's own half cell and the
    tree's smoothing: within 10%."""
    N, box, n = 32, 4.0 * PC_CM, 100.0
    dx = box / N
    w = Workload("u", N, box, uniform_density(N, n), np.zeros((0, 3)), np.zeros(0), theta_lim=0.2)
    t = orc.Tree(w)
    tgt = (16 * N + 16) * N + 16
    c = np.array([16.5, 16.5, 16.5])
    rng = np.random.default_rng(0)
    v = rng.normal(size=(40000, 3))
    v /= np.linalg.norm(v, axis=1)[:, None]
    with np.errstate(divide="ignore"):
        R = np.min(np.abs(np.where(v > 0, (N - c) / v, -c / v)), axis=1)
    for nside in (1, 2):
        cd = t.column_density(orc.params_for(w, nside=nside, theta_lim=0.2), tgt) / (n * dx)
        pix = np.array([orc.ang2pix(nside, x) for x in v])
        Rk = np.array([R[pix == k].mean() for k in range(12 * nside ** 2)])
        ratio = cd / Rk
        assert np.all(ratio > 0.9) and np.all(ratio < 1.02), ratio


def test_cd_amr_brute_force_when_every_cell_is_a_leaf(orc):
    """The same identity on an AMR grid (cells of three sizes): mass
    n_H s^3 at each cell's centre."""
    g = amr_cluster(N_base=8, max_level=2, threshold=1000.0, n_src=0, box_pc=4.0, theta_lim=1e-9, nside=1)
    t = orc.AmrTree(g)
    p = orc.params_for(g)
    corner, size = amr_cells(g)
    cen = corner + 0.5 * size[:, None]
    m = g.n_H.ravel() * size.astype(float) ** 3
    omega = 4 * math.pi / 12
    for tgt in (0, int(np.argmax(size)), g.n_leaves - 1):
        cd = t.column_density(p, tgt)
        d2 = ((cen - cen[tgt]) ** 2).sum(axis=1)
        mask = np.arange(g.n_leaves) != tgt
        want = np.sum(m[mask] / d2[mask]) * g.dx_fine
        assert np.sum(cd) * omega == pytest.approx(want, rel=1e-12)
