"""Pin of the oracle against brute-force reverse ray tracing on a tiny grid
(theta_lim -> 0, so every cell is a leaf node).

Brute force: the straight line from the target centre to the source cell's
centre is sampled finely through the voxels, and the recombination loss per
steradian of the source, sum of alpha_B n^2 (D - s)^2 ds along it, is taken
from Q / 4 pi (the On-the-Spot balance of Sec. 2.5 along one line).  The
oracle treats the same problem on cones of solid angle 4 pi / N_PIX with
radial evaluation points, so it agrees in the mean and scatters per target
by the cone's angular extent and the radial resolution; where a source cell
spans several rays each ray subtracts the full per-steradian loss from its
share of the budget, so the comparison keeps sources whose cell lies in one
ray (zeta_g off, no earlier pass, a single source).
"""
import math

import numpy as np
import pytest

from workloads import ALPHA_B, PC_CM, Workload

N, BOX = 16, 4.0 * PC_CM
DX = BOX / N
TARGET = (7, 7, 7)


def absorbed_brute_force(nH, src, Q, nsamp=100000):
    t = np.array(TARGET) + 0.5
    s = np.array(src) + 0.5
    D = np.linalg.norm(s - t)
    u = (np.arange(nsamp) + 0.5) / nsamp
    idx = np.floor(t[None, :] + u[:, None] * (s - t)[None, :]).astype(int)
    n = nH[idx[:, 2], idx[:, 1], idx[:, 0]]
    loss = np.sum(ALPHA_B * n ** 2 * (D - u * D) ** 2) * (D / nsamp) * DX ** 3
    return loss / (Q / (4 * math.pi))


def media():
    z, y, x = np.meshgrid(np.arange(N) + 0.5, np.arange(N) + 0.5, np.arange(N) + 0.5, indexing="ij")
    r = np.sqrt((x - 7.5) ** 2 + (y - 7.5) ** 2 + (z - 7.5) ** 2)
    return {"uniform": np.full((N, N, N), 12.0),
            "shell": np.where((r >= 2.5) & (r < 5.0), 14.0, 3.0)}


@pytest.mark.parametrize("medium", ["uniform", "shell"])
def test_absorbed_fraction_matches_brute_force(orc, medium):
    nH = media()[medium]
    rng = np.random.default_rng(1)
    q = (TARGET[2] * N + TARGET[1]) * N + TARGET[0]
    rel = []
    for Q in (1e47, 4e46):
        for _ in range(120):
            src = tuple(int(v) for v in rng.integers(1, N - 1, 3))
            D = float(np.linalg.norm(np.array(src) - np.array(TARGET)))
            if D < 4.5 or D > 7.5:
                continue
            a_bf = absorbed_brute_force(nH, src, Q)
            if a_bf > 0.9:                      # fully absorbed: no relative measure
                continue
            for nside in (1, 2):
                o = 2 * np.array(src) + 1 - 2 * np.array(TARGET) - 1
                pix, _ = orc.table_entry(nside, orc.table_key(o, 1))
                if len(pix) != 1:
                    continue
                w = Workload("bf", N, BOX, nH, ((np.array(src) + 0.5) * DX)[None, :], np.array([Q]),
                             theta_lim=1e-9, theta_src=1e-9)
                F, _, _ = orc.Tree(w).solve_pass(orc.params_for(w, nside=nside, zeta_g=False), targets=[q])
                a_orc = 1.0 - F[0] / (Q / (4 * math.pi * (D * DX) ** 2))
                rel.append((a_orc - a_bf) / a_bf)
    rel = np.array(rel)
    assert rel.size > 60
    assert abs(np.median(rel)) < 0.12, np.median(rel)
    assert np.all(np.abs(rel) < 0.6), np.sort(np.abs(rel))[-3:]
