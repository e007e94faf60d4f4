"""Pins for the walk's boundary conditions (Sec. 2.8): periodic (nearest
copy of each node) and corner of symmetry (the original plus 7 mirror
images through the low corner)."""
import math

import numpy as np
import pytest

from workloads import ALPHA_B, PC_CM, Workload, lognormal_density, uniform_density, uniform_sources


def scene(N=8, n_src=3, seed=41, box_pc=2.0, **kw):
    box = box_pc * PC_CM
    rho = lognormal_density(N, seed, sigma_ln=1.0)
    xyz, q = uniform_sources(n_src, box, seed + 1, 45.0, 46.5)
    return Workload(f"bc{N}", N, box, rho, xyz, q, **kw)


def test_corner_equals_mirrored_full_grid_when_every_cell_is_a_leaf(orc):
    """With theta -> 0 every node the walk accepts is a cell, and the 7
    mirror images reproduce exactly the cells of the full mirrored grid:
    the corner-of-symmetry fluxes of the original equal the isolated fluxes
    of the (2N)^3 grid built by mirroring it, source copies included."""
    w = scene(theta_lim=1e-9)
    N, dx = w.N, w.dx
    F_c, _, ion_c = orc.Tree(w).solve_pass(orc.params_for(w, bc=orc.BC_CORNER))
    # the full grid spans [-L, L)^3; index i of the full axis is cell i - N
    full_rho = w.n_H
    for ax in range(3):
        full_rho = np.concatenate([np.flip(full_rho, axis=ax), full_rho], axis=ax)
    xyz, q = [], []
    for mask in range(8):
        sgn = np.array([-1.0 if (mask >> a) & 1 else 1.0 for a in range(3)])
        xyz.append(w.src_xyz * sgn)
        q.append(w.src_Q)
    wf = Workload("full", 2 * N, 2 * w.box_cm, full_rho, np.concatenate(xyz), np.concatenate(q), theta_lim=1e-9)
    tf = orc.Tree(wf, box_lo=(-w.box_cm, -w.box_cm, -w.box_cm))
    idx = np.arange(N ** 3)
    ix, iy, iz = idx % N, (idx // N) % N, idx // (N * N)
    targets = ((iz + N) * 2 * N + (iy + N)) * 2 * N + (ix + N)
    F_f, _, ion_f = tf.solve_pass(orc.params_for(wf), targets=targets)
    np.testing.assert_allclose(F_c, F_f, rtol=1e-11, atol=0)
    np.testing.assert_array_equal(ion_c, ion_f)


def test_periodic_translation_invariant_when_every_cell_is_a_leaf(orc):
    """With theta -> 0 the nearest copy of every cell depends only on its
    offset from the target modulo the box, so shifting the whole periodic
    scene (density and sources) shifts the fluxes with it."""
    w = scene(theta_lim=1e-9)
    N, dx = w.N, w.dx
    F, _, _ = orc.Tree(w).solve_pass(orc.params_for(w, bc=orc.BC_PERIODIC))
    shift = np.array([3, 5, 1])                     # cells, (x, y, z)
    w2 = scene(theta_lim=1e-9)
    w2.n_H = np.roll(w.n_H, shift=tuple(shift[::-1]), axis=(0, 1, 2))
    w2.src_xyz = np.mod(w.src_xyz + shift * dx, w.box_cm)
    F2, _, _ = orc.Tree(w2).solve_pass(orc.params_for(w2, bc=orc.BC_PERIODIC))
    F2 = F2.reshape(N, N, N)
    np.testing.assert_allclose(np.roll(F.reshape(N, N, N), shift=tuple(shift[::-1]), axis=(0, 1, 2)), F2,
                               rtol=1e-11)


def test_periodic_sees_sources_across_the_boundary(orc):
    """Negligible gas, one source near the low x face, periodic: a target
    near the high x face gets the flux of the nearest copy of the source,
    Q / (4 pi d^2) with d measured across the boundary."""
    N, box = 16, 4.0 * PC_CM
    dx = box / N
    src = np.array([1, 7, 8])
    w = Workload("thin", N, box, uniform_density(N, 1e-20), ((src + 0.5) * dx)[None, :], np.array([1e48]),
                 theta_src=1e-3)
    t = orc.Tree(w)
    tgt = np.array([14, 7, 8])
    q = int((tgt[2] * N + tgt[1]) * N + tgt[0])
    F_p, _, _ = t.solve_pass(orc.params_for(w, bc=orc.BC_PERIODIC), targets=[q])
    F_i, _, _ = t.solve_pass(orc.params_for(w), targets=[q])
    d_wrap = (N - (tgt[0] - src[0])) * dx
    d_direct = (tgt[0] - src[0]) * dx
    assert F_p[0] == pytest.approx(1e48 / (4 * math.pi * d_wrap ** 2), rel=1e-9)
    assert F_i[0] == pytest.approx(1e48 / (4 * math.pi * d_direct ** 2), rel=1e-9)


def test_corner_stromgren_octant(orc):
    """Corner of symmetry with one eighth of a Strömgren sphere (the
    effective-resolution use of Sec. 2.8): a source of Q/8 in the corner
    cell of a uniform 16^3 octant gives an ionised volume of one eighth of
    the sphere of radius R_S(Q) (Eq. 17), within the radial resolution of
    the rays (ζ_g off)."""
    N, box = 16, 4.0 * PC_CM
    dx = box / N
    Q, n = 1e49, 300.0
    w = Workload("oct", N, box, uniform_density(N, n), np.array([[0.5 * dx] * 3]), np.array([Q / 8]),
                 theta_src=1e-2)
    F, _, ion = orc.Tree(w).solve_pass(orc.params_for(w, zeta_g=False, bc=orc.BC_CORNER))
    rs = (3 * Q / (4 * math.pi * n ** 2 * ALPHA_B)) ** (1 / 3) / dx
    r_eff = (3 * 8 * ion.sum() / (4 * math.pi)) ** (1 / 3)
    i = math.sqrt(2 * 2 ** 2 * rs)
    half_seg = 0.5 * (2 * i + 1) / (2 * 2 ** 2)
    assert abs(r_eff - rs) < max(1.0, half_seg), (r_eff, rs)
