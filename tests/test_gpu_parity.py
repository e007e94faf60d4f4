"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Bars: bit-exact table entries and tree topology (FP64 node masses and
centres); accepted-node lists bit-exact in every form (the FP32 forms re-take
in FP64 every opening decision FP32 cannot settle); ray bins within 1e-12
(FP64) and 2e-5 (FP32 forms); cell flux within 1e-5 (FP64) and 1e-3 (both
FP32 forms) away from the ionisation front, with the ionised/neutral
classification identical except within one cell of the front.  No fraction
of the cells is exempt from these bars, at any size.
"""
import json
import math

import numpy as np
import pytest

from helpers import KAPPA, flux_misses, interior_mask
from oracle_pool import oracle_free, oracle_pass, sampled_check, uniform_neighbours
from workloads import Workload, PC_CM, lognormal_density, uniform_density, uniform_sources, workload

pytestmark = pytest.mark.gpu

RTOL = {0: 1e-5, 1: 1e-3, 2: 1e-3}
FORMS = [0, 1, 2]


@pytest.fixture(scope="module")
def B():
    import torch
    import paper_2105_09644_gb300 as pkg
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    pkg.build()
    from paper_2105_09644_gb300 import binding
    binding.load()
    return binding


def dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def small_turbulent(N=32, n_src=6, seed=7, box_pc=4.0, **kw):
    box = box_pc * PC_CM
    rho = lognormal_density(N, seed)
    xyz, q = uniform_sources(n_src, box, seed + 1, 46.0, 48.5)
    return Workload(f"turb{N}", N, box, rho, xyz, q, seed=seed, **kw)


def gpu_params(B, w, precision=0, zeta_g=True, **kw):
    d = dict(theta_lim=w.theta_lim, theta_if=w.theta_if, theta_src=w.theta_src, nside=w.nside,
             eta_r=w.eta_r, alpha_B=w.alpha_B, hnu=w.hnu, precision=precision, zeta_g=int(zeta_g))
    d.update(kw)
    return B.tr_params_default(**d)


def gpu_tree(B, w, precision=0, e_prev=None, **kw):
    import torch
    keep = [dev(w.n_H), dev(w.src_xyz), dev(w.src_Q)]
    ep = dev(e_prev.reshape(w.N, w.N, w.N)) if e_prev is not None else None
    nd = dev(w.ndot_cell) if w.ndot_cell is not None else None
    g = B.make_grid(keep[0], w.dx, ndot=nd, e_prev=ep)
    s = B.make_sources(keep[1], keep[2])
    t = B.tr_build_tree(g, s, gpu_params(B, w, precision, **kw))
    torch.cuda.synchronize()
    t._keep = keep + [ep, nd]
    return t


def gpu_solve(B, w, precision=0, e_prev=None, **kw):
    import torch
    ep = dev(e_prev.reshape(w.N, w.N, w.N)) if e_prev is not None else None
    nd = dev(w.ndot_cell) if w.ndot_cell is not None else None
    F, e, ion, it, dl = B.solve(dev(w.n_H), w.dx, dev(w.src_xyz), dev(w.src_Q), ndot=nd, e_prev=ep,
                                **{k: v for k, v in gpu_params_dict(w, precision, **kw).items()})
    torch.cuda.synchronize()
    return F.cpu().numpy().ravel(), e.cpu().numpy().ravel(), ion.cpu().numpy().ravel()


def gpu_params_dict(w, precision=0, zeta_g=True, **kw):
    d = dict(theta_lim=w.theta_lim, theta_if=w.theta_if, theta_src=w.theta_src, nside=w.nside,
             eta_r=w.eta_r, alpha_B=w.alpha_B, hnu=w.hnu, precision=precision, zeta_g=int(zeta_g))
    d.update(kw)
    return d


def compare_fields(F, ion, F_orc, ion_orc, N, rtol, kappa=0.0, free_fn=None):
    """Every cell away from the oracle's front: the oracle's class, the flux
    within rtol (FP32 forms: within the conditioning bound where the plain
    bar is missed; free_fn(cell indices) gives the oracle's unattenuated
    flux), exactly zero where the oracle's is."""
    inner = interior_mask(ion_orc.reshape(N, N, N)).ravel()
    bad = np.nonzero(ion[inner] != ion_orc[inner])[0]
    assert bad.size == 0, f"{bad.size} cells away from the front change class"
    lit = np.nonzero(inner & (F_orc > 0))[0]
    if lit.size:
        err = np.abs(F[lit] - F_orc[lit]) / F_orc[lit]
        miss = flux_misses(F[lit], F_orc[lit], rtol, kappa, None if free_fn is None else (lambda k: free_fn(lit[k])))
        worst = lit[np.argsort(-err)[:3]]
        assert miss.size == 0, (f"{miss.size} cells miss the flux bar; max rel error {err.max():.3e} > {rtol} "
                                f"(median {np.median(err):.2e}), worst cells {worst.tolist()}")
    dark = inner & (F_orc == 0)
    assert np.all(F[dark] == 0.0)
    # cells that differ in class lie within one cell of the oracle's front
    diff = ion != ion_orc
    assert not np.any(diff & inner)
    stats = {"cells": int(ion.size), "interior_lit": int(lit.size),
             "rel_err_max": float(err.max()) if lit.size else 0.0,
             "rel_err_p99": float(np.percentile(err, 99)) if lit.size else 0.0,
             "rel_err_median": float(np.median(err)) if lit.size else 0.0,
             "class_flips_at_front": int(diff.sum()), "front_cells": int((~inner).sum())}
    print("field errors vs oracle:", json.dumps(stats))
    return stats


# --------------------------------------------------------------------------

@pytest.mark.parametrize("nside", [1, 2, 4])
def test_table_bit_exact(B, orc, nside):
    import torch
    nkeys, nent = B.tr_table_info(nside)
    assert nkeys == orc.NKEYS
    off = torch.empty(nkeys + 1, dtype=torch.int32, device="cuda")
    pix = torch.empty(nent, dtype=torch.int32, device="cuda")
    cnt = torch.empty(nent, dtype=torch.int32, device="cuda")
    B.tr_table_export(nside, off, pix, cnt)
    torch.cuda.synchronize()
    off, pix, cnt = off.cpu().numpy(), pix.cpu().numpy(), cnt.cpu().numpy()
    mismatches = []
    for k in range(nkeys):
        p, c = orc.table_entry(nside, k)
        gp, gc = pix[off[k]:off[k + 1]], cnt[off[k]:off[k + 1]]
        if not (np.array_equal(p, gp) and np.array_equal(c, gc)):
            mismatches.append(k)
    assert not mismatches, f"{len(mismatches)} of {nkeys} keys differ, first {mismatches[:5]}"


@pytest.mark.parametrize("precision", [0, 1])
def test_tree_nodes(B, orc, precision):
    import torch
    w = small_turbulent(N=16)
    rng = np.random.default_rng(3)
    e_prev = rng.uniform(0, 1e-9, w.N ** 3) * (rng.random(w.N ** 3) < 0.4)
    t = gpu_tree(B, w, precision, e_prev=e_prev)
    info = t.info()
    out = torch.empty((info["n_nodes"], 8), dtype=torch.float64, device="cuda")
    B.tr_tree_nodes(t, out)
    torch.cuda.synchronize()
    out = out.cpu().numpy()
    ot = orc.Tree(w, e_prev=e_prev)
    L = info["levels"] - 1
    assert L == 4
    off = 0
    for level in range(L + 1):
        n = 2 ** level
        for m in range(n ** 3):
            ix = iy = iz = 0
            for b in range(level):
                ix |= ((m >> (3 * b)) & 1) << b
                iy |= ((m >> (3 * b + 1)) & 1) << b
                iz |= ((m >> (3 * b + 2)) & 1) << b
            want = ot.node(level, ix, iy, iz)
            got = out[off + m]
            if precision == 0:
                assert np.array_equal(got[:4], want[:4]), (level, m, got[:4], want[:4])   # m, centre of mass
                np.testing.assert_allclose(got[4:], want[4:], rtol=1e-13, atol=1e-300)
            else:
                np.testing.assert_allclose(got[:4], want[:4], rtol=2e-6)
                np.testing.assert_allclose(got[4:], want[4:], rtol=2e-6, atol=1e-30 + 1e-6 * np.abs(want[4:]).max())
        off += n ** 3


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("theta,theta_src", [(0.5, math.inf), (0.3, 0.2), (1.0, 0.5)])
def test_walk_lists_and_bins(B, orc, theta, theta_src, precision):
    """Accepted-node lists bit-exact in both walks (the FP32 walk re-takes in
    FP64 what FP32 cannot settle); bins to 1e-12 (FP64) or 2e-5 (FP32)."""
    import torch
    w = small_turbulent(N=32, theta_lim=theta, theta_src=theta_src)
    t = gpu_tree(B, w, precision)
    rng = np.random.default_rng(11)
    targets = np.unique(np.concatenate([rng.integers(0, w.N ** 3, 40), [0, w.N ** 3 - 1]]))
    r = B.tr_walk_map(t, dev(targets.astype(np.int64)))
    info = r.info()
    nt, npix, nr, cap = info["n_targets"], info["npix"], info["nr"], info["acc_cap"]
    a = torch.empty((nt, npix, nr), dtype=torch.float64, device="cuda")
    e = torch.empty_like(a)
    ids = torch.empty((nt, cap), dtype=torch.int64, device="cuda")
    counts = torch.empty(nt, dtype=torch.int32, device="cuda")
    B.tr_rays_export(r, a, e, None, ids, counts)
    torch.cuda.synchronize()
    a, e, ids, counts = a.cpu().numpy(), e.cpu().numpy(), ids.cpu().numpy(), counts.cpu().numpy()
    ot = orc.Tree(w)
    p = orc.params_for(w)
    tol = 1e-12 if precision == 0 else 2e-5
    for k, tgt in enumerate(targets):
        res = ot.walk(p, int(tgt))
        assert counts[k] == res["n_accepted"]
        assert np.array_equal(np.sort(ids[k, :counts[k]]), np.sort(res["accepted"]))
        scale = max(res["alpha"].max(), 1e-300)
        np.testing.assert_allclose(a[k], res["alpha"], rtol=tol, atol=tol * scale)
        escale = max(res["eps"].max(), 1e-300)
        np.testing.assert_allclose(e[k], res["eps"], rtol=tol, atol=tol * escale)


def test_fp32_lists_with_if_mac(B, orc):
    """The IF MAC of the FP32 walk (ionised mass from a previous pass,
    delta_IF = 1e-8, decided on the FP64 masses when the tree is built):
    accepted lists bit-exact with the oracle."""
    import torch
    w = small_turbulent(N=32, theta_lim=0.5, theta_src=0.3)
    w.theta_if = 0.2
    F0, _, _ = orc.Tree(w).solve_pass(orc.params_for(w))
    e_prev = F0 * w.hnu / 2.99792458e10
    t = gpu_tree(B, w, 1, e_prev=e_prev)
    rng = np.random.default_rng(12)
    targets = rng.integers(0, w.N ** 3, 60).astype(np.int64)
    r = B.tr_walk_map(t, dev(targets))
    info = r.info()
    ids = torch.empty((info["n_targets"], info["acc_cap"]), dtype=torch.int64, device="cuda")
    counts = torch.empty(info["n_targets"], dtype=torch.int32, device="cuda")
    B.tr_rays_export(r, None, None, None, ids, counts)
    torch.cuda.synchronize()
    ids, counts = ids.cpu().numpy(), counts.cpu().numpy()
    ot = orc.Tree(w, e_prev=e_prev)
    p = orc.params_for(w)
    for k, tgt in enumerate(targets):
        res = ot.walk(p, int(tgt))
        assert np.array_equal(np.sort(ids[k, :counts[k]]), np.sort(res["accepted"]))


@pytest.mark.parametrize("name", ["stromgren32", "turbulent32"])
@pytest.mark.parametrize("precision", FORMS)
def test_solve_matches_oracle(B, orc, name, precision):
    w = workload(name, theta_src=0.25) if name == "stromgren32" else workload(name)
    F, e, ion = gpu_solve(B, w, precision)
    ot, p = orc.Tree(w), orc.params_for(w)
    F_orc, e_orc, ion_orc = ot.solve_pass(p)
    compare_fields(F, ion, F_orc, ion_orc, w.N, RTOL[precision], KAPPA[precision],
                   lambda c: ot.free_flux(p, targets=c))
    np.testing.assert_allclose(e, F * w.hnu / 2.99792458e10, rtol=1e-14)


@pytest.mark.parametrize("precision", FORMS)
def test_unfused_equals_fused(B, precision):
    """tr_walk_map + tr_ray_sweep reproduces tr_solve: to rounding in FP64
    (its deposits are atomic adds in any order), bit for bit in the FP32
    forms (their fixed-point deposits do not depend on the order)."""
    import torch
    w = small_turbulent(N=16, theta_src=0.3)
    F, e, ion = gpu_solve(B, w, precision)
    t = gpu_tree(B, w, precision)
    r = B.tr_walk_map(t, None, n_targets=w.N ** 3)
    F2 = torch.empty(w.N ** 3, dtype=torch.float64, device="cuda")
    e2 = torch.empty_like(F2)
    ion2 = torch.empty(w.N ** 3, dtype=torch.uint8, device="cuda")
    B.tr_ray_sweep(r, F2, e2, ion2)
    torch.cuda.synchronize()
    if precision == 0:
        compare_fields(F2.cpu().numpy(), ion2.cpu().numpy(), F, ion, w.N, 1e-12)
    else:
        assert np.array_equal(F2.cpu().numpy(), F) and np.array_equal(ion2.cpu().numpy(), ion)


@pytest.mark.parametrize("precision", FORMS)
def test_repeatable(B, precision):
    """FP64: two runs agree to rounding (the order of the FP64 atomic
    deposits varies).  FP32 forms: bit for bit (fixed-point deposits)."""
    w = small_turbulent(N=32)
    a = gpu_solve(B, w, precision)
    b = gpu_solve(B, w, precision)
    if precision == 0:
        compare_fields(a[0], a[2], b[0], b[2], w.N, 1e-12)
    else:
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[2], b[2])


@pytest.mark.parametrize("case", ["N8", "no_sources", "outside", "nside1", "nside4", "eta1", "eta4",
                                  "lray", "zeta_g_off", "e_prev_if", "diffuse"])
def test_edge_cases(B, orc, case):
    kw = {}
    w = small_turbulent(N=16, theta_src=0.3)
    e_prev = None
    pkw = {}
    if case == "N8":
        w = small_turbulent(N=8, n_src=2)
    elif case == "no_sources":
        w.src_xyz, w.src_Q = np.zeros((0, 3)), np.zeros(0)
    elif case == "outside":
        w.src_xyz = np.array([[-1.0, 0.5, 0.5], [2.0, 1.1, 0.3]]) * w.box_cm
        w.src_Q = np.array([1e48, 3e47])
    elif case == "nside1":
        w.nside, w.theta_lim = 1, 1.0
    elif case == "nside4":
        w.nside, w.theta_lim = 4, 0.25
    elif case == "eta1":
        w.eta_r = 1
    elif case == "eta4":
        w.eta_r = 4
    elif case == "lray":
        pkw["L_ray_cm"] = 6.0 * w.dx
    elif case == "zeta_g_off":
        kw["zeta_g"] = False
    elif case == "e_prev_if":
        F0, _, _ = orc.Tree(w).solve_pass(orc.params_for(w))
        e_prev = F0 * w.hnu / 2.99792458e10
        w.theta_if = 0.2
    elif case == "diffuse":
        w.ndot_cell = 1e45 * (w.n_H / w.n_H.mean()) ** 2
    zg = kw.get("zeta_g", True)
    lray_cells = pkw.get("L_ray_cm", 0.0) / w.dx
    ot = orc.Tree(w, e_prev=e_prev)
    p = orc.params_for(w, zeta_g=zg, lray_cells=lray_cells)
    F_orc, _, ion_orc = ot.solve_pass(p)
    for precision in FORMS:
        F, e, ion = gpu_solve(B, w, precision, e_prev=e_prev, zeta_g=zg, **pkw)
        compare_fields(F, ion, F_orc, ion_orc, w.N, RTOL[precision], KAPPA[precision],
                       lambda c: ot.free_flux(p, targets=c))


def test_errors_are_reported(B):
    import torch
    n = torch.ones((12, 12, 12), dtype=torch.float64, device="cuda")
    with pytest.raises(B.TreeRayError) as ei:
        B.solve(n, 1e18)
    assert ei.value.status == B.TR_EINVAL
    n = torch.ones((16, 16, 16), dtype=torch.float64, device="cuda")
    with pytest.raises(B.TreeRayError) as ei:
        B.solve(n, 1e18, nside=3)
    assert ei.value.status == B.TR_EINVAL


_FULL = {}


def oracle_full_field(name):
    """The oracle's single pass over every cell of a workload, over the host
    cores (computed once per test session)."""
    if name not in _FULL:
        w = workload(name)
        F, e, ion = oracle_pass("uniform", name, np.arange(w.N ** 3), nproc=None)
        _FULL[name] = (F, ion)
    return _FULL[name]


@pytest.mark.slow
@pytest.mark.parametrize("precision", FORMS)
def test_full_size_turbulent128_every_cell(B, precision):
    """The bench workload at full size (128^3, N_PIX = 48, N_R = 43), every
    cell against the oracle: the same bars as the small cases, no cell
    exempt except the front band."""
    w = workload("turbulent128")
    F, e, ion = gpu_solve(B, w, precision)
    F_orc, ion_orc = oracle_full_field("turbulent128")
    compare_fields(F, ion, F_orc, ion_orc, w.N, RTOL[precision], KAPPA[precision],
                   lambda c: oracle_free("uniform", "turbulent128", c))


@pytest.mark.slow
@pytest.mark.parametrize("name", ["sourcecount256_s100", "sourcecount256_s10000"])
@pytest.mark.parametrize("precision", [1, 2])
def test_full_size_sourcecount256_sampled(B, name, precision):
    """The 256^3 source-count workloads (30 pc box, N_R = 59), FP32 forms:
    sampled targets and their face neighbours against the oracle; every
    sampled cell away from the oracle's front meets the bar."""
    w = workload(name)
    F, e, ion = gpu_solve(B, w, precision)
    rng = np.random.default_rng(256)
    targets = rng.choice(w.N ** 3, 60, replace=False).astype(np.int64)
    nb = uniform_neighbours(targets, w.N)
    checked, worst = sampled_check(F, ion, targets, nb, lambda c: oracle_pass("uniform", name, c, nproc=8),
                                   RTOL[precision], KAPPA[precision], lambda c: oracle_free("uniform", name, c, nproc=8))
    assert checked >= 30


def test_bins_beyond_shared_memory_are_refused(B):
    """Ray bins larger than a CTA's shared memory (here N_PIX 192 with
    N_R 127 from a long L_ray) give TR_EUNSUPPORTED with a message, and the
    library stays usable."""
    import torch
    w = small_turbulent(N=16)
    n = dev(w.n_H)
    with pytest.raises(B.TreeRayError) as ei:
        B.solve(n, w.dx, nside=4, L_ray_cm=2000.0 * w.dx)
    assert ei.value.status == B.TR_EUNSUPPORTED and "shared memory" in str(ei.value)
    F, e, ion, it, dl = B.solve(n, w.dx)
    torch.cuda.synchronize()
    assert torch.isfinite(F).all()
