"""Continuous batching on the GPU: every request's result is the same alone
and in the mix (tr_walk_sweep_batch through the serving loop; to rounding in
FP64, whose deposits are FP64 atomics in any order, bit for bit in the FP32
forms), and the footprint that admission charges covers what a request
really allocates on the device."""
import math

import numpy as np
import pytest

from helpers import interior_mask
from workloads import PC_CM, lognormal_density, uniform_sources

pytestmark = pytest.mark.gpu

RTOL = {0: 1e-12, 1: 0.0, 2: 0.0}


@pytest.fixture(scope="module")
def B():
    import torch
    import paper_2105_09644_gb300 as pkg
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    pkg.build()
    from paper_2105_09644_gb300 import binding
    binding.load()
    return binding


def requests():
    from paper_2105_09644_gb300.serving import Request
    out = []
    rng = np.random.default_rng(77)
    for k, (N, nside, S) in enumerate([(16, 2, 3), (32, 1, 1), (8, 2, 5), (32, 2, 20), (16, 1, 2), (32, 2, 7)]):
        box = 4.0 * PC_CM
        rho = lognormal_density(N, 900 + k)
        xyz, q = uniform_sources(S, box, 950 + k, 46.0, 48.0)
        out.append(Request(k, 0.01 * k, N, box / N, rho, xyz, q, nside=nside,
                           theta_lim=1.0 if nside == 1 else 0.5, theta_src=0.3))
    return out


def alone(B, r, precision):
    import torch
    F, e, ion, _, _ = B.solve(torch.from_numpy(r.n_H).cuda(), r.dx, torch.from_numpy(r.src_xyz).cuda(),
                              torch.from_numpy(r.src_Q).cuda(), nside=r.nside, theta_lim=r.theta_lim,
                              theta_src=r.theta_src, precision=precision)
    torch.cuda.synchronize()
    return F.cpu().numpy(), ion.cpu().numpy()


@pytest.mark.parametrize("precision", [0, 1, 2])
def test_mix_equals_alone(B, precision):
    from paper_2105_09644_gb300.serving import Server
    reqs = requests()
    # a small tick forces requests to share launches and large ones to be sliced
    srv = Server(budget_bytes=1 << 30, tick_targets=6000, precision=precision)
    done = srv.run(reqs)
    assert len(done) == len(reqs) and srv.launches > len(reqs) // 2
    for r in reqs:
        F_a, ion_a = alone(B, r, precision)
        F_m, ion_m = r.result["F"], r.result["ion"]
        inner = interior_mask(ion_a)
        assert np.array_equal(ion_m[inner], ion_a[inner]), r.rid
        lit = inner & (F_a > 0)
        assert np.all(np.abs(F_m[lit] - F_a[lit]) <= RTOL[precision] * F_a[lit]), r.rid
        assert r.latency is not None and r.latency >= 0


def test_batch_entry_point_ranges(B):
    """Explicit ranges: two halves of one tree in one launch plus another tree."""
    import torch
    reqs = requests()
    r0, r1 = reqs[0], reqs[3]
    F0, ion0 = alone(B, r0, 1)
    F1, ion1 = alone(B, r1, 1)
    trees, outs = [], []
    for r in (r0, r1):
        n = torch.from_numpy(r.n_H).cuda()
        x, q = torch.from_numpy(r.src_xyz).cuda(), torch.from_numpy(r.src_Q).cuda()
        p = B.tr_params_default(nside=r.nside, theta_lim=r.theta_lim, theta_src=r.theta_src, precision=1)
        t = B.tr_build_tree(B.make_grid(n, r.dx), B.make_sources(x, q), p)
        t._keep = (n, x, q)
        trees.append(t)
        outs.append(torch.full((r.N,) * 3, -1.0, dtype=torch.float64, device="cuda"))
    n0 = r0.N ** 3
    B.tr_walk_sweep_batch([trees[0], trees[1], trees[0]], [0, 0, n0 // 3], [n0 // 3, r1.N ** 3, n0 - n0 // 3],
                          [outs[0], outs[1], outs[0]])
    torch.cuda.synchronize()
    assert np.allclose(outs[0].cpu().numpy(), F0, rtol=1e-6, atol=0)
    assert np.allclose(outs[1].cpu().numpy(), F1, rtol=1e-6, atol=0)


@pytest.mark.parametrize("precision", [0, 1])
def test_footprint_covers_allocations(B, precision):
    """Device memory taken by one request (inputs, outputs, tree, ray
    tables) against footprint_bytes: admission never under-counts, and
    over-counts by at most 2x + 64 MB (the device allocator packs small
    allocations that the model rounds up one by one)."""
    import torch
    from paper_2105_09644_gb300.serving import footprint_bytes
    for N, S in ((32, 10), (64, 300), (128, 1000)):
        box = 4.0 * PC_CM
        rho = lognormal_density(N, 5)
        xyz, q = uniform_sources(S, box, 6, 46.0, 48.0)
        p = B.tr_params_default(precision=precision)

        def one():
            d = [torch.from_numpy(a).cuda() for a in (rho, xyz, q)]
            out = [torch.empty((N,) * 3, dtype=torch.float64, device="cuda") for _ in range(2)]
            out.append(torch.empty((N,) * 3, dtype=torch.uint8, device="cuda"))
            t = B.tr_build_tree(B.make_grid(d[0], box / N), B.make_sources(d[1], d[2]), p)
            torch.cuda.synchronize()
            return d, out, t
        keep = one()                             # the node->ray table of N_side 2 is built and cached here
        del keep
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
        free0 = torch.cuda.mem_get_info()[0]
        keep = one()
        used = free0 - torch.cuda.mem_get_info()[0]
        fp = footprint_bytes(N, precision, S)
        assert used <= fp <= 2 * used + (64 << 20), (N, used, fp)
        del keep
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
