"""The CPU oracle over many targets, split across host processes, and the
face neighbours that decide which sampled cells sit at an ionisation front.

Test infrastructure: the workers rebuild the named workload themselves (the
inputs come from `workloads`, whose generators are seeded) and run the
oracle's one-pass solve on their share of the targets.  The pool is started
with `spawn`, so it is safe after the parent has touched the GPU.
"""
from __future__ import annotations

import multiprocessing as mp
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(args):
    kind, spec, over, targets = args[:4]
    free = len(args) > 4 and args[4]
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    import oracle
    if kind == "uniform":
        from workloads import workload
        w = workload(spec, **over)
        t = oracle.Tree(w)
        p = oracle.params_for(w)
    elif kind == "scene":
        from workloads import scenes
        w = getattr(scenes, spec["fn"])(**spec.get("kw", {}))
        t = oracle.Tree(w)
        p = oracle.params_for(w, **over)
    else:
        from workloads.amr import amr_cluster
        w = amr_cluster(**spec)
        t = oracle.AmrTree(w)
        p = oracle.params_for(w, **over)
    if free:
        return t.free_flux(p, targets=np.asarray(targets, dtype=np.int64))
    return t.solve_pass(p, targets=np.asarray(targets, dtype=np.int64))


def processes(n_targets: int, per_process: int = 2000) -> int:
    return max(1, min(os.cpu_count() or 1, 16, (n_targets + per_process - 1) // per_process))


def oracle_pass(kind: str, spec, targets, over=None, nproc: int | None = None):
    """F, e, ion of the oracle's single pass at `targets` (cell indices).
    kind "uniform": spec is a workload name; "scene": spec = {"fn": a
    generator of workloads.scenes, "kw": its keyword arguments}; "amr": spec
    holds the keyword arguments of workloads.amr.amr_cluster."""
    targets = np.asarray(targets, dtype=np.int64)
    over = over or {}
    nproc = nproc or processes(targets.size)
    if nproc == 1:
        return _worker((kind, spec, over, targets))
    chunks = [c for c in np.array_split(targets, nproc) if c.size]
    with mp.get_context("spawn").Pool(len(chunks)) as pool:
        parts = pool.map(_worker, [(kind, spec, over, c) for c in chunks])
    return tuple(np.concatenate([p[k] for p in parts]) for k in range(3))


def oracle_free(kind: str, spec, targets, over=None, nproc: int | None = None):
    """The oracle's unattenuated flux at `targets` (see oracle_pass)."""
    targets = np.asarray(targets, dtype=np.int64)
    over = over or {}
    nproc = nproc or processes(targets.size)
    if nproc == 1 or targets.size < 64:
        return _worker((kind, spec, over, targets, True))
    chunks = [c for c in np.array_split(targets, nproc) if c.size]
    with mp.get_context("spawn").Pool(len(chunks)) as pool:
        parts = pool.map(_worker, [(kind, spec, over, c, True) for c in chunks])
    return np.concatenate(parts)


def uniform_neighbours(targets, N: int):
    """[n, 6] C-order indices of the face neighbours (-1 outside the box)."""
    t = np.asarray(targets, dtype=np.int64)
    x, y, z = t % N, (t // N) % N, t // (N * N)
    out = np.full((t.size, 6), -1, dtype=np.int64)
    k = 0
    for ax in range(3):
        for sh in (-1, 1):
            c = [x.copy(), y.copy(), z.copy()]
            c[ax] = c[ax] + sh
            ok = (c[ax] >= 0) & (c[ax] < N)
            out[ok, k] = ((c[2] * N + c[1]) * N + c[0])[ok]
            k += 1
    return out


def amr_neighbours(g, targets):
    """Face neighbours of AMR cells: for each target, the list of cells that
    touch one of its faces (cells of any size), from the cells painted onto
    the finest lattice."""
    N = g.N_fine
    owner = np.empty((N, N, N), dtype=np.int32)          # [z, y, x] -> cell index
    cid = np.arange(g.n_blocks * 512, dtype=np.int32).reshape(g.n_blocks, 8, 8, 8)
    for b in range(g.n_blocks):
        s = g.cell_size(b)
        x0, y0, z0 = 8 * s * g.blk_pos[b]
        blk = np.repeat(np.repeat(np.repeat(cid[b], s, 0), s, 1), s, 2)
        owner[z0:z0 + 8 * s, y0:y0 + 8 * s, x0:x0 + 8 * s] = blk
    out = []
    for t in np.asarray(targets, dtype=np.int64):
        b, c = int(t) >> 9, int(t) & 511
        s = g.cell_size(b)
        corner = (8 * g.blk_pos[b] + np.array([c & 7, (c >> 3) & 7, c >> 6])) * s      # [x, y, z]
        nb = set()
        for ax in range(3):
            for side in (-1, s):
                p = corner[ax] + side
                if p < 0 or p >= N:
                    continue
                sl = [slice(corner[0], corner[0] + s), slice(corner[1], corner[1] + s), slice(corner[2], corner[2] + s)]
                sl[ax] = slice(p, p + 1)
                nb.update(np.unique(owner[sl[2], sl[1], sl[0]]).tolist())
        nb.discard(int(t))
        out.append(sorted(nb))
    return out


def sampled_check(F, ion, targets, nbrs, oracle_fn, rtol, kappa=0.0, free_fn=None):
    """Compare the GPU field at sampled targets with the oracle, cell by
    cell.  A sampled cell is at the front when the oracle puts one of its
    face neighbours in the other class; every other sampled cell must have
    the oracle's class and, if lit, its flux within rtol (FP32 forms: within
    rtol F + kappa (F_free - F) where the plain bar is missed, free_fn(cells)
    giving the oracle's unattenuated flux), or exactly zero flux if dark.
    No fraction of the sample is exempt.  oracle_fn(cells) returns the
    oracle's (F, e, ion) at those cells.  Returns the number of interior
    cells checked and the largest relative error."""
    targets = np.asarray(targets, dtype=np.int64)
    allc = np.unique(np.concatenate([targets] + [np.asarray(n, dtype=np.int64) for n in nbrs]))
    allc = allc[allc >= 0]
    Fo, _, io = oracle_fn(allc)
    pos = {int(c): k for k, c in enumerate(allc)}
    checked, worst = 0, 0.0
    bad = []
    for t, nb in zip(targets, nbrs):
        k = pos[int(t)]
        cls = io[k]
        if any(io[pos[int(n)]] != cls for n in nb if n >= 0):
            continue                                     # at the front: no bound holds there
        checked += 1
        if ion[t] != cls:
            bad.append((int(t), "class", int(ion[t]), int(cls)))
            continue
        if Fo[k] > 0:
            err = abs(F[t] - Fo[k]) / Fo[k]
            worst = max(worst, err)
            if err > rtol:
                bad.append((int(t), "flux", float(F[t]), float(Fo[k])))
        elif F[t] != 0.0:
            bad.append((int(t), "dark", float(F[t]), 0.0))
    flux_bad = [b for b in bad if b[1] == "flux"]
    if flux_bad and kappa > 0.0 and free_fn is not None:
        cells = np.array([b[0] for b in flux_bad], dtype=np.int64)
        Ff = np.asarray(free_fn(cells))
        keep = {int(c) for c, f, b in zip(cells, Ff, flux_bad)
                if abs(b[2] - b[3]) > rtol * b[3] + kappa * (f - b[3])}
        bad = [b for b in bad if b[1] != "flux" or b[0] in keep]
    assert not bad, f"{len(bad)} of {checked} interior sampled cells miss the bar: {bad[:5]}"
    return checked, worst
