"""Run the fused walk kernel on a named workload, for profiling.

python -m paper_2105_09644_gb300.walkprobe --workload turbulent64 --precision 1 --reps 2
python -m paper_2105_09644_gb300.walkprobe --workload amr_cluster --precision 1 --reps 2

Builds the tree once, then runs tr_walk_sweep `reps` times and prints the
walk counters and the mean time per launch (CUDA events).
"""
from __future__ import annotations

import argparse
import os
import sys


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="turbulent64")
    ap.add_argument("--precision", type=int, default=1)
    ap.add_argument("--reps", type=int, default=2)
    a = ap.parse_args(argv)
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if root not in sys.path:
        sys.path.insert(0, root)
    import torch
    from paper_2105_09644_gb300 import binding as B
    from workloads import workload
    B.load()
    if a.workload.startswith("amr"):
        from workloads.amr import amr_cluster
        # amr_cluster: base 64^3 refined twice (5.9 M cells); amr_mid: base 16^3 (161,792 cells)
        w = amr_cluster(N_base=16) if a.workload == "amr_mid" else amr_cluster()
        n = torch.from_numpy(w.n_H.ravel()).cuda()
        grid = B.make_amr_grid(w.N_base, w.max_level, w.blk_level, w.blk_pos, n, w.dx_fine)
        build = B.tr_build_tree_amr
        shape = (w.n_leaves,)
    else:
        w = workload(a.workload)
        n = torch.from_numpy(w.n_H).cuda()
        grid = B.make_grid(n, w.dx)
        build = B.tr_build_tree
        shape = (w.N,) * 3
    x = torch.from_numpy(w.src_xyz).cuda()
    q = torch.from_numpy(w.src_Q).cuda()
    tree = build(grid, B.make_sources(x, q),
                 B.tr_params_default(nside=w.nside, theta_lim=w.theta_lim, theta_if=w.theta_if,
                                     theta_src=w.theta_src, precision=a.precision))
    F = torch.empty(shape, dtype=torch.float64, device="cuda")
    E = torch.empty_like(F)
    ion = torch.empty(shape, dtype=torch.uint8, device="cuda")
    ms = []
    for _ in range(a.reps):
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record()
        B.tr_walk_sweep(tree, F, E, ion)
        e.record()
        torch.cuda.synchronize()
        ms.append(s.elapsed_time(e))
    print(a.workload, "precision", a.precision, B.tr_tree_stats(tree), tree.info(),
          "ms per launch", sum(ms) / len(ms))


if __name__ == "__main__":
    main()
