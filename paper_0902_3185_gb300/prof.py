"""Profiling driver: build a superblock and run a few products (for ncu).

python -m paper_0902_3185_gb300.prof --workload ladder_m1000 --prec bf16x3 --reps 3
"""
from __future__ import annotations

import argparse
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="ladder_m1000", choices=["ladder_m1000", "random64"])
    ap.add_argument("--batch", type=int, default=16)
    ap.add_argument("--prec", default="bf16x3", choices=["fp64", "tf32", "bf16x3"])
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--lanczos-iters", type=int, default=0, help="also run a fixed-length Lanczos")
    ap.add_argument("--autotune", action="store_true", help="autotune, then time eager and graph-captured products")
    a = ap.parse_args()
    import torch
    from paper_0902_3185_gb300.binding import GpuSuperblock
    from workloads.superblock import seeded_normal
    if a.workload == "ladder_m1000":
        from workloads.grown import ladder_m1000
        sb = ladder_m1000(batch=a.batch)
    else:
        from workloads.synthetic import random_sectored
        sb = random_sectored(seed=0, batch=a.batch)
    g = GpuSuperblock(sb)
    x = torch.from_numpy(np.stack([seeded_normal(b, sb.dim) for b in range(sb.batch)])).cuda()
    y = g.empty()
    for _ in range(a.reps):
        g.apply_H(x, y, prec=a.prec)
    if a.autotune and a.prec != "fp64":
        import json
        rep = g.autotune(prec=a.prec, reps=7)
        # products replayed from a CUDA graph (the library launches on the capturing stream)
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            for _ in range(2):
                g.apply_H(x, y, prec=a.prec)
        torch.cuda.current_stream().wait_stream(s)
        graph = torch.cuda.CUDAGraph()
        n_rep = 10
        with torch.cuda.graph(graph):
            for _ in range(n_rep):
                g.apply_H(x, y, prec=a.prec)
        graph.replay()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(5):
            graph.replay()
        e1.record()
        torch.cuda.synchronize()
        rep["graph_ms"] = e0.elapsed_time(e1) / (5 * n_rep)
        rep["flops"] = g.info["flops_per_matvec"]
        rep["tflops_best"] = rep["flops"] / (rep["best_ms"] * 1e-3) / 1e12
        rep["tflops_per_block"] = rep["flops"] / (rep["per_block_ms"] * 1e-3) / 1e12
        rep["workload"] = a.workload
        rep["prec"] = a.prec
        print(json.dumps(rep))
    if a.lanczos_iters:
        g.lanczos_ground(x, tol=1e-300, max_iter=a.lanczos_iters, prec=a.prec, refine=False)
    torch.cuda.synchronize()
    print(f"D={sb.dim} batch={sb.batch} pairs={len(sb.pairs)} flops/product={g.info['flops_per_matvec']:.4g}")


if __name__ == "__main__":
    main()
