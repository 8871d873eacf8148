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
    if a.lanczos_iters:
        g.lanczos_ground(x, tol=1e-300, max_iter=a.lanczos_iters, prec=a.prec, refine=False)
    torch.cuda.synchronize()
    print(f"D={sb.dim} batch={sb.batch} pairs={len(sb.pairs)} flops/product={g.info['flops_per_matvec']:.4g}")


if __name__ == "__main__":
    main()
