"""Profiling driver: build a superblock and run a few products (for ncu).

python -m paper_0902_3185_gb300.prof --workload ladder_m1000 --prec bf16x3 --reps 3

The real config-5 superblock (the device DMRG's m = 1000 ladder, as bench.py
builds it), saved once and then profiled without the DMRG run:

python -m paper_0902_3185_gb300.prof --save-real /tmp/real.npz
python -m paper_0902_3185_gb300.prof --workload npz:/tmp/real.npz --prec bf16x3 --reps 3 [--step]

--step runs, after the products, one bench step (mixed solve with double-float
refinement and the gradient) inside the NVTX range "step" (ncu --nvtx
--nvtx-include "step/" captures exactly its launches).

--reorth J times only full Gram-Schmidt passes at Krylov index J (the
Lanczos kernels k_multidot, k_reduce_rows, k_multiaxpy; one untimed pass,
then --reps passes).

Recording the DRAM traffic of one product from an ncu capture of exactly its
launches (``ncu -i <rep> --page raw --csv > raw.csv``) for bench.py:

python -m paper_0902_3185_gb300.prof --record-traffic tensor_product_bf16x3 raw.csv
"""
from __future__ import annotations

import argparse
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


# kernel sources whose hash keys each traffic record (a change voids the record)
TRAFFIC_SOURCES = {
    "tensor_product_bf16x3": ["paper_0902_3185_gb300/csrc/matvec_tc.cu", "paper_0902_3185_gb300/csrc/tc_kernel.cuh"],
    "tensor_product_tf32": ["paper_0902_3185_gb300/csrc/matvec_tc.cu", "paper_0902_3185_gb300/csrc/tc_kernel.cuh"],
    "tensor_product_bf16x3_real": ["paper_0902_3185_gb300/csrc/matvec_tc.cu",
                                   "paper_0902_3185_gb300/csrc/tc_kernel.cuh"],
    "df64_product_real": ["paper_0902_3185_gb300/csrc/matvec_df.cu", "paper_0902_3185_gb300/csrc/df.cuh",
                          "paper_0902_3185_gb300/csrc/tc_kernel.cuh"],
    "fp64_product": ["paper_0902_3185_gb300/csrc/matvec_f64.cu"],
    "gram_schmidt_pass_bf16x3_real": ["paper_0902_3185_gb300/csrc/lanczos.cu", "paper_0902_3185_gb300/csrc/lanczos.h",
                                      "paper_0902_3185_gb300/csrc/df.cuh"],
    "df64_product": ["paper_0902_3185_gb300/csrc/matvec_df.cu", "paper_0902_3185_gb300/csrc/tc_kernel.cuh"],
}


def record_traffic(name, csv_path, note=""):
    import csv
    import hashlib
    import json
    rows = [r for r in csv.reader(open(csv_path)) if r and not r[0].startswith("==")]
    hdr = rows[0]
    scales = {"byte": 1.0, "kbyte": 1e3, "mbyte": 1e6, "gbyte": 1e9}
    total, launches = 0.0, 0
    if "Metric Name" in hdr:  # --csv --log-file: one row per (launch, metric)
        ids = set()
        for r in rows[1:]:
            d = dict(zip(hdr, r))
            if d.get("Metric Name") in ("dram__bytes_read.sum", "dram__bytes_write.sum"):
                total += float(d["Metric Value"].replace(",", "")) * scales[d["Metric Unit"].lower()]
                ids.add(d["ID"])
        launches = len(ids)
    else:  # --page raw --csv: one row per launch, units in the second row
        units = rows[1]
        for r in rows[2:]:
            d = dict(zip(hdr, r))
            for k in ("dram__bytes_read.sum", "dram__bytes_write.sum"):
                total += float(d[k]) * scales[units[hdr.index(k)].lower()]
            launches += 1
    h = hashlib.sha256()
    for f in TRAFFIC_SOURCES[name]:
        h.update(open(os.path.join(ROOT, f), "rb").read())
    out_path = os.path.join(ROOT, "profiles", "traffic.json")
    data = json.load(open(out_path)) if os.path.exists(out_path) else {}
    data[name] = {"dram_bytes_per_product": total, "launches": launches, "sources": TRAFFIC_SOURCES[name],
                  "source_sha": h.hexdigest()[:16], "capture": note}
    with open(out_path, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    print(name, total, "bytes over", launches, "launches")


def main():
    if len(sys.argv) >= 4 and sys.argv[1] == "--record-traffic":
        return record_traffic(sys.argv[2], sys.argv[3], " ".join(sys.argv[4:]))
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="ladder_m1000", help="ladder_m1000, random64 or npz:<path>")
    ap.add_argument("--save-real", default=None, help="build the real m = 1000 superblock and save it here")
    ap.add_argument("--step", action="store_true", help="one bench step inside the NVTX range 'step'")
    ap.add_argument("--batch", type=int, default=16)
    ap.add_argument("--prec", default="bf16x3", choices=["fp64", "tf32", "bf16x3", "df64"])
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--lanczos-iters", type=int, default=0, help="also run a fixed-length Lanczos")
    ap.add_argument("--autotune", action="store_true", help="autotune, then time eager and graph-captured products")
    ap.add_argument("--reorth", type=int, default=-1,
                    help="only time full Gram-Schmidt passes at this Krylov index (one untimed pass, then --reps)")
    a = ap.parse_args()
    import torch
    from paper_0902_3185_gb300.binding import GpuSuperblock
    from workloads.superblock import Superblock, seeded_normal
    if a.save_real:
        import bench
        from paper_0902_3185_gb300 import binding
        sb, stats = bench.build_real(binding, a.batch, 0)
        sb.save(a.save_real)
        print(f"saved D={sb.dim} pairs={len(sb.pairs)} dmrg {stats['s']:.1f} s")
        return
    if a.workload.startswith("npz:"):
        sb = Superblock.load(a.workload[4:])
    elif a.workload == "ladder_m1000":
        from workloads.grown import ladder_m1000
        sb = ladder_m1000(batch=a.batch)
    else:
        from workloads.synthetic import random_sectored
        sb = random_sectored(seed=0, batch=a.batch)
    g = GpuSuperblock(sb)
    if a.reorth >= 0:
        ms, nbytes = g.time_reorth(a.reorth, prec=a.prec, reps=a.reps)
        print(f"D={sb.dim} batch={sb.batch} Gram-Schmidt pass at j={a.reorth}: {ms:.4f} ms, "
              f"{nbytes / ms / 1e6:.1f} GB/s")
        return
    x = torch.from_numpy(np.stack([seeded_normal(b, sb.dim) for b in range(sb.batch)])).cuda()
    y = g.empty()
    for _ in range(a.reps):
        g.apply_H(x, y, prec=a.prec)
    if a.autotune and a.prec in ("tf32", "bf16x3"):
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
    if a.step:
        def step():
            return g.lanczos_ground(x, tol=2e-4, max_iter=300, prec=a.prec, refine="newton_df64", refine_tol=1e-10,
                                    graph_iters=8, grad=True)
        step()
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("step")
        e0, _, infos, st, _ = step()
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        print(f"step status {st} launches {infos[0]['kernel_launches']} iters {[i['iters'] for i in infos]} "
              f"restarts {[i['restarts'] for i in infos]}")
    torch.cuda.synchronize()
    print(f"D={sb.dim} batch={sb.batch} pairs={len(sb.pairs)} flops/product={g.info['flops_per_matvec']:.4g}")


if __name__ == "__main__":
    main()
