"""Benchmark of the superblock H*psi + Lanczos hot path on GB300.

Workload (default, config 5): the 2 x 32 Hubbard ladder at m = 1000 kept
states, N_up = N_dn = 28 (1/8 hole doping).  The superblock is built by the
device DMRG driver (infinite algorithm to L = 64 at U = 8, untimed setup):
the last step's superblock, in its density-matrix basis, carries 16 members
with U = 4 .. 12 that share every operator block.

One timed step = the whole hot path for the 16-member batch: a ground-state
solve (dmrg_lanczos_ground: products, float64 Lanczos scalars, full
reorthogonalisation, tridiagonal test, CUDA graphs; mixed precision followed
by double-float Newton refinement) with the Hellmann-Feynman gradient of the
refined state (dmrg_lanczos_ground_grad).  value = algorithmic H*psi flops
executed in the step / step time.

Outside the timed step: the accuracy leg (a float64 residual certificate of
every returned state, and the float64 GPU solve of the same batch),
kernel-only product times, Lanczos rates at fixed Krylov length, and the
isometry-grown stand-in of config 5 (the earlier headline workload) with its
own accuracy leg and the local density of states.

roofline: the product kernel with the largest event-timed share of the step
(tensor-core, double-float or float64), its algorithmic flops per product /
its event-timed duration, against its peak; roofline_kernels lists them.
traffic: DRAM bytes per product from the committed ncu record
(profiles/traffic.json), reported only while the kernel sources still hash to
the recorded value.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun every rank runs its own batch (weak scaling, no collective on
the data path); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("H·ψ TFLOP/s & Lanczos steps/s at m=1000, mixed vs FP64 same GPU, "
          "|ΔE0|≤1e-8")
WORKLOAD = "hubbard_ladder_2x32_m1000_dmrg_U4-12_batch16"
GROWN_WORKLOAD = "hubbard_ladder_2x32_m1000_isogrown_U4-12_batch16"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--prec", default="auto", choices=["auto", "fp64", "tf32", "bf16x3"])
    ap.add_argument("--batch", type=int, default=16)
    ap.add_argument("--tol", type=float, default=1e-10)
    ap.add_argument("--max-iter", type=int, default=300)
    ap.add_argument("--mixed-tol", type=float, default=3e-4,
                    help="Lanczos tolerance of the mixed solve on the headline superblock (measured there: 1e-4 "
                         "458 ms, 2e-4 440, 3e-4 430, 4e-4 423, 6e-4 461 ms: a fourth residual product)")
    ap.add_argument("--refine", default="newton_df64", choices=["newton", "newton_df64", "lanczos", "none"])
    ap.add_argument("--no-grown", action="store_true", help="skip the isometry-grown stand-in leg")
    ap.add_argument("--no-fp64-solve", action="store_true",
                    help="skip the float64 solve of the accuracy leg (about 90 s on the headline superblock)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def max_over_ranks(ms, dist, device):
    """Timed milliseconds of the slowest rank (the step ends when every rank is done)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def member_products(infos):
    """Products of one solve in units of whole-batch products: the members'
    own product counts summed over the batch, divided by its size.  Members
    stop at different iterations and a stopped member gets no more products,
    so the batch's longest member overstates the work."""
    return sum(i["mixed_matvecs"] + i["fp64_matvecs"] for i in infos) / len(infos)


def job_value(world, products, flops, ms_total):
    """Whole-job algorithmic TFLOP/s: every rank ran `products` products of
    `flops` flops within the max-over-ranks time."""
    return world * products * flops / (ms_total / 1e3) / 1e12


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


# float64 FMA issue rate of the chip (ncu: 304 DFMA thread-instructions per cycle, 2 per SM x 152)
FP64_FMA_PER_CLK = 304
# float32 lanes of the chip per cycle (128 per SM x 152) and the float32
# operations of one double-float multiply-add (product with its error terms,
# two-sum, error accumulation)
FP32_OPS_PER_CLK = 128 * 152
DF_OPS_PER_FMA = 12


def source_sha(files):
    import hashlib
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


GS_TRAFFIC_J = 60  # Krylov index of the recorded Gram-Schmidt pass capture
GROWN_MIXED_TOL = 2e-4  # mixed Lanczos tolerance of the isometry-grown stand-in leg


def recorded_traffic(name):
    """DRAM bytes per product from profiles/traffic.json, or None if the
    kernel's sources changed since the capture."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        rec = json.load(f).get(name)
    if not rec or source_sha(rec["sources"]) != rec["source_sha"]:
        return None
    return rec["dram_bytes_per_product"]


def make_workload(batch, rank):
    from workloads.grown import ladder_m1000
    return ladder_m1000(batch=batch, seed=rank)


def measure_ldos(binding, torch, inp, psi, e0, prec, dev, stream, n_coef=100, n_omega=2001, eta=0.1):
    """Local density of states of the last system site (spin up) for every
    member, from the refined ground states: c|psi> and c^dag|psi> by the
    transition products (float64), n_coef Lanczos coefficients on the N - 1
    and N + 1 superblocks (products in `prec`, float64 scalars and full
    reorthogonalisation), continued fractions at n_omega points of [-20, 20] (the
    whole spectrum of these superblocks: weight_in_window checks it)
    with broadening eta.  Superblock creation stays outside the timed region;
    one untimed run first."""
    omega = np.linspace(-20.0, 20.0, n_omega)
    objs = {}
    for part, sgn in (("hole", -1.0), ("particle", 1.0)):
        sb_p, tr = inp[part]
        gp = binding.GpuSuperblock(sb_p, device=dev)
        gt = binding.GpuSuperblock(tr, device=dev)
        n_out = tr.meta["dim_out"]
        x = torch.zeros(psi.shape[0], tr.dim, dtype=torch.float64, device=dev)
        x[:, n_out:] = psi
        z = torch.from_numpy((e0[:, None] + sgn * omega[None, :]) + 1j * eta).to(dev)
        objs[part] = (gp, gt, n_out, x, z, sb_p.dim)

    def run():
        out = {}
        for part, (gp, gt, n_out, x, z, _) in objs.items():
            y = gt.apply_H(x)
            norm2, a, b, n = gp.lanczos_coeffs(y[:, :n_out].contiguous(), n_coef, prec=prec)
            out[part] = (binding.continued_fraction(norm2, a, b, n, z), norm2, n)
        return out

    run()
    torch.cuda.synchronize(dev)
    ea = torch.cuda.Event(enable_timing=True)
    eb = torch.cuda.Event(enable_timing=True)
    ea.record(stream)
    out = run()
    eb.record(stream)
    torch.cuda.synchronize(dev)
    ms = ea.elapsed_time(eb)
    dens = sum(-o[0].imag / np.pi for o in out.values())
    dw = omega[1] - omega[0]
    return {"ms": ms, "members": int(psi.shape[0]), "site": int(inp["site"]), "spin": "up",
            "coefficients": int(n_coef), "n_omega": int(n_omega), "eta": eta, "prec": prec,
            "dims": {p: int(o[5]) for p, o in objs.items()},
            "lanczos_steps_per_s": 2 * n_coef / (ms / 1e3),
            "sum_rule_max_dev": float((out["hole"][1] + out["particle"][1] - 1.0).abs().max()),
            "weight_in_window": float((dens.sum(dim=1) * dw).mean()),
            "min_coefficients": int(min(o[2].min() for o in out.values()))}


# ------------------------------------------------------------ reference arm
def run_reference(args, rank, world):
    """The CPU oracle as it stands, on the host cores: a bounded sample of the
    same workload (two batch members: a few blocked products and Lanczos
    iterations), scaled to the metric's unit."""
    if rank != 0:
        return 0
    from oracle import superblock as osb
    from workloads.superblock import seeded_normal
    sb = make_workload(args.batch, 0)
    flops_member = osb.matvec_flops(sb)
    cores = len(os.sched_getaffinity(0))
    x = seeded_normal(0, sb.dim)
    warm = max(1, args.warmup)
    for w in range(warm):  # untimed warm-up steps, as many as asked
        for b in (0, 1):
            x = osb.apply_H(sb, x, b)
            x /= np.linalg.norm(x)
    times = []
    n = 0
    t_end = time.perf_counter() + 20.0
    for step in range(max(1, args.steps)):
        t0 = time.perf_counter()
        for b in (0, 1):
            x = osb.apply_H(sb, x, b)
            x /= np.linalg.norm(x)
            n += 1
        times.append(time.perf_counter() - t0)
        if time.perf_counter() > t_end:
            break
    sec = sum(times)
    tflops = n * flops_member / sec / 1e12
    line = {"impl": "reference", "metric": METRIC, "value": tflops, "unit": "TFLOP/s", "n_gpus": args.gpus,
            "steps": len(times), "warmup": warm, "ms_per_step": 1000 * sec / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": GROWN_WORKLOAD,
                       "sample": "each step = one blocked float64 product (the solve's dominant operation) on "
                                 "each of 2 of the 16 members; TFLOP/s of those products (not a whole solve, "
                                 "which takes the oracle minutes per member)",
                       "note": "the headline superblock comes from the device DMRG driver, which this arm does "
                               "not run; the oracle's product is timed on the isometry-grown superblock of the "
                               "same lattice, m and members (D = 165,055 per member instead of 886,884)"},
            "cpu_baseline": {"value": tflops, "unit": "TFLOP/s", "cores": cores, "kind": "oracle",
                             "sample": f"{n} blocked float64 products of single members (NumPy, default BLAS "
                                       f"threading; blocks this small mostly run on one thread), D={sb.dim}"},
            "e2e": {"value": tflops, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def _oracle_products(sb, seconds, max_n=200):
    """Time the oracle's blocked float64 product (one member per call)."""
    from oracle import superblock as osb
    from workloads.superblock import seeded_normal
    x = seeded_normal(1, sb.dim)
    osb.apply_H(sb, x, 0)
    n = 0
    t0 = time.perf_counter()
    while n < 3 or time.perf_counter() - t0 < seconds:
        x = osb.apply_H(sb, x, n % sb.batch)
        x /= np.linalg.norm(x)
        n += 1
        if n >= max_n:
            break
    return n, time.perf_counter() - t0


_ONE_THREAD = r"""
import sys, time
sys.path.insert(0, sys.argv[1])
import bench
sb = bench.make_workload(int(sys.argv[2]), 0)
n, sec = bench._oracle_products(sb, float(sys.argv[3]), int(sys.argv[4]))
print(n, sec)
"""


def cpu_baseline_sample(sb):
    """The oracle's blocked product on one host thread (BLAS threads pinned
    to 1 before NumPy loads, in a child process), and in this process with
    NumPy's default BLAS threading over the host cores for comparison."""
    from oracle import superblock as osb
    flops = osb.matvec_flops(sb)
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    r = subprocess.run([sys.executable, "-c", _ONE_THREAD, ROOT, str(sb.batch), "10.0", "200"],
                       env=env, capture_output=True, text=True, timeout=600)
    n1, s1 = r.stdout.split()[-2:]
    n1, s1 = int(n1), float(s1)
    n, sec = _oracle_products(sb, 5.0)
    return {"value": n1 * flops / s1 / 1e12, "unit": "TFLOP/s", "cores": 1, "kind": "oracle",
            "sample": f"{n1} blocked float64 products (one member each, NumPy, one thread) of the same "
                      f"workload, {s1:.1f} s",
            "value_all_cores": n * flops / sec / 1e12, "host_cores": len(os.sched_getaffinity(0)),
            "sample_all_cores": f"{n} products with NumPy's default BLAS threading, {sec:.1f} s"}


# ------------------------------------------------------------------- ours
def build_real(binding, batch, seed):
    """Config 5 from the device DMRG driver: the infinite algorithm on the
    2 x 32 Hubbard ladder (t_leg = t_rung = 1, U = 8, N_up = N_dn = 28,
    m = 1000; BF16x3 Lanczos refined to 1e-10 in every step); the last step's
    superblock (density-matrix basis) carries `batch` members U = 4 .. 12."""
    from workloads import lattice_models as lm
    t0 = time.perf_counter()
    dm = binding.GpuDmrg(lm.hubbard_ladder(1.0, 1.0, 8.0, density=56 / 64), 64, m=1000, tol=1e-10,
                         prec="bf16x3", refine="newton_df64", mixed_tol=2e-4, seed=1 + seed)
    steps = dm.infinite()
    sb1, _ = dm.last_superblock()
    dm.close()
    secs = time.perf_counter() - t0
    Us = 4.0 + 8.0 * np.arange(batch) / max(batch - 1, 1)
    cp = np.zeros((batch, len(sb1.class_names)))
    cp[:] = sb1.couplings[0]
    cp[:, sb1.class_names.index("U")] = Us
    sb = sb1.with_coeffs(sb1.coeffs_from_couplings(cp))
    stats = {"driver": "device DMRG (dmrg_sys_infinite), 31 steps to L = 64, m = 1000, BF16x3 + double-float "
                       "refinement to 1e-10 per step", "s": secs, "steps": len(steps),
             "energy_L64_U8": steps[-1]["energy"], "eps_last": steps[-1]["eps_S"],
             "truncation_s": sum(x["ms_truncate"] for x in steps) / 1e3,
             "superblock_s": sum(x["ms_superblock"] for x in steps) / 1e3,
             "solve_s": sum(x["ms_solve"] for x in steps) / 1e3,
             "status": max(x["status"] for x in steps)}
    return sb, stats


def event_ms(torch, stream, dev, fn, reps=1):
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(reps):
        r = fn()
    b.record(stream)
    torch.cuda.synchronize(dev)
    return a.elapsed_time(b) / reps, r


def product_ms(torch, g, x, stream, dev, prec, reps):
    y = g.empty()
    g.apply_H(x, y, prec=prec)
    return event_ms(torch, stream, dev, lambda: g.apply_H(x, y, prec=prec), reps)[0]


def dpsi_max(torch, p, q):
    p = p / p.norm(dim=1, keepdim=True)
    q = q / q.norm(dim=1, keepdim=True)
    return float(torch.minimum((p - q).norm(dim=1), (p + q).norm(dim=1)).max())


def measure_grown(binding, torch, args, prec, dev, stream, rank):
    """The isometry-grown stand-in of config 5 (the workload of the earlier
    headline): the same step, its float64 solve of the same batch, and the
    local density of states of the last system site."""
    from workloads.grown import ladder_m1000_ldos
    from workloads.superblock import seeded_normal
    inp = ladder_m1000_ldos(batch=args.batch, seed=rank)
    sb = inp["N"]
    g = binding.GpuSuperblock(sb, device=dev)
    tune = g.autotune(prec=prec, reps=5)
    flops = g.info["flops_per_matvec"]
    x0 = torch.from_numpy(np.stack([seeded_normal(1000 * rank + b, sb.dim) for b in range(sb.batch)])).to(dev)

    def step():  # the stand-in keeps the tolerance of its own measured history
        return g.lanczos_ground(x0, tol=GROWN_MIXED_TOL, max_iter=args.max_iter, prec=prec, refine=args.refine,
                                refine_tol=args.tol, graph_iters=8, grad=True)
    for _ in range(3):
        step()
    n_t = 5
    ms, (e0, psi, infos, st, dE) = event_ms(torch, stream, dev, step, n_t)
    mv = member_products(infos)
    t64, (e64, p64, i64, s64, dE64) = event_ms(torch, stream, dev, lambda: g.lanczos_ground(
        x0, tol=args.tol, max_iter=max(600, args.max_iter), prec="fp64", refine="none", graph_iters=8, grad=True))
    e0, e64 = np.asarray(e0, dtype=np.float64), np.asarray(e64, dtype=np.float64)
    mv_ms = product_ms(torch, g, x0, stream, dev, prec, 20)
    ldos = measure_ldos(binding, torch, inp, psi, e0, prec, dev, stream)
    out = {"workload": "hubbard_ladder_2x32_m1000_isogrown_U4-12_batch16",
           "source": "isometry-grown superblock (random q-preserving isometries beyond m; workloads/grown.py)",
           "D": sb.dim, "sectors": sb.n_sectors, "pairs": len(sb.pairs), "autotune": tune,
           "step_ms": ms, "step_tflops": mv * flops / (ms / 1e3) / 1e12, "status": st,
           "lanczos_iters": max(i["iters"] for i in infos),
           "matvec_ms": mv_ms, "matvec_tflops": flops / (mv_ms / 1e3) / 1e12,
           "accuracy": {"reference": f"float64 GPU solve of the same members (tol {args.tol:g}), status {s64}",
                        "dE0_rel_max": float(np.max(np.abs(e0 - e64) / np.abs(e64))),
                        "dpsi_max": dpsi_max(torch, psi, p64), "fp64_solve_ms": t64,
                        "fp64_solve_iters": max(i["iters"] for i in i64),
                        "speedup_mixed_vs_fp64_solve": t64 / ms},
           "ldos": ldos}
    del g
    torch.cuda.empty_cache()
    return out


_ONE_THREAD_REAL = r"""
import sys, time
sys.path.insert(0, sys.argv[1])
import bench
from workloads.superblock import Superblock
sb = Superblock.load(sys.argv[2])
n, sec = bench._oracle_products(sb, float(sys.argv[3]), int(sys.argv[4]))
print(n, sec)
"""


def cpu_baseline_real(sb):
    """The oracle's blocked float64 product on the headline superblock (saved
    to a temporary npz for a child process whose BLAS threads are pinned to 1
    before NumPy loads), and in this process with NumPy's default threading."""
    import tempfile
    from oracle import superblock as osb
    flops = osb.matvec_flops(sb)
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "sb.npz")
        sb.save(path)
        env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
        r = subprocess.run([sys.executable, "-c", _ONE_THREAD_REAL, ROOT, path, "10.0", "50"],
                           env=env, capture_output=True, text=True, timeout=900)
        n1, s1 = r.stdout.split()[-2:]
    n1, s1 = int(n1), float(s1)
    n, sec = _oracle_products(sb, 5.0, 50)
    return {"value": n1 * flops / s1 / 1e12, "unit": "TFLOP/s", "cores": 1, "kind": "oracle",
            "sample": f"{n1} blocked float64 products (one member each, NumPy, one thread) of the headline "
                      f"superblock, {s1:.1f} s",
            "value_all_cores": n * flops / sec / 1e12, "host_cores": len(os.sched_getaffinity(0)),
            "sample_all_cores": f"{n} products with NumPy's default BLAS threading, {sec:.1f} s"}


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        return run_reference(args, rank, world)
    import torch
    import torch.distributed as dist
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_0902_3185_gb300 import binding
    from workloads.superblock import seeded_normal
    stream = torch.cuda.current_stream(dev)
    peaks, kind = measured_peaks()

    # config 5 from the device DMRG driver (setup, outside the timed region)
    sb, dmrg_stats = build_real(binding, args.batch, rank)
    g = binding.GpuSuperblock(sb, device=dev)
    prec = args.prec
    if prec == "auto":
        prec = "fp64"
        try:
            g.apply_H(g.empty().zero_(), prec="bf16x3")
            prec = "bf16x3"
        except binding.DmrgError:
            pass
    tune = g.autotune(prec=prec, reps=5) if prec != "fp64" else None
    flops_mv = g.info["flops_per_matvec"]
    X0 = np.stack([seeded_normal(1000 * rank + 5000 + b, sb.dim) for b in range(sb.batch)])
    x0 = torch.from_numpy(X0).to(dev)

    def step(x):
        # ground state and its Hellmann-Feynman gradient (with the Newton
        # refinement the gradient comes out of its last residual product)
        e0, psi, infos, st, dEdc = g.lanczos_ground(x, tol=args.tol if prec == "fp64" else args.mixed_tol,
                                                    max_iter=args.max_iter, prec=prec, refine=args.refine,
                                                    refine_tol=args.tol, graph_iters=8, grad=True)
        step.status = st
        return e0, psi, infos, dEdc

    for _ in range(max(3, args.warmup)):
        e0, psi, infos, dEdc = step(x0)
    torch.cuda.synchronize(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    clocks = ClockSampler(local)
    clocks.start()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    ev = []
    mv_count = it_count = launches = 0
    for k in range(args.steps):
        flush.fill_(float(k))  # L2 flush between timed steps
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        e0, psi, infos, dEdc = step(x0)
        b.record(stream)
        ev.append((a, b))
        mv_count += member_products(infos)
        it_count += max(i["iters"] + i["refine_iters"] for i in infos)
        launches += infos[0]["kernel_launches"]
    torch.cuda.synchronize(dev)
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in ev), dist if world > 1 else None, dev)
    ms_per_step = ms / args.steps
    value = job_value(world, mv_count, flops_mv, ms)
    e_step, psi_step, dE_step = np.asarray(e0, dtype=np.float64), psi, dEdc
    sm_mhz = clk.get("sm_mhz") or peaks.get("sm_max_mhz", 2070.0)

    def timed(fn):
        return event_ms(torch, stream, dev, fn)
    # where the step goes: the mixed Lanczos alone, then with the refinement
    t_lz, (_, _, info_lz, _) = timed(lambda: g.lanczos_ground(
        x0, tol=args.tol if prec == "fp64" else args.mixed_tol, max_iter=args.max_iter, prec=prec,
        refine="none", graph_iters=8))
    t_full, (_, _, info_full, _) = timed(lambda: g.lanczos_ground(
        x0, tol=args.tol if prec == "fp64" else args.mixed_tol, max_iter=args.max_iter, prec=prec,
        refine=args.refine, refine_tol=args.tol, graph_iters=8))
    lz_iters = max(i["iters"] for i in info_lz)
    breakdown = {"lanczos_ms": t_lz, "refine_ms": t_full - t_lz, "solve_status": step.status,
                 "mixed_lanczos_steps_per_s": lz_iters / (t_lz / 1e3),
                 "lanczos_iters": max(i["iters"] for i in info_full),
                 "fp64_products": max(i["fp64_matvecs"] for i in info_full),
                 "mixed_products": max(i["mixed_matvecs"] for i in info_full),
                 "residual_max": max(i["residual"] for i in info_full),
                 "lanczos_iters_per_member": [int(i["iters"]) for i in info_full],
                 "lanczos_restarts": sum(int(i["restarts"]) for i in info_full)}

    # kernel-only product timing (events on the launching stream)
    mv_ms = product_ms(torch, g, x0, stream, dev, prec, 20)
    mv64_ms = product_ms(torch, g, x0, stream, dev, "fp64", 2) if prec != "fp64" else mv_ms
    df = prec != "fp64" and args.refine == "newton_df64"
    rprec = "df64" if df else "fp64"  # arithmetic of the refinement's residual products
    mvr_ms = product_ms(torch, g, x0, stream, dev, "df64", 3) if df else mv64_ms
    t_pdot, _ = timed(lambda: g.apply_H_term_dots(x0, prec=rprec))
    t_grad, _ = timed(lambda: g.energy_grad(psi))

    # end to end through the public API with host buffers
    xh = torch.from_numpy(X0).pin_memory()
    ph = torch.empty_like(xh).pin_memory()
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        xd = xh.to(dev, non_blocking=True)
        e0h, psi_e, infos_e, dEdc_e = step(xd)
        ph.copy_(psi_e, non_blocking=True)
        dh = dEdc_e.cpu()
    torch.cuda.synchronize(dev)
    e2e_s = (time.perf_counter() - t0) / args.steps
    e2e = {"value": world * mv_count / args.steps * flops_mv / e2e_s / 1e12, "unit": "TFLOP/s",
           "h2d_bytes_per_step": int(X0.nbytes), "d2h_bytes_per_step": int(X0.nbytes + dh.numel() * 8)}

    # Lanczos iteration rate at fixed Krylov length j (no early stop)
    fixed_j = {}
    for pj, js in ([(prec, (20, 100)), ("fp64", (20, 100))] if prec != "fp64" else [("fp64", (20, 100))]):
        for j in js:
            t_j, _ = timed(lambda: g.lanczos_ground(x0, tol=1e-300, max_iter=j, prec=pj, refine="none",
                                                    graph_iters=10))
            fixed_j[f"{pj}_j{j}_steps_per_s"] = j / (t_j / 1e3)
    for j in (20, 100):  # one full Gram-Schmidt pass reads the Krylov basis twice (dots, then update)
        fixed_j[f"reorth_bytes_per_step_j{j}"] = 2 * (j + 1) * sb.batch * sb.dim * 8

    # accuracy leg: a float64 certificate of every returned state (the
    # residual recomputed with the float64 product bounds |theta - E0| by |r|,
    # Weinstein) and the float64 GPU solve of the same batch from the same
    # start vectors (float64 products and Lanczos to the same tolerance)
    accuracy = None
    if prec != "fp64":
        hp = g.apply_H(psi_step, prec="fp64")
        nrm = psi_step.norm(dim=1)
        theta = ((psi_step * hp).sum(dim=1) / nrm ** 2)
        res = ((hp - theta[:, None] * psi_step).norm(dim=1) / nrm).cpu().numpy()
        th = theta.cpu().numpy()
        accuracy = {"fp64_certificate": {"residual_rel_max": float(np.max(res / np.abs(th))),
                                         "weinstein_bound_dE0_rel_max": float(np.max(res / np.abs(th))),
                                         "theta_fp64_vs_e0_rel_max": float(np.max(np.abs(th - e_step) / np.abs(th)))}}
        if not args.no_fp64_solve:
            t_f64, (e64, psi64, info64, st64, dE64) = timed(lambda: g.lanczos_ground(
                x0, tol=args.tol, max_iter=600, prec="fp64", refine="none", graph_iters=8, grad=True))
            e64 = np.asarray(e64, dtype=np.float64)
            dE_rel = np.abs(e_step - e64) / np.abs(e64)
            accuracy.update({
                "reference": "float64 GPU solve of the same 16 members from the same start vectors (float64 "
                             f"products and Lanczos, tol {args.tol:g}, at most 600 iterations), status {st64}",
                "dE0_rel_max": float(dE_rel.max()), "dE0_rel_per_member": [float(v) for v in dE_rel],
                "dpsi_max": dpsi_max(torch, psi_step, psi64), "dE_dc_max_abs_diff": float((dE_step - dE64).abs().max()),
                "meets_1e-8": bool(dE_rel.max() <= 1e-8),
                "fp64_solve_ms": t_f64, "fp64_solve_iters": max(i["iters"] for i in info64),
                "fp64_lanczos_steps_per_s": max(i["iters"] for i in info64) / (t_f64 / 1e3),
                "mixed_solve_ms": ms_per_step, "speedup_mixed_vs_fp64_solve": t_f64 / ms_per_step})

    n_mixed = mv_count / args.steps - max(i["fp64_matvecs"] for i in infos) if prec != "fp64" else 0
    n_f64 = max(i["fp64_matvecs"] for i in infos) if prec != "fp64" else mv_count / args.steps
    kernels = {}
    if prec != "fp64":
        pk = peaks["bf16_tflops"] / 3.0 if prec == "bf16x3" else peaks["bf16_tflops"] * 1100.0 / 2250.0
        a_t = flops_mv / (mv_ms / 1e3) / 1e12
        kernels["tensor_product"] = {
            "bound": "tensor", "achieved": a_t, "peak": pk, "unit": "TFLOP/s", "frac": a_t / pk,
            "traffic": recorded_traffic(f"tensor_product_{prec}_real"),
            "kernel": f"tcgen05 product, {prec} (staging + 3 grouped launches per dmrg_apply_H)",
            "peak_source": (f"{kind} bf16 peak / 3 (three bf16 MMAs per algorithmic product)" if prec == "bf16x3"
                            else f"{kind} bf16 peak x nominal 1100/2250"),
            "ms_per_step": n_mixed * mv_ms}
    pk64 = FP64_FMA_PER_CLK * 2 * sm_mhz * 1e6 / 1e12
    pkdf = FP32_OPS_PER_CLK / DF_OPS_PER_FMA * 2 * sm_mhz * 1e6 / 1e12
    newton = prec != "fp64" and args.refine.startswith("newton")
    # the refinement computes the per-term dots with the residual product it
    # expects to be the last (one per step, unless a residual met the
    # tolerance earlier than expected)
    n_dots = 1 if newton and n_f64 >= 2 else 0
    if df:
        pk_r, name_r = pkdf, "df64"
        src_r = (f"{FP32_OPS_PER_CLK} float32 ops/clock / {DF_OPS_PER_FMA} per double-float FMA x 2 x "
                 f"{sm_mhz:.0f} MHz (median SM clock of the timed region)")
        kern_r = "grouped double-float product, seg_gemm_df_kernel (3 launches per product)"
        kern_d = ("double-float product with the per-term dots (unscaled intermediates + seg_gemm_df_dots_kernel, "
                  "the refinement's residual expected to be the last)")
    else:
        pk_r, name_r = pk64, "fp64"
        src_r = f"304 float64 FMA/clock x 2 x {sm_mhz:.0f} MHz (median SM clock of the timed region)"
        kern_r = "grouped float64 product, seg_gemm_f64_kernel (3 launches per dmrg_apply_H)"
        kern_d = ("float64 product with the per-term dots (unscaled intermediates + seg_gemm_f64_dots_kernel, "
                  "the refinement's residual expected to be the last)")
    a_r = flops_mv / (mvr_ms / 1e3) / 1e12
    kernels[f"{name_r}_product"] = {
        "bound": "alu", "achieved": a_r, "peak": pk_r, "unit": "TFLOP/s", "frac": a_r / pk_r,
        "traffic": recorded_traffic(f"{name_r}_product_real"), "kernel": kern_r, "peak_source": src_r,
        "ms_per_step": (n_f64 - n_dots) * mvr_ms + (0.0 if newton else t_grad)}
    if n_dots:
        a_d = flops_mv / (t_pdot / 1e3) / 1e12
        kernels[f"{name_r}_product_with_dots"] = {
            "bound": "alu", "achieved": a_d, "peak": pk_r, "unit": "TFLOP/s", "frac": a_d / pk_r,
            "traffic": None, "kernel": kern_d, "peak_source": src_r, "ms_per_step": n_dots * t_pdot}
    # the full Gram-Schmidt pass (HBM-bound): event-timed at the solve's mean
    # Krylov index; its share of the step estimated from every member's own
    # iteration count (converged members are skipped) at the measured rate
    jm = max(1, lz_iters // 2)
    gs_ms, gs_bytes = g.time_reorth(jm, prec=prec, reps=5)
    a_gs = gs_bytes / (gs_ms / 1e3) / 1e9
    gs_step_bytes = sum((2.0 * (jj + 1) + 3.0) * sb.dim * 8.0 for i in info_full for jj in range(i["iters"]))
    # the recorded pass (ncu, Krylov index GS_TRAFFIC_J) scaled to index jm by
    # the rows read: its traffic equals the algorithmic bytes, which grow in
    # proportion to 2 (j + 1) + 3 vectors
    gs_traffic = recorded_traffic(f"gram_schmidt_pass_{prec}_real")
    if gs_traffic is not None:
        gs_traffic *= (2.0 * (jm + 1) + 3.0) / (2.0 * (GS_TRAFFIC_J + 1) + 3.0)
    kernels["gram_schmidt_pass"] = {
        "bound": "hbm", "achieved": a_gs, "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": a_gs / peaks["hbm_gbs"],
        "traffic": gs_traffic,
        "kernel": (f"full Gram-Schmidt pass at Krylov index {jm} (k_multidot + k_reduce_rows + k_multiaxpy, "
                   f"{'double-float pair' if prec != 'fp64' else 'float64'} basis), {gs_bytes / 1e9:.2f} GB moved"),
        "peak_source": f"{kind} HBM copy bandwidth",
        "ms_per_step": gs_step_bytes / (a_gs * 1e6)}
    dom = max(kernels, key=lambda k: kernels[k]["ms_per_step"])
    roof = dict(kernels[dom])
    roof["share_of_step"] = roof["ms_per_step"] / ms_per_step
    for k in kernels:
        kernels[k]["share_of_step"] = kernels[k]["ms_per_step"] / ms_per_step
    sb_info = {"D": sb.dim, "sectors": sb.n_sectors, "pairs": len(sb.pairs),
               "max_sector": int(max(sb.r.max(), sb.c.max()))}
    del g, step
    torch.cuda.empty_cache()

    grown = measure_grown(binding, torch, args, prec, dev, stream, rank) if (prec != "fp64" and not args.no_grown) \
        else None

    out = {"metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps,
           "warmup": max(3, args.warmup), "ms_per_step": ms_per_step, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None,
           "dtype": "f64" if prec == "fp64" else f"{prec}+f32acc (products), f64 (Lanczos)",
           "data": "synthetic (the model's own DMRG superblock from the device driver; no dataset)",
           "config": dict({"workload": WORKLOAD, "batch": sb.batch, "m": 1000, "prec": prec, "tol": args.tol, "mixed_tol": args.mixed_tol,
                           "l2": "256 MB flush between timed steps; Krylov basis > L2", "autotune": tune},
                          **sb_info),
           "dmrg_setup": dmrg_stats,
           "lanczos_steps_per_s": world * it_count / (ms / 1e3),
           "matvec_ms": mv_ms, "matvec_tflops": flops_mv / (mv_ms / 1e3) / 1e12, "matvec_fp64_ms": mv64_ms,
           "matvec_fp64_tflops": flops_mv / (mv64_ms / 1e3) / 1e12,
           "residual_products": rprec, "matvec_residual_ms": mvr_ms,
           "speedup_mixed_vs_fp64_matvec": mv64_ms / mv_ms,
           "iters_per_step": it_count / args.steps, "e0": [float(v) for v in e_step[:4]],
           "breakdown": dict(breakdown, energy_grad_ms=t_grad, residual_product_with_dots_ms=t_pdot),
           "lanczos_fixed_j": fixed_j, "accuracy": accuracy, "isometry_grown": grown,
           "roofline": roof, "roofline_kernels": kernels, "e2e": e2e, "gpu_launches": launches, "clocks": clk}
    if rank == 0:
        # the oracle baseline is timed at N = 1 only (host cores shared by N ranks would not be the same baseline)
        out["cpu_baseline"] = cpu_baseline_real(sb) if world == 1 else None
        print(json.dumps(out), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
