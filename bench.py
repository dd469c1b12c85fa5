#!/usr/bin/env python3
"""Benchmark of the GB300 cooperative conjugate gradient (cCG) solver.

One step = one complete FP64 cCG solve (initial residual, iterations to
relative residual 1e-10, true-residual check, copy-out) of the dense SPD
system A x = b with A the exponential kernel exp(-|z_i - z_j| / 0.2) on 8192
points uniform in [0, 1]^3 (seed 1) plus 1e-2 I, b ~ N(0, 1), x0 = 0, p = 8
agents.  The metric is solves/s.  By default the solve forms its block
products A D_k exactly on the FP8 tensor cores from 4-bit slices of A and D_k
(CCG_FP64_SLICED: FP64 accuracy, parity-tested against the FP64 oracle);
``--product fp64`` runs them on the FP64 pipe instead.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--p P] [--impl ours|reference]

N > 1 runs independent replicas (one solve per rank per step; the method has
no cross-GPU data path), launched by torchrun.
``--impl reference`` times the FP64 CPU oracle on the host cores instead: each
timed step is one full oracle solve of the same system (warm-up steps are
short samples).

Output: one JSON line per additional measurement ({"detail": ...}: agent
sweeps, the precision workload, tensor-core block products, batching,
serving), then the result line, kept short, whose "targets" key collects the
figures the method's targets rest on.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_DEFAULT = 8192
TOL = 1e-10
WORKLOAD = ("FP64 cCG: A = exp(-|z_i-z_j|/0.2) + 1e-2 I on n=8192 points U[0,1]^3 (seed 1), "
            "b ~ N(0,1), x0 = 0, tol 1e-10 relative")
METRIC = "solves/s at relres 1e-10 (FP64 cCG)"
GOLDEN_ITERS = os.path.join(ROOT, "tests", "golden", "oracle_iterations.json")
# DRAM bytes (read + write) per pass over A of the persistent solve kernels,
# measured with ncu (dram__bytes_read.sum + dram__bytes_write.sum) on
# 20-iteration solves of the benchmark system (22 passes; the traffic grows
# with the passes, so a full solve is scaled from it).  FP64 pipe, p = 8:
# 11 853.2 MB; sliced product (21 sliced passes and one FP64 check over the
# FP64 A): 946.8 MB per sliced pass, profiles/sliced_fp64_solve_traffic_n8192_p8.md.
NCU_BYTES_PER_PASS = {("fp64", 8192, 8): (11814291712 + 45762304) / 22.0,
                      ("sliced", 8192, 8): (20263912960 + 66062080 - 8.0 * 8192 ** 2) / 21.0}


def run_config(n, p, product):
    """The config dict both arms print (same workload, same keys)."""
    return {"workload": WORKLOAD, "n": n, "p": p, "tol": TOL,
            "product": "FP64 from exact FP8 slices (tensor cores)" if product == "sliced"
                       else "FP64 pipe",
            "l2": "inputs > L2 (A 512 MiB)",
            "parallelism": "replicas"}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--p", type=int, default=8)
    ap.add_argument("--product", default="sliced", choices=["sliced", "fp64"],
                    help="block product of the timed FP64 solve")
    ap.add_argument("--n", type=int, default=N_DEFAULT)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0,
                    help="target CPU time of the oracle sample")
    ap.add_argument("--maxit", type=int, default=0, help="iteration cap (0 = 20 n)")
    ap.add_argument("--profile", default="none",
                    choices=["none", "solve", "block", "lowp", "mixed", "lowp32", "sliced",
                             "cheb", "batched"],
                    help="profiling mode: run only K solves, K FP64 block products or K "
                         "tensor-core block products (n = 32768)")
    ap.add_argument("--no-mixed", action="store_true",
                    help="skip the additional measurements (sweeps, precision, batching, serving)")
    ap.add_argument("--lowp-n", type=int, default=32768,
                    help="size of the tensor-core block-product measurement")
    ap.add_argument("--lowp-fmt", default="bf16", choices=["bf16", "fp8"],
                    help="storage format of A for --profile lowp")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def workload(n):
    from paper_1204_0069_gb300 import workloads as wl
    return wl.exp_kernel(n, seed=1, length=0.2, nugget=1e-2)


def oracle_golden_iterations(n, p):
    """The oracle's iteration count on the benchmark system, as stored by
    tests/golden/make_oracle_iterations.py (inputs generated on an x86 host)."""
    try:
        rows = json.load(open(GOLDEN_ITERS))["rows"]
    except (OSError, ValueError, KeyError):
        return None
    for r in rows:
        if r["n"] == n and r["p"] == p and r["workload"].startswith("exp_kernel"):
            return int(r["iterations"])
    return None


def cpu_full_solve(A, b, p):
    """One full oracle solve on all host cores.  Returns (seconds, cores,
    iterations)."""
    import oracle
    n = b.shape[0]
    cores = os.cpu_count() or 1
    X0 = oracle.initial_block(n, p, None, 1.0, 0)
    t0 = time.perf_counter()
    r = oracle.ccg(A, b, X0, TOL, 20 * n, nthreads=cores)
    return time.perf_counter() - t0, cores, r["iterations"]


def cpu_sample(A, b, p, target_s):
    """Time a bounded sample of oracle iterations on all host cores and scale
    it to one full solve with the oracle's own iteration count (from a run of
    the first sample to the end when target_s allows, else the stored count).
    Returns (solves_per_s, cores, sample_text)."""
    import oracle
    n = b.shape[0]
    cores = os.cpu_count() or 1
    X0 = oracle.initial_block(n, p, None, 1.0, 0)
    t0 = time.perf_counter()
    oracle.ccg(A, b, X0, 1e-300, 2, residual_replacement=False, nthreads=cores)
    t2 = time.perf_counter() - t0          # init + 2 iterations + residual check
    m = max(2, int(target_s / max(t2 / 2.0, 1e-6)))
    t0 = time.perf_counter()
    oracle.ccg(A, b, X0, 1e-300, m, residual_replacement=False, nthreads=cores)
    tm = time.perf_counter() - t0
    full = oracle_golden_iterations(n, p)
    per_it = (tm - t2) / max(m - 2, 1)
    fixed = max(t2 - 2 * per_it, 0.0)      # init A X_0 + final true residual
    if full is None:
        full = m
        note = "full iteration count unknown: scaled to the sample length"
    else:
        note = f"scaled to its stored count of {full}"
    t_solve = fixed + per_it * full
    return 1.0 / t_solve, cores, (f"{m} oracle iterations ({tm:.1f} s, {cores} threads), "
                                  f"{note}")


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
                power.append(float(f[3]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "power_w_max": max(power), "samples": len(sm), "reasons": sorted(reasons)}


def max_over_ranks(seconds, dist, device):
    """The largest of the ranks' times (the job's time), or the value itself
    on a single process."""
    if dist is None:
        return seconds
    import torch
    t = torch.tensor([seconds], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world, steps, seconds):
    """Whole-job solves/s: every rank solves `steps` systems in `seconds`."""
    return world * steps / seconds


def p_bucket(p):
    q = 1
    while q < p:
        q *= 2
    return q


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


def solve_flops(n, p, iters, checks, replacements):
    """Algorithmic FP64 flops of one solve (Table 1 counts x 2 for multiply-add):
    A X_0 (2 n^2 p), per iteration A D (2 n^2 p) + six n x p x p products
    (12 n p^2), one true-residual product (2 n^2) per check, and one A X per
    residual replacement."""
    return (2.0 * n * n * p + iters * (2.0 * n * n * p + 12.0 * n * p * p)
            + checks * 2.0 * n * n + replacements * 2.0 * n * n * p)


def solve_bytes(n, p, iters, checks, replacements):
    """Algorithmic HBM bytes: A (8 n^2) once per block product plus the
    n x p blocks each pass touches (about 10 n p doubles per iteration)."""
    passes = 1 + iters + checks + replacements
    return 8.0 * n * n * passes + iters * 80.0 * n * p


def device_exp_kernel(n, seed, length, nugget, dev):
    """Exponential-kernel SPD matrix built on the device, the same family as
    ``workloads.exp_kernel`` (points drawn with numpy from `seed`); used for
    the n = 32768 precision workload and the serving pool.  Distances are
    taken from coordinate differences, sqrt(dx^2 + dy^2 + dz^2), so that the
    diagonal is exactly 1 + nugget and the matrix exactly symmetric (a
    distance through |x|^2 + |y|^2 - 2 x.y leaves sqrt(eps) on the diagonal)."""
    import numpy as np
    import torch
    rng = np.random.default_rng(seed)
    z = torch.from_numpy(rng.random((n, 3))).to(dev)
    A = torch.empty((n, n), dtype=torch.float64, device=dev)
    for i0 in range(0, n, 4096):
        zi = z[i0:i0 + 4096]
        d2 = (zi[:, 0:1] - z[:, 0]).square_()
        for k in (1, 2):
            d2.add_((zi[:, k:k + 1] - z[:, k]).square_())
        torch.exp(d2.sqrt_().div_(-length), out=A[i0:i0 + 4096])
        del d2
    A.diagonal().add_(nugget)
    return A


def lowp_roofline(ccg, solver, dev, A, p, hbm_gbs, steps=10):
    """HBM bandwidth of the tensor-core block products (A in BF16, FP8 E4M3,
    FP32 as TF32 halves, FP64 as 14 exact FP8 slices) on the precision
    workload (exponential kernel, length 0.1, nugget 1e-3, seed 2).  Bytes are
    the stored A; the FP32 and sliced products run through the solver's
    persistent kernel and include its operand conversion, barriers and fixup."""
    import numpy as np
    import torch
    n = A.shape[0]
    out = {}
    for fmt, name in [(ccg.LOWP_BF16, "bf16"), (ccg.LOWP_FP8_E4M3, "fp8_e4m3"),
                      (ccg.LOWP_FP32, "fp32_tf32_halves"), (ccg.LOWP_FP64_SLICED, "fp64_sliced")]:
        m = solver.lowp_matrix(A, fmt)
        V = torch.randn(n, p, dtype=torch.float64, device=dev)
        W = torch.empty(n, p, dtype=torch.float64, device=dev)
        for _ in range(3):
            m.block_product(V, W)
        ts = [m.block_product(V, W)[1] for _ in range(steps)]
        ms = float(np.mean(ts))
        gbs = m.nbytes() / (ms / 1e3) / 1e9
        out[name] = {"n": n, "p": p, "ms": ms, "bytes": m.nbytes(), "gbs": gbs,
                     "frac_of_measured_hbm": gbs / hbm_gbs if hbm_gbs else None}
        m.close()
    return out


def mixed_lines(ccg, dev, stream, A, b, p, steps, tol=TOL):
    """solves/s of FP64 cCG (FP64 pipe and sliced product) and of the
    mixed-precision solves (default methods) on (A, b)."""
    import numpy as np
    import torch
    n = b.shape[0]
    dA = torch.from_numpy(A).to(dev)
    db = torch.from_numpy(b).to(dev)
    out = {}
    for name, prec in [("fp64_pipe", ccg.FP64), ("fp64_sliced", ccg.FP64_SLICED),
                       ("fp32", ccg.FP32_IR), ("bf16", ccg.BF16_IR), ("fp8", ccg.FP8_IR)]:
        x = torch.zeros(n, dtype=torch.float64, device=dev)
        with ccg.Solver(stream=stream.cuda_stream, precision=prec) as s:
            s.solve(dA, db, x, p=p, tol=tol, maxit=20 * n)      # warm-up
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            rs = [s.solve(dA, db, x, p=p, tol=tol, maxit=20 * n) for _ in range(steps)]
            e1.record(stream)
            torch.cuda.synchronize()
        t = e0.elapsed_time(e1) / 1e3 / steps
        xs = x.cpu().numpy()
        relres = float(np.linalg.norm(b - A @ xs) / np.linalg.norm(b))
        r = rs[-1]
        out[name] = {"solves_per_s": 1.0 / t, "ms_per_solve": 1e3 * t, "status": r.status_name,
                     "relres_true": relres, "iterations": r.iterations,
                     "outer_steps": r.outer_steps}
    for k in ("fp32", "bf16", "fp8"):
        ok = out[k]["status"] == "CCG_OK"
        out[k]["speedup_vs_fp64_pipe"] = (out[k]["solves_per_s"] / out["fp64_pipe"]["solves_per_s"]
                                          if ok else None)
        out[k]["speedup_vs_fp64_sliced"] = (out[k]["solves_per_s"] /
                                            out["fp64_sliced"]["solves_per_s"] if ok else None)
    return out


def sliced_sweep(ccg, stream, dA, db, x, n, ps=(1, 4, 8, 16)):
    """FP64 cCG with the block product formed exactly from FP8 slices of A and
    D on the tensor cores (CCG_FP64_SLICED), on the benchmark system."""
    with ccg.Solver(stream=stream.cuda_stream, precision=ccg.FP64_SLICED) as s:
        return p_sweep(ccg, s, stream, dA, db, x, n, ps)


def p_sweep(ccg, solver, stream, dA, db, x, n, ps=(1, 4, 8, 16, 32)):
    """FP64 cCG on the benchmark system for every agent count of the sweep:
    one warm-up and one timed solve each."""
    import torch
    out = {}
    for p in ps:
        solver.solve(dA, db, x, p=p, tol=TOL, maxit=20 * n)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        r = solver.solve(dA, db, x, p=p, tol=TOL, maxit=20 * n)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        out[str(p)] = {"solves_per_s": 1e3 / ms, "ms": ms, "iterations": r.iterations,
                       "status": r.status_name, "relres_true": r.relres_true,
                       "ms_per_iteration": r.device_ms / max(r.iterations, 1)}
    return out


PRECISION_METHODS = [
    # name, precision, solver options, repetitions
    ("fp64_pipe", 0, {}, 1),
    ("fp64_sliced", 4, {}, 2),
    ("fp32_refine", 1, {"mixed_method": 1}, 2),
    ("fp32_precond", 1, {"mixed_method": 2}, 2),
    ("bf16_precond", 2, {"mixed_method": 2}, 2),
    ("fp8_precond", 3, {"mixed_method": 2}, 2),
    ("bf16_refine", 2, {"mixed_method": 1, "max_outer": 12}, 1),
    ("fp8_refine", 3, {"mixed_method": 1, "max_outer": 12}, 1),
]


def precision_lines(ccg, stream, A, p=16, tol=TOL, seed=2):
    """The precision workload at full size: A (FP64, on the device) is the
    exponential kernel on n points (length 0.1, nugget 1e-3), b ~ N(0, 1);
    FP64 cCG (FP64 pipe and sliced product), then A in FP32 / BF16 / FP8 by
    refinement and by the preconditioned FP64 solve.  Each line states its
    true relative residual and its distance to the FP64 (FP64-pipe) answer."""
    import torch
    n = A.shape[0]
    dev = A.device
    g = torch.Generator(device=dev)
    g.manual_seed(seed)
    b = torch.randn(n, dtype=torch.float64, device=dev, generator=g)
    bn = float(torch.linalg.vector_norm(b))
    out = {"workload": f"exponential kernel, n = {n} points U[0,1]^3 (seed {seed}), length 0.1, "
                       f"nugget 1e-3, b ~ N(0,1), p = {p}, tol {tol}", "n": n, "p": p}
    x64 = None
    for name, prec, opts, reps in PRECISION_METHODS:
        x = torch.zeros(n, dtype=torch.float64, device=dev)
        with ccg.Solver(stream=stream.cuda_stream, precision=prec, **opts) as s:
            s.solve(A, b, x, p=p, tol=tol, maxit=2)  # warm-up (kernels, workspace)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            rs = [s.solve(A, b, x, p=p, tol=tol, maxit=20000) for _ in range(reps)]
            e1.record(stream)
            torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        r = rs[-1]
        relres = float(torch.linalg.vector_norm(b - A @ x)) / bn
        line = {"solves_per_s": 1e3 / ms, "ms_per_solve": ms, "status": r.status_name,
                "iterations": r.iterations, "outer_steps": r.outer_steps,
                "relres_true": relres}
        if x64 is None:
            x64 = x.clone()
        else:
            line["err_vs_fp64"] = float(torch.linalg.vector_norm(x - x64) /
                                        torch.linalg.vector_norm(x64))
        out[name] = line
    for k, _, _, _ in PRECISION_METHODS[1:]:
        ok = out[k]["status"] == "CCG_OK"
        out[k]["speedup_vs_fp64_pipe"] = (out[k]["solves_per_s"] / out["fp64_pipe"]["solves_per_s"]
                                          if ok else None)
        out[k]["speedup_vs_fp64_sliced"] = (out[k]["solves_per_s"] /
                                            out["fp64_sliced"]["solves_per_s"] if ok else None)
    return out


def fp64_dgemm_tflops(dev, n=8192, reps=5):
    """FP64 rate of this GPU as cuBLAS DGEMM reaches it (torch.matmul,
    2 n^3 flops, best of reps): the measured FP64 peak of the roofline."""
    import torch
    a = torch.randn(n, n, dtype=torch.float64, device=dev)
    b = torch.randn(n, n, dtype=torch.float64, device=dev)
    torch.matmul(a, b)
    torch.cuda.synchronize()
    best = None
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        torch.matmul(a, b)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        best = ms if best is None else min(best, ms)
    del a, b
    return 2.0 * n ** 3 / (best / 1e3) / 1e12


def batched_line(ccg, dev, stream, count=4096, p=4, seed=3):
    """4096 independent systems, n log-uniform in [32, 1024], A = G G^T / n +
    s I with s ~ U(0.05, 1), b ~ N(0, 1) (generated on the device), one
    persistent launch each in FP64 and in FP32 + FP64 refinement."""
    import numpy as np
    import torch
    rng = np.random.default_rng(seed)
    sizes = [int(v) for v in np.round(np.exp(rng.uniform(np.log(32), np.log(1024), count)))]
    shifts = rng.uniform(0.05, 1.0, count)
    a_off, v_off, at, vt = ccg.batch_offsets(sizes)
    Ap = torch.zeros(at, dtype=torch.float64, device=dev)
    g = torch.Generator(device=dev)
    g.manual_seed(seed)
    for n, sh, ao in zip(sizes, shifts, a_off):
        G = torch.randn(n, n, dtype=torch.float64, device=dev, generator=g)
        ld = n + (n & 1)
        blk = Ap[ao:ao + n * ld].view(n, ld)
        blk[:, :n] = G @ G.T / n
        blk.diagonal().add_(float(sh))
    bp = torch.randn(vt, dtype=torch.float64, device=dev, generator=g)
    nsq = float(np.sum(np.array(sizes, dtype=np.float64) ** 2))
    out = {"workload": f"{count} systems, n log-uniform [32, 1024], A = G G^T/n + U(0.05,1) I, "
                       f"p = {p}, tol 1e-10, one launch per batch", "systems": count,
           "a_bytes_fp64": 8.0 * nsq}
    for name, prec in (("fp64", ccg.FP64), ("fp32_ir", ccg.FP32_IR)):
        x = torch.zeros_like(bp)
        with ccg.Solver(stream=stream.cuda_stream, precision=prec) as s:
            s.solve_batched(sizes, Ap, bp, x, p=p, tol=TOL, maxit=20000)   # warm-up, tunes
            summ, st, it, rr = s.solve_batched(sizes, Ap, bp, x, p=p, tol=TOL, maxit=20000)
            table = s.batch_tuning(p, prec)
        t = summ.device_ms / 1e3
        line = {"solves_per_s": count / t, "ms": summ.device_ms, "status": summ.status_name,
                "all_ok": bool(np.all(st == 0)), "max_relres": float(np.max(rr)),
                "iterations_total": int(np.sum(it)), "ctas": summ.ctas,
                "apass_variant_by_size_bucket": table}
        if prec == ccg.FP64:
            flops = float(np.sum(2.0 * np.array(sizes, dtype=np.float64) ** 2 * p * it))
            line["fp64_tflops"] = flops / t / 1e12
        else:
            line["outer_steps_max"] = summ.outer_steps
        out[name] = line
    out["speedup_fp32_ir_vs_fp64"] = (out["fp32_ir"]["solves_per_s"] / out["fp64"]["solves_per_s"]
                                      if out["fp32_ir"]["all_ok"] else None)
    return out


def serving_line(ccg, dev, precision, count=48, rate=2000.0, seed=4, workers=8, slots=0):
    """Poisson arrivals (mean 2000/s) of SPD solves with A drawn from a pool of
    16 device-resident exponential-kernel matrices (n log-uniform in
    [256, 16384], length U(0.05, 0.5), nugget 10^U(-4, -1)), tol in
    {1e-6, 1e-10}, p = 8, budget 150 GB.  Latency = completion - arrival."""
    import numpy as np
    import torch
    rng = np.random.default_rng(seed)
    pool = []
    for k in range(16):
        n = int(np.round(np.exp(rng.uniform(np.log(256), np.log(16384)))))
        A = device_exp_kernel(n, 1000 + k, float(rng.uniform(0.05, 0.5)),
                              float(10 ** rng.uniform(-4, -1)), dev)
        if slots and n % 2:
            # the serving kernel streams A with 16-byte loads: even leading dimension
            Ap = torch.zeros((n, n + 1), dtype=torch.float64, device=dev)
            Ap[:, :n] = A
            A = Ap
        pool.append(A)
    arrivals = np.cumsum(rng.exponential(1.0 / rate, count))
    picks = rng.integers(0, len(pool), count)
    tols = rng.choice([1e-6, 1e-10], count)
    bs = [torch.randn(pool[k].shape[0], dtype=torch.float64, device=dev) for k in picks]
    xs = [torch.zeros_like(b) for b in bs]
    torch.cuda.synchronize()
    srv = ccg.Server(workers=workers, precision=precision, budget_bytes=150e9, slots=slots,
                     max_n=16384)
    t0 = srv.stats()["now_ms"]
    got = {}
    k = 0
    while len(got) < count:
        now = srv.stats()["now_ms"] - t0
        while k < count and arrivals[k] * 1e3 <= now:
            rc = srv.submit(k, pool[picks[k]], bs[k], xs[k], p=8, tol=float(tols[k]), maxit=50000)
            if rc != 0:
                raise RuntimeError(f"submit failed: {rc}")
            k += 1
        for r in srv.poll(64, wait_ms=1):
            got[r["id"]] = r
    peak = srv.stats()
    srv.close()
    lat = np.array([got[i]["done_ms"] - (t0 + arrivals[i] * 1e3) for i in range(count)])
    span = max(r["done_ms"] for r in got.values()) - t0
    ok = sum(1 for r in got.values() if r["status"] == 0)
    return {"requests": count, "ok": ok, "p50_ms": float(np.percentile(lat, 50)),
            "p99_ms": float(np.percentile(lat, 99)), "solves_per_s": count / (span / 1e3),
            "peak_in_flight": peak["peak_in_flight"],
            "peak_reserved_gb": peak["peak_reserved_bytes"] / 1e9}


def run_reference(args, rank, world):
    """The oracle arm: warm-up steps time short samples; each timed step is one
    full FP64 oracle solve of the benchmark system on the host cores."""
    if rank != 0:
        return
    A, b = workload(args.n)
    for _ in range(args.warmup):
        cpu_sample(A, b, args.p, 1.0)
    secs, its = [], None
    cores = os.cpu_count() or 1
    for _ in range(args.steps):
        t, cores, its = cpu_full_solve(A, b, args.p)
        secs.append(t)
    total = sum(secs)
    value = args.steps / total
    sample = (f"{args.steps} full oracle solves (n={args.n}, p={args.p}, {its} iterations each, "
              f"{statistics.mean(secs):.1f} s each on {cores} threads)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 * total / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": run_config(args.n, args.p, args.product),
            "cpu_baseline": {"value": value, "unit": "solves/s", "cores": cores,
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def detail(name, obj):
    """One additional measurement on its own output line."""
    print(json.dumps({"detail": name, **obj}), flush=True)


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import numpy as np
    import torch
    import __graft_entry__ as ge
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if rank == 0 or world == 1:
        ge.build()
    if dist is not None:
        dist.barrier()
    from paper_1204_0069_gb300 import ccg

    n, p = args.n, args.p
    A, b = workload(n)
    dev = torch.device("cuda", local)
    dA = torch.from_numpy(A).to(dev)
    db = torch.from_numpy(b).to(dev)
    x = torch.zeros(n, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)
    prec = ccg.FP64_SLICED if args.product == "sliced" else ccg.FP64
    solver = ccg.Solver(device=local, stream=stream.cuda_stream, precision=prec)
    maxit = args.maxit if args.maxit > 0 else 20 * n

    if args.profile == "mixed":
        # mixed-precision (FP32_IR) solves of the benchmark system
        with ccg.Solver(stream=stream.cuda_stream, precision=ccg.FP32_IR) as sm:
            for _ in range(args.warmup + args.steps):
                r = sm.solve(dA, db, x, p=p, tol=TOL, maxit=maxit)
                print(json.dumps({"status": r.status_name, "iterations": r.iterations,
                                  "outer": r.outer_steps, "ms": r.device_ms}), flush=True)
        solver.close()
        return
    if args.profile in ("lowp32", "sliced"):
        # FP32 (TF32x3) or sliced FP64 block products of the benchmark matrix
        # through the persistent kernel's tensor-core A-pass
        m = solver.lowp_matrix(dA, ccg.LOWP_FP32 if args.profile == "lowp32"
                               else ccg.LOWP_FP64_SLICED)
        V = torch.randn(n, p, dtype=torch.float64, device=dev)
        W = torch.empty(n, p, dtype=torch.float64, device=dev)
        for _ in range(args.warmup + args.steps):
            rc, ms = m.block_product(V, W)
            print(json.dumps({"rc": rc, "ms": ms}), flush=True)
        m.close()
        solver.close()
        return
    if args.profile == "batched":
        # the batched FP64 solver on the first 512 systems of the batching
        # family, default A-pass shapes (no autotuning launches)
        import numpy as np
        rng = np.random.default_rng(3)
        sizes = [int(v) for v in np.round(np.exp(rng.uniform(np.log(32), np.log(1024), 512)))]
        shifts = rng.uniform(0.05, 1.0, 512)
        a_off, v_off, at, vt = ccg.batch_offsets(sizes)
        Ap = torch.zeros(at, dtype=torch.float64, device=dev)
        g = torch.Generator(device=dev)
        g.manual_seed(3)
        for nn, sh, ao in zip(sizes, shifts, a_off):
            G = torch.randn(nn, nn, dtype=torch.float64, device=dev, generator=g)
            blk = Ap[ao:ao + nn * (nn + (nn & 1))].view(nn, nn + (nn & 1))
            blk[:, :nn] = G @ G.T / nn
            blk.diagonal().add_(float(sh))
        bp = torch.randn(vt, dtype=torch.float64, device=dev, generator=g)
        xb = torch.zeros_like(bp)
        with ccg.Solver(stream=stream.cuda_stream, batch_autotune=False) as sb:
            for _ in range(args.warmup + args.steps):
                summ, st, it, rr = sb.solve_batched(sizes, Ap, bp, xb, p=4, tol=TOL, maxit=20000)
                print(json.dumps({"status": summ.status_name, "ms": summ.device_ms,
                                  "iterations": int(np.sum(it)),
                                  "fp64_flops": float(np.sum(2.0 * np.array(sizes, dtype=float) ** 2
                                                             * 4 * it))}), flush=True)
        solver.close()
        return
    if args.profile == "cheb":
        # the preconditioned FP8 solve of the precision family, two FP64
        # iterations: the launches are solve, preconditioner, solve, ...
        A32 = device_exp_kernel(args.lowp_n, 2, 0.1, 1e-3, dev)
        b32 = torch.randn(args.lowp_n, dtype=torch.float64, device=dev)
        with ccg.Solver(stream=stream.cuda_stream, mixed_method=ccg.MIXED_PRECOND) as sp:
            m = sp.lowp_matrix(A32, ccg.LOWP_FP8_E4M3)
            x32 = torch.zeros(args.lowp_n, dtype=torch.float64, device=dev)
            for _ in range(args.warmup + args.steps):
                r = sp.solve_mixed(m, A32, b32, x32, p=p, tol=TOL, maxit=2)
                if r.status not in (0, 1):
                    raise RuntimeError(f"status {r.status}")
            m.close()
        torch.cuda.synchronize()
        solver.close()
        print(json.dumps({"profile": "cheb", "n": args.lowp_n, "p": p}))
        return
    if args.profile == "lowp":
        A32 = device_exp_kernel(args.lowp_n, 2, 0.1, 1e-3, dev)
        m = solver.lowp_matrix(A32, ccg.LOWP_BF16 if args.lowp_fmt == "bf16" else ccg.LOWP_FP8_E4M3)
        del A32
        torch.cuda.empty_cache()
        V = torch.randn(args.lowp_n, p, dtype=torch.float64, device=dev)
        W = torch.empty(args.lowp_n, p, dtype=torch.float64, device=dev)
        for _ in range(args.warmup + args.steps):
            if m.block_product(V, W)[0] != 0:
                raise RuntimeError("block product failed")
        torch.cuda.synchronize()
        m.close()
        solver.close()
        print(json.dumps({"profile": "lowp", "fmt": args.lowp_fmt, "n": args.lowp_n, "p": p}))
        return
    if args.profile != "none":
        # profiling mode: the launches ncu captures, nothing else timed
        V = torch.randn(n, p, dtype=torch.float64, device=dev)
        W = torch.empty(n, p, dtype=torch.float64, device=dev)
        for _ in range(args.warmup + args.steps):
            if args.profile == "block":
                rc = solver.block_product(dA, V, W, want_grams=True)[0]
            else:
                rc = solver.solve(dA, db, x, p=p, tol=TOL, maxit=maxit).status
            if rc not in (0, 1):
                raise RuntimeError(f"status {rc}")
        torch.cuda.synchronize()
        solver.close()
        print(json.dumps({"profile": args.profile, "n": n, "p": p, "launches": args.steps + args.warmup}))
        return

    def step():
        r = solver.solve(dA, db, x, p=p, tol=TOL, maxit=maxit)
        if r.status != 0:
            raise RuntimeError(f"solve failed: {r}")
        return r

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    clocks = ClockSampler(local)
    clocks.start()
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    results = [step() for _ in range(args.steps)]
    e1.record(stream)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    clk = clocks.stop()
    elapsed = e0.elapsed_time(e1) / 1000.0
    elapsed = max_over_ranks(elapsed, dist, dev)
    value = job_throughput(world, args.steps, elapsed)
    kernel_ms = [r.device_ms for r in results]
    r0 = results[-1]

    # end to end through the C ABI with pinned host buffers
    e2e = None
    if not args.no_e2e:
        hA = torch.from_numpy(A).pin_memory()
        hb = torch.from_numpy(b).pin_memory()
        hx = torch.zeros(n, dtype=torch.float64).pin_memory()
        solver.solve(hA, hb, hx, p=p, tol=TOL, maxit=maxit)
        torch.cuda.synchronize()
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        for _ in range(args.steps):
            r = solver.solve(hA, hb, hx, p=p, tol=TOL, maxit=maxit)
            if r.status != 0:
                raise RuntimeError(f"e2e solve failed: {r}")
        f1.record(stream)
        torch.cuda.synchronize()
        et = f0.elapsed_time(f1) / 1000.0
        et = max_over_ranks(et, dist, dev)
        e2e = {"value": job_throughput(world, args.steps, et), "unit": "solves/s",
               "h2d_bytes_per_step": int(A.nbytes + b.nbytes),
               "d2h_bytes_per_step": int(8 * n + 192)}

    peaks = measured_peaks()
    hbm = peaks.get("hbm_gbs")
    targets = {}
    if rank == 0 and not args.no_mixed:
        from paper_1204_0069_gb300 import workloads as wl
        fp64_tf = fp64_dgemm_tflops(dev)
        detail("fp64_peak", {"dgemm_tflops": fp64_tf,
                             "how": "torch.matmul FP64 8192^3 (cuBLAS DGEMM), best of 5"})
        with ccg.Solver(stream=stream.cuda_stream) as s64:
            sweep = p_sweep(ccg, s64, stream, dA, db, x, n)
        sweep_sliced = sliced_sweep(ccg, stream, dA, db, x, n)
        golden = {str(q): oracle_golden_iterations(n, q) for q in (1, 4, 8, 16, 32)}
        detail("p_sweep_n8192", {"fp64_pipe": sweep, "fp64_sliced": sweep_sliced,
                                 "oracle_iterations_stored": golden})
        qs = (1, 4, 8, 16, 32)
        targets["p_sweep_n8192"] = {
            "p": list(qs),
            "it_oracle_stored": [golden[str(q)] for q in qs],
            "it_pipe": [sweep[str(q)]["iterations"] for q in qs],
            "it_sliced": [sweep_sliced[str(q)]["iterations"] if str(q) in sweep_sliced else None
                          for q in qs],
            "ms_pipe": [round(sweep[str(q)]["ms"], 1) for q in qs],
            "ms_sliced": [round(sweep_sliced[str(q)]["ms"], 1) if str(q) in sweep_sliced
                          else None for q in qs]}
        A3 = device_exp_kernel(args.lowp_n, 2, 0.1, 1e-3, dev)
        lowp = lowp_roofline(ccg, solver, dev, A3, 16, hbm)
        detail("apass_lowp_n32768", lowp)
        targets["apass_frac_of_measured_hbm_n32768_p16"] = {
            k.split("_")[0] if k != "fp64_sliced" else "sliced":
            round(v["frac_of_measured_hbm"], 3) if v["frac_of_measured_hbm"] else None
            for k, v in lowp.items()}
        precision = precision_lines(ccg, stream, A3, p=16)
        detail("precision_n32768", precision)
        del A3
        torch.cuda.empty_cache()
        def prow(v):
            sp = [round(v[k], 2) if v.get(k) else None
                  for k in ("speedup_vs_fp64_pipe", "speedup_vs_fp64_sliced")]
            return [round(v["solves_per_s"], 3), v["status"].replace("CCG_", ""),
                    float("%.1e" % v["relres_true"]),
                    float("%.1e" % v["err_vs_fp64"]) if "err_vs_fp64" in v else None] + sp
        targets["precision_n32768_p16"] = {
            "cols": ["solves/s", "status", "relres", "err_vs_fp64", "x_vs_pipe", "x_vs_sliced"],
            **{k: prow(precision[k]) for k, _, _, _ in PRECISION_METHODS}}
        mixed = {"exp_kernel_n8192": mixed_lines(ccg, dev, stream, A, b, p, 2)}
        Ag, bg = wl.gram_shift(n, seed=3, shift=0.5)
        mixed["gram_shift_n8192"] = mixed_lines(ccg, dev, stream, Ag, bg, p, 3)
        detail("mixed_n8192", mixed)
        batched = batched_line(ccg, dev, stream)
        detail("batched", batched)
        targets["batched_4096"] = {"fp64_solves_per_s": round(batched["fp64"]["solves_per_s"]),
                                   "fp32_ir_solves_per_s": round(batched["fp32_ir"]["solves_per_s"]),
                                   "all_ok": batched["fp64"]["all_ok"] and batched["fp32_ir"]["all_ok"]}
        serving = {"workload": ("Poisson(2000/s) arrivals, A from a pool of 16 device-resident "
                                "exponential-kernel matrices, n log-uniform [256, 16384], "
                                "tol {1e-6, 1e-10}, p = 8, budget 150 GB; 8 workers, or one "
                                "serving kernel with 8 slots (fp64_pipe_slots)")}
        for name, pr, sl in (("fp64_sliced", ccg.FP64_SLICED, 0), ("fp32", ccg.FP32_IR, 0),
                             ("bf16", ccg.BF16_IR, 0), ("fp8", ccg.FP8_IR, 0),
                             ("fp64_pipe", ccg.FP64, 0), ("fp64_pipe_slots", ccg.FP64, 8)):
            serving[name] = serving_line(ccg, dev, pr, slots=sl)
        # a longer window of arrivals for the fastest path
        serving["fp8_400_arrivals"] = serving_line(ccg, dev, ccg.FP8_IR, count=400)
        detail("serving", serving)
        targets["serving_p50_p99_ms"] = {k: [round(v["p50_ms"]), round(v["p99_ms"])]
                                         for k, v in serving.items() if isinstance(v, dict)}
        targets["fp64_dgemm_tflops"] = round(fp64_tf, 3)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, cores, sample = cpu_sample(A, b, p, args.cpu_seconds)
        cpu = {"value": v, "unit": "solves/s", "cores": cores, "kind": "oracle",
               "sample": sample}

    if rank == 0:
        checks = 1 + r0.replacements
        kms = statistics.mean(kernel_ms)
        passes = 1 + r0.iterations + r0.replacements
        if args.product == "sliced":
            # the sliced A (14 n^2 bytes) per block product, the FP64 A per check
            byts = 14.0 * n * n * passes + 8.0 * n * n * checks + 80.0 * n * p * r0.iterations
            achieved = byts / (kms / 1e3) / 1e9
            per_pass = NCU_BYTES_PER_PASS.get(("sliced", n, p))
            roof = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                    "frac": achieved / hbm if hbm else None,
                    "traffic": (per_pass * passes + 8.0 * n * n * checks) if per_pass else None,
                    "kernel": f"fp64_kernel<{p_bucket(p)},true,POL_SLICED>",
                    "note": "14n^2 B per block product, 8n^2 per FP64 check; peak measured"}
        else:
            fl = solve_flops(n, p, r0.iterations, checks, r0.replacements)
            achieved = fl / (kms / 1e3) / 1e12
            fp64_peak = 1.25
            per_pass = NCU_BYTES_PER_PASS.get(("fp64", n, p))
            roof = {"bound": "alu", "achieved": achieved, "peak": fp64_peak, "unit": "TFLOP/s",
                    "frac": achieved / fp64_peak,
                    "traffic": per_pass * (passes + checks) if per_pass else None,
                    "kernel": f"fp64_kernel<{p_bucket(p)},true>",
                    "note": "nominal FP64 peak (targets.fp64_dgemm_tflops: measured)"}
        line = {
            "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 * elapsed / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": run_config(n, p, args.product),
            "iterations": r0.iterations, "relres_true": r0.relres_true,
            "roofline": roof, "clocks": clk,
            # per step: the slicing of A and the persistent solve (sliced), or the solve
            "gpu_launches": (2 if args.product == "sliced" else 1) * args.steps,
        }
        if e2e is not None:
            line["e2e"] = e2e
        if cpu is not None:
            line["cpu_baseline"] = cpu
        if targets:
            line["targets"] = targets
        print(json.dumps(line, separators=(",", ":")), flush=True)
    solver.close()
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
