#!/usr/bin/env python3
"""Benchmark: one DFC-LRR solve (Algorithm 1: D step input, all t block ALM
solves, column projection) per step on a synthetic union-of-subspaces input,
timed on the GPU, plus an end-to-end run from host buffers, a roofline entry
for the dominant kernel family and the CPU oracle as a baseline.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun with N > 1 every rank solves its own replica of the workload
(the solve is one batch on one GPU; there is no inter-GPU exchange).
"""
from __future__ import annotations

import argparse
import atexit
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "DFC-LRR solve s & ALM iter/s, batched mixed vs plain FP32 at rel err ≤1e-5"


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            pk = json.load(f)
        return pk, "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "sm_max_mhz": 2070.0}, \
            "fallback"


# FP32 CUDA-core peak: 152 SMs x 128 FP32 lanes x 2 flop (FMA) x max SM clock
def fp32_alu_peak_tflops(sm_mhz: float) -> float:
    return 152 * 128 * 2 * sm_mhz * 1e6 / 1e12


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.proc = None
        self.gpu = gpu_index
        self.path = os.path.join(tempfile.gettempdir(), f"dfc_lrr_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
            atexit.register(self._kill)
        except OSError:
            self.proc = None

    def _kill(self):
        if self.proc is not None and self.proc.poll() is None:
            self.proc.kill()

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["not sampled"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------ algorithmic work
def algorithmic_work(w, rank_M, iters):
    """Per-phase algorithmic flop and byte counts of one solve, from the
    problem sizes, rank(M) and the per-block iteration counts."""
    m, n = w.M.shape
    r = rank_M
    l = np.diff(w.offsets)
    it = np.asarray(iters, dtype=np.float64)
    fb = 4  # float32
    out = {}
    # U^T P and U diag(sigma) Z: 2 r m l flops per block-iteration; bytes: read the
    # m x l and r x l operands and U once, write the r x l / m x l result
    out["zgemm"] = {"flops": float(np.sum(it * 2 * r * m * l)),
                    "bytes": float(np.sum(it * fb * (m * l + r * l))) + fb * m * r * float(it.max())}
    out["mzgemm"] = dict(out["zgemm"])
    # Gram: tall blocks A^T A (2 l^2 r), wide A A^T (2 r^2 l)
    g = np.where(l <= r, 2.0 * l * l * r, 2.0 * r * r * l)
    out["gram"] = {"flops": float(np.sum(it * g)), "bytes": float(np.sum(it * fb * r * l))}
    return _elementwise(out, w, r, m, l, it, fb)


def jacobi_work(w, rank_M, sweeps):
    """Flops of the Jacobi sweeps, given the per-block sweep counts.

    Returns (method, implementation):
      method          4 p^3 per block-sweep: the eigensolve of the p x p Gram
                      of the SVT input, one cyclic sweep (p = min(rank(M), l));
      implementation  8 L p^2 + 4 p^3 per block-sweep: what the one-sided
                      block Jacobi executes (every pivot Gram formed afresh
                      from the L-long columns, 4 L p^2 over a sweep, plus the
                      rotations of X and W, 4 (L + p) p^2), L = rank(M) for a
                      tall block and L = l for a wide one."""
    r = rank_M
    l = np.diff(w.offsets).astype(np.float64)
    L = np.where(l <= r, r, l)
    p = np.where(l <= r, l, r)
    sw = np.asarray(sweeps, dtype=np.float64)
    return float(np.sum(sw * 4 * p ** 3)), float(np.sum(sw * (8 * L * p * p + 4 * p ** 3)))


def _elementwise(out, w, r, m, l, it, fb):
    # element-wise kernels: bytes moved per block-iteration
    out["zupdate"] = {"flops": float(np.sum(it * 9 * r * l)), "bytes": float(np.sum(it * fb * r * l * 7))}
    out["eupdate"] = {"flops": float(np.sum(it * 14 * m * l)), "bytes": float(np.sum(it * fb * m * l * 8))}
    return out


def workload_config(args, w, world: int) -> dict:
    """The `config` object of both arms' JSON lines: the workload and how it is
    run (the oracle arm times the same workload)."""
    m, n = w.M.shape
    return {"workload": args.workload, "m": int(m), "n": int(n), "t": int(w.t), "lambda": w.lam, "eps": w.eps,
            "precision": args.precision, "batched": not args.sequential,
            "parallelism": "replicas" if world > 1 else "single", "autotune": not args.no_autotune,
            "l2": "no flush: the per-iteration working set (C, P, MZ, E, Y1 and the reduced state) "
                  "exceeds the 129 MB L2"}


def replica_seed(seed: int, rank: int) -> int:
    """Seed of the workload replica a rank solves: the solve is one batch on
    one GPU, so N GPUs run N independent replicas (weak scaling)."""
    return seed + rank


def max_over_ranks(x: float, world: int, device=None) -> float:
    """The slowest rank's value (every rank gets it); x itself when world == 1."""
    if world <= 1:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def bench_ours(args, rank, world):
    import torch
    from paper_1304_5583_gb300 import binding, synth
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    w = synth.workload(args.workload, seed=replica_seed(args.seed, rank))
    m, n = w.M.shape
    dt = np.float64 if args.precision == "f64" else np.float32
    Mh = np.asfortranarray(w.M.astype(dt))
    Md = torch.from_numpy(Mh).to(dev)
    opts = binding.options(w.lam, rho=w.rho, mu0=w.mu0, mu_max=w.mu_max, eps=w.eps, max_iter=w.max_iter,
                           precision=args.precision, batched=not args.sequential, profile=True,
                           autotune=not args.no_autotune)
    ws = torch.empty(binding.workspace_bytes(binding.column_major(Md), w.perm, w.offsets, opts), dtype=torch.uint8,
                     device=dev)

    def step():
        return binding.dfc_lrr_solve(Md, w.perm, w.offsets, opts, workspace=ws)

    for _ in range(args.warmup):
        res = step()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clocks = ClockSampler(dev.index)
    if not args.no_clocks:
        clocks.start()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    try:
        torch.cuda.synchronize()
        e0.record(stream)
        results = []
        for _ in range(args.steps):
            results.append(step())
        e1.record(stream)
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
    finally:
        # the sampler is a child process: never leave it running (a profiler
        # waits for every child of its target before it exits)
        clk = clocks.stop()
    ms = max_over_ranks(e0.elapsed_time(e1) / args.steps, world, dev)
    res = results[-1]
    for r_ in results:
        if r_.status < 0:
            raise RuntimeError(f"solve failed: {binding.status_string(r_.status)}")
    iters_total = int(np.sum(res.iters))
    launches = int(np.mean([r_.stats["launches"] for r_ in results]))

    # per-phase times over the timed steps
    phase_ms = {k: float(np.mean([r_.stats["phase_ms"][k] for r_ in results])) for k in binding.PHASES}
    phase_launch = {k: int(np.mean([r_.stats["phase_launches"][k] for r_ in results])) for k in binding.PHASES}

    # ---- end to end: host M (pinned) -> device, solve, Z and S back to pinned host buffers
    Mpin = torch.empty((n, m), dtype=Md.dtype, pin_memory=True).t()
    Mpin.copy_(torch.from_numpy(Mh))
    Zh = torch.empty((n, n), dtype=Md.dtype, pin_memory=True).t()
    Sh = torch.empty((n, m), dtype=Md.dtype, pin_memory=True).t()
    e_steps = max(1, args.e2e_steps)
    torch.cuda.synchronize()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    for _ in range(e_steps):
        Mdev = torch.empty((n, m), dtype=Md.dtype, device=dev).t()
        Mdev.copy_(Mpin, non_blocking=True)
        rr = binding.dfc_lrr_solve(Mdev, w.perm, w.offsets, opts, workspace=ws)
        Zh.copy_(rr.Z, non_blocking=True)
        Sh.copy_(rr.S, non_blocking=True)
    f1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = f0.elapsed_time(f1) / e_steps
    h2d = Mh.nbytes
    d2h = Zh.numel() * Zh.element_size() + Sh.numel() * Sh.element_size()

    # ---- the same with Z returned in factored form (Z = F[:, :k] G[:k], Section
    #      2.2's low-rank output) instead of the dense n x n matrix
    kmax = binding.factor_max_rank(Md, w.perm, w.offsets)
    Fh = torch.empty((kmax, n), dtype=Md.dtype, pin_memory=True).t()
    Gh = torch.empty((n, kmax), dtype=Md.dtype, pin_memory=True).t()
    torch.cuda.synchronize()
    g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    g0.record(stream)
    for _ in range(e_steps):
        Mdev = torch.empty((n, m), dtype=Md.dtype, device=dev).t()
        Mdev.copy_(Mpin, non_blocking=True)
        rr = binding.dfc_lrr_solve(Mdev, w.perm, w.offsets, opts, workspace=ws, want_Z=False, want_factors=True)
        Fh.copy_(rr.F, non_blocking=True)
        Gh.copy_(rr.G, non_blocking=True)
        Sh.copy_(rr.S, non_blocking=True)
    g1.record(stream)
    torch.cuda.synchronize()
    e2e_fact_ms = g0.elapsed_time(g1) / e_steps
    d2h_fact = (Fh.numel() + Gh.numel() + Sh.numel()) * Sh.element_size()

    # ---- roofline of the dominant kernel family
    peaks, src = _peaks()
    work = algorithmic_work(w, res.rank_M, res.iters)
    jm, ji = jacobi_work(w, res.rank_M, res.sweeps)
    work["jacobi"] = {"flops": jm, "flops_impl": ji, "bytes": None}
    loop_phases = [k for k in binding.PHASES if k not in ("setup", "combine", "host")]
    dom = max(loop_phases, key=lambda k: phase_ms[k])
    sm_max = peaks.get("sm_max_mhz", 2070.0)
    roof = None
    if dom in work and phase_ms[dom] > 0:
        wk = work[dom]
        sec = phase_ms[dom] / 1e3
        if dom in ("zupdate", "eupdate"):
            ach = wk["bytes"] / sec / 1e9
            roof = {"bound": "hbm", "achieved": ach, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                    "frac": ach / peaks["hbm_gbs"], "traffic": None, "kernel": dom, "peak_source": src}
        else:
            ach = wk["flops"] / sec / 1e12
            pk = fp32_alu_peak_tflops(sm_max) if args.precision != "f64" else 1.19
            roof = {"bound": "alu", "achieved": ach, "peak": pk, "unit": "TFLOP/s", "frac": ach / pk,
                    "traffic": None, "kernel": dom,
                    "peak_source": "derived: 152 SM x 128 FP32 lanes x 2 x sm_max_mhz"}
            if "flops_impl" in wk:
                roof["count"] = "4 p^3 per block-sweep (the p x p Gram eigensolve), per-block sweep counts"
                roof["achieved_impl"] = wk["flops_impl"] / sec / 1e12
                roof["frac_impl"] = roof["achieved_impl"] / pk
                roof["count_impl"] = "8 L p^2 + 4 p^3 per block-sweep (fresh pivot Grams + rotations)"
    else:
        roof = {"bound": "alu", "achieved": None, "peak": fp32_alu_peak_tflops(sm_max), "unit": "TFLOP/s",
                "frac": None, "traffic": None, "kernel": dom,
                "note": "dominant phase has no closed-form algorithmic count"}
    solve_s = ms / 1e3
    dtype = {"f64": "f64", "f32": "f32", "mixed": "bf16+f32"}[args.precision]
    line = {
        "metric": METRIC, "value": solve_s, "unit": "s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": dtype, "data": "synthetic",
        "config": workload_config(args, w, world),
        "rank_M": res.rank_M, "k1": res.k1,
        "alm_iters_per_s": float(np.max(res.iters)) / solve_s,
        "block_iters_per_s": iters_total / solve_s,
        "iters": {"max": int(np.max(res.iters)), "sum": iters_total, "per_block": res.iters.tolist()},
        "phase_ms": phase_ms, "phase_launches": phase_launch,
        "svt": {"sweeps": res.stats["svt_sweeps"], "calls": res.stats["svt_calls"]},
        "roofline": roof,
        "e2e": {"value": e2e_ms / 1e3, "unit": "s", "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)},
        "e2e_factored": {"value": e2e_fact_ms / 1e3, "unit": "s", "h2d_bytes_per_step": int(h2d),
                         "d2h_bytes_per_step": int(d2h_fact), "k": int(rr.factor_k), "kmax": int(kmax)},
        "gpu_launches": launches * args.steps,
        "clocks": clk,
    }
    line["svt"]["sweeps_per_block"] = res.sweeps.tolist()
    if not args.no_compare and not args.sequential and rank == 0:
        if args.precision == "mixed":
            # the same batched solve in plain float32: separates the gain of
            # the bf16 products from that of batching
            line["fp32_batched"] = compare_sequential(binding, w, Md, dev, stream, res, batched=True)
        line["fp32_one_block_at_a_time"] = compare_sequential(binding, w, Md, dev, stream, res)
    return line, w, res


def compare_sequential(binding, w, Md, dev, stream, res_batched, warmup=0, steps=1, batched=False):
    """The plain float32 form on the same input, solving the blocks one after
    another (batched=False: the comparison point for the batched mixed solve)
    or all together (batched=True).  Returns its solve time, iteration counts
    and the relative Frobenius difference of its Z against the batched
    solve's Z.  One solve, not warmed up (the kernels are already loaded by
    the batched runs)."""
    import torch
    if Md.dtype != torch.float32:
        return None
    opts = binding.options(w.lam, rho=w.rho, mu0=w.mu0, mu_max=w.mu_max, eps=w.eps, max_iter=w.max_iter,
                           precision="f32", batched=batched, profile=False)
    ws = torch.empty(binding.workspace_bytes(binding.column_major(Md), w.perm, w.offsets, opts), dtype=torch.uint8,
                     device=dev)
    for _ in range(warmup):
        rr = binding.dfc_lrr_solve(Md, w.perm, w.offsets, opts, workspace=ws)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        rr = binding.dfc_lrr_solve(Md, w.perm, w.offsets, opts, workspace=ws)
    e1.record(stream)
    torch.cuda.synchronize()
    if rr.status < 0:
        raise RuntimeError(f"sequential solve failed: {binding.status_string(rr.status)}")
    ms = e0.elapsed_time(e1) / steps
    dz = float(torch.linalg.norm(rr.Z - res_batched.Z) / torch.linalg.norm(rr.Z))
    del ws
    return {"value": ms / 1e3, "unit": "s", "steps": steps, "warmup": warmup, "iters_max": int(np.max(rr.iters)),
            "iters_sum": int(np.sum(rr.iters)), "rel_diff_Z_vs_batched": dz}


# ALM iterations the float64 oracle takes on block 1 of each workload, run to
# convergence (eps of the workload, max_iter 1000) with oracle.lrr.lrr_alm
ORACLE_BLOCK1_ITERS = {"dfc_1000x20000": 213, "dfc_500x5000": 237, "dfc_faces_2016x2432": 243,
                       "plain_lrr_100x500": 279, "small_dfc_60x240": 166}


def oracle_sample(w, n_iter=3, threads=None):
    """Time the float64 oracle on a bounded sample: n_iter ALM iterations of
    block 0 (plus the one-time factor).  Returns (seconds per block-iteration,
    setup seconds, cores used, description)."""
    from oracle import lrr as olrr
    M = w.M
    cols = w.perm[w.offsets[0]:w.offsets[1]]
    t0 = time.perf_counter()
    zs = olrr.ZSolve(M)
    t1 = time.perf_counter()
    olrr.lrr_alm(M[:, cols], M, w.lam, fixed_iters=n_iter, zsolve=zs)
    t2 = time.perf_counter()
    cores = threads or os.cpu_count()
    desc = f"{n_iter} ALM iterations of block 0 ({len(cols)} columns) + the one-time factor, float64 numpy/LAPACK"
    return (t2 - t1) / n_iter, t1 - t0, cores, desc


def oracle_sample_one_thread(workload, seed, n_iter):
    """oracle_sample in a child process restricted to one BLAS/OpenMP thread."""
    env = dict(os.environ, OPENBLAS_NUM_THREADS="1", OMP_NUM_THREADS="1", MKL_NUM_THREADS="1")
    cmd = [sys.executable, os.path.abspath(__file__), "--cpu-sample", "--workload", workload, "--seed", str(seed),
           "--oracle-iters", str(n_iter)]
    try:
        out = subprocess.run(cmd, env=env, capture_output=True, text=True, timeout=600, check=True).stdout
        return json.loads(out.strip().splitlines()[-1])
    except (subprocess.SubprocessError, ValueError, IndexError):
        return None


def extrapolate(w, per_iter_s, setup_s, iters):
    l = np.diff(w.offsets).astype(np.float64)
    l0 = float(l[0])
    # per-iteration cost grows ~ linearly with the block width at fixed m, n
    return setup_s + float(np.sum(np.asarray(iters) * per_iter_s * l / l0))


def bench_gemm(args):
    """The iteration's tensor-core products on their own, at the shape of U^T P
    for the whole batch: M = rank(M), N = n, K = m (1000 x 20000 x 1000 for
    the 1000 x 20000 workload).  Device time per launch from CUDA events
    around `steps` back-to-back launches (lrr_gemm_timing), as a fraction of
    the measured bf16 peak (the split products do three MMAs per term: their
    algorithmic rate counts the float32 product's 2 M N K flops).
    Also the command the tensor-pipe counters are captured from."""
    import torch
    from paper_1304_5583_gb300 import binding
    M, N, K = args.gemm_shape
    torch.cuda.set_device(0)
    peaks, src = _peaks()
    out = {"shape": [M, N, K], "peak_source": src, "bf16_peak_tflops": peaks["bf16_tflops"]}
    for kind in ("bf16", "bf16x3", "3xtf32"):
        ms = binding.gemm_timing(kind, M, N, K, repeat=max(1, args.steps))
        tf = 2.0 * M * N * K / (ms / 1e3) / 1e12
        out[kind] = {"ms_per_launch": ms, "tflops": tf, "frac_of_bf16_peak": tf / peaks["bf16_tflops"]}
    print(json.dumps(out))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gemm-only", action="store_true", help="time lrr_gemm_bf16 alone (see bench_gemm)")
    ap.add_argument("--gemm-shape", type=int, nargs=3, default=[1000, 20000, 1000])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="dfc_1000x20000")
    ap.add_argument("--precision", default="mixed", choices=["f32", "f64", "mixed"])
    ap.add_argument("--sequential", action="store_true", help="solve the blocks one at a time")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--e2e-steps", type=int, default=1)
    ap.add_argument("--no-autotune", action="store_true", help="fixed launch shapes instead of the autotuner")
    ap.add_argument("--oracle-iters", type=int, default=3)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-clocks", action="store_true",
                    help="no nvidia-smi sampling (for runs under a profiler, which waits for child processes)")
    ap.add_argument("--no-compare", action="store_true",
                    help="skip the float32 one-block-at-a-time comparison solve")
    ap.add_argument("--cpu-sample", action="store_true", help=argparse.SUPPRESS)
    args = ap.parse_args()

    if args.cpu_sample:
        # child of oracle_sample_one_thread: time the oracle sample, print it
        from paper_1304_5583_gb300 import synth
        w = synth.workload(args.workload, seed=args.seed)
        p_iter, s_setup, _, desc = oracle_sample(w, n_iter=args.oracle_iters)
        print(json.dumps({"per_iter": p_iter, "setup": s_setup, "desc": desc}))
        return

    if args.gemm_only:
        bench_gemm(args)
        return

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))

    if args.impl == "reference":
        # the oracle arm runs on rank 0's host cores only
        if rank != 0:
            return
        from paper_1304_5583_gb300 import synth
        w = synth.workload(args.workload, seed=args.seed)
        per = []
        for i in range(args.warmup + args.steps):
            p_iter, s_setup, cores, desc = oracle_sample(w, n_iter=1)
            if i >= args.warmup:
                per.append((p_iter, s_setup))
        # the oracle is not run to convergence here (that takes minutes to
        # hours); every block is extrapolated at the iteration count the
        # oracle needs on block 1 of the workload
        it1 = ORACLE_BLOCK1_ITERS.get(args.workload, 250)
        iters = np.full(w.t, it1)
        vals = [extrapolate(w, p, s, iters) for p, s in per]
        v = float(np.mean(vals))
        print(json.dumps({
            "impl": "reference", "metric": METRIC, "value": v, "unit": "s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": v * 1e3, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(args, w, args.gpus),
            "cpu_baseline": {"value": v, "unit": "s", "cores": cores, "kind": "oracle",
                             "sample": desc + f"; extrapolated to all blocks at {it1} iterations each (the "
                                       "oracle's own count on block 1)"},
            "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))
        return

    if world > 1:
        import torch
        torch.distributed.init_process_group("nccl")
    line, w, res = bench_ours(args, rank, world)
    if rank == 0 and not args.no_cpu_baseline:
        p_iter, s_setup, cores, desc = oracle_sample(w, n_iter=args.oracle_iters)
        v = extrapolate(w, p_iter, s_setup, res.iters)
        line["cpu_baseline"] = {"value": v, "unit": "s", "cores": cores, "kind": "oracle",
                                "sample": desc + "; extrapolated to every block at the GPU's iteration counts"}
        # the same sample on one host core (BLAS threads fixed before numpy
        # loads, hence a child process), beside the paper's single-core setting
        one = oracle_sample_one_thread(args.workload, args.seed, 1)
        if one is not None:
            v1 = extrapolate(w, one["per_iter"], one["setup"], res.iters)
            line["cpu_baseline_1thread"] = {"value": v1, "unit": "s", "cores": 1, "kind": "oracle",
                                            "sample": one["desc"] + "; one BLAS thread; extrapolated as above"}
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
