#!/usr/bin/env python3
"""Throughput of the randomized Tikhonov solver on one GB300 (or N replicas).

Workload (default): ridge_over_262144x2048_f64 -- A = U diag(sigma) V^T with
m = 2^18, n = 2048 (4 GiB float64), sigma log-spaced 1..1e-8, b = A x + 1e-3
noise, N = 32 lambda log-spaced 1e-8..1, SRHT sketch s = 4n.  One step = one
full pass of the path for all 32 lambda (sketch, Gram, 32 Cholesky factors,
batched preconditioned LSQR; the mixed form adds the float64 refinement).

Timed: the batched mixed-precision solve (float32 LSQR + float64 refinement),
inputs resident in HBM.  Reported beside it, on the same inputs: the plain
float64 batched solve and the plain float64 one-lambda-at-a-time solve, and
the oracle's CPU cost on a bounded sample.

Prints one JSON line.  --impl reference times the CPU oracle instead.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "lambda-solves/s to 1e-10 rel. error (batched mixed vs plain FP64); A-stream HBM GB/s"
UNIT = "lambda-solves/s"
WORKLOAD = "ridge_over_262144x2048_f64"

# FP64 and FP32 SIMT peaks derived from unit counts and the maximum SM clock:
# 152 SMs x 2 DFMA/clk (FP64) or 128 FFMA/clk (FP32) x 2 flop x 2.07 GHz.
PEAK_FP64_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
PEAK_FP32_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12


# ncu dram__bytes_read.sum + dram__bytes_write.sum per launch of the kernel behind a phase, from a
# capture of the 65536 x 2048 float64 case (profiles/): (elements of A of that case, bytes).  A
# launch streams every element of A once, so the figure scales with m n; kernels changed since
# their capture are left out (traffic null).
MEASURED_TRAFFIC = {
    # profiles/k_oz_tc_lsqr_digits_65536x2048.md: k_oz_tc<4, 2, 32> and k_oz_tc<4, 1, 32> (32 lambda)
    "A_times_W_digits": (65536 * 2048, 1083622912 + 5114880),
    "At_times_U_digits": (65536 * 2048, 1091296512 + 1207296),
}

# How each phase is bounded: "hbm" phases are compared as algorithmic bytes / time with the
# measured copy bandwidth; "fp32" / "fp64" as algorithmic flops / time with the peaks above.
# The digit products read 8 bytes per element of A (4 BF16 digit planes); the emulated float64
# passes 16 (8 planes) and flush at most 8 float64 adds per output and 256 values of K.
PHASE_BOUND = {
    "A_times_W_digits": "hbm", "At_times_U_digits": "hbm", "lsqr_step_fused": "hbm", "refine_residual64": "hbm",
    "refine_normal64": "hbm", "slice_A": "hbm", "sketch": "hbm", "precond_apply": "hbm",
    "A_times_W": "fp32", "At_times_U": "fp32", "precond_inverse": "fp32",
    "cholesky": "fp64", "svd": "fp64",
    # emulated float64 products: compared as the BF16 tensor work they issue (36 digit pairs per
    # float64 multiply-add) with the measured BF16 peak
    "gram": "tensor", "cholesky_update": "tensor",
}
EMULATED_PAIRS = 36


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
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
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_env():
    from paper_2203_07329_gb300 import replicas
    return replicas.env()


# ------------------------------------------------------------ oracle arm ---
def oracle_iteration_sample(A_np, b_np, lam, iters, threads):
    """Seconds per LSQR iteration of the oracle on the full workload (one lambda).

    The preconditioned operator costs the same for any upper triangular R, so
    the sample uses R = sqrt(1 + lambda) I built on the CPU."""
    import oracle
    n = A_np.shape[1]
    R = np.eye(n) * math.sqrt(1.0 + lam)
    os.environ["OMP_NUM_THREADS"] = str(threads)
    t0 = time.perf_counter()
    oracle.lsqr_over_chol(A_np, b_np, lam, R, 1e-300, iters)
    return (time.perf_counter() - t0) / iters


def oracle_parallel_sample(A_np, b_np, lams, threads):
    """Seconds for one oracle LSQR iteration of `threads` lambdas at once, each on its own host
    thread (the lambda loop is independent, Section 2.1.1; the C oracle releases the GIL)."""
    from concurrent.futures import ThreadPoolExecutor
    import oracle
    n = A_np.shape[1]
    lam_t = [float(lams[i % len(lams)]) for i in range(threads)]
    Rs = [np.eye(n) * math.sqrt(1.0 + l) for l in lam_t]
    t0 = time.perf_counter()
    with ThreadPoolExecutor(max_workers=threads) as ex:
        list(ex.map(lambda k: oracle.lsqr_over_chol(A_np, b_np, lam_t[k], Rs[k], 1e-300, 1), range(threads)))
    return time.perf_counter() - t0


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def oracle_baseline(A_np, b_np, lams, ips, reps=2):
    """The oracle's lambda-solves/s on one host thread and on every core (lambda-parallel).  A lower
    bound on the oracle's time per lambda-solve: `ips` LSQR iterations, the sketch, Gram matrix and
    Cholesky factors excluded."""
    t1 = float(np.mean([oracle_iteration_sample(A_np, b_np, float(lams[0]), 1, 1) for _ in range(reps)]))
    cores = host_cores()
    tp = float(np.mean([oracle_parallel_sample(A_np, b_np, lams, cores) for _ in range(reps)]))
    return {"one_thread": 1.0 / (t1 * ips), "all_cores": cores / (tp * ips), "cores": cores,
            "s_per_iteration_one_thread": t1, "s_per_iteration_all_cores": tp}


def oracle_iters_per_solve():
    """The oracle's own LSQR iteration count at the smallest lambda on a reduced
    problem of the same family (SRHT s = 4n, sigma 1..1e-8, lambda 1e-8)."""
    import oracle
    from paper_2203_07329_gb300 import datagen
    p = datagen.make_ridge_problem(4096, 64, datagen.spectrum("log", 64, hi=1.0, lo=1e-8),
                                   datagen.log_lambdas(1, 1e-8, 1e-8), seed=5)
    _, it, _, _ = oracle.alg1(p.A.numpy(), p.b.numpy(), np.array([1e-8]), 0, 256, 1, 1e-14, 500)
    return int(it[0])


def run_reference(args):
    """--impl reference: the CPU oracle as it stands, bounded samples of the workload."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    import torch
    import oracle
    from paper_2203_07329_gb300 import datagen
    oracle.build()
    threads = host_cores()
    m, n = (args.m, args.n)
    prob, w = datagen.workload_problem(WORKLOAD, device="cpu", m=m, n=n)
    A_np = prob.A.numpy()
    b_np = prob.b.numpy()
    lams = prob.lambdas.numpy()
    ips = oracle_iters_per_solve()
    for _ in range(min(args.warmup, 1)):
        oracle_parallel_sample(A_np, b_np, lams, threads)
    times = [oracle_parallel_sample(A_np, b_np, lams, threads) for _ in range(args.steps)]
    t_iter = float(np.mean(times))  # one iteration of `threads` lambdas at once
    value = threads / (t_iter * ips)
    sample = (f"oracle LSQR iterations on the full {m}x{n} float64 A (plain C loops), {threads} lambdas at once "
              f"on {threads} host threads, {args.steps} timed; lambda-solve = {ips} iterations (the oracle's own "
              "count on the same family); a lower bound on the oracle's time: sketch, Gram and Cholesky excluded")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_iter * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "m": m, "n": n, "N": w["N"], "sketch": "srht", "s": w["s"]},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------- GPU arm ---
def small_workload_step(tk, datagen, stream, barrier, reps=20):
    """The 4096 x 256 float64 workload (8 lambda, Gaussian sketch s = 1024): it
    fits in L2, so the figure of merit is microseconds per lambda-solve."""
    import torch
    prob, w = datagen.workload_problem("ridge_over_4096x256_f64", device="cuda")
    lams = prob.lambdas.numpy()
    out = {}
    for key, prec in (("fp64", tk.TK_PREC_FP64), ("mixed", tk.TK_PREC_MIXED)):
        o = tk.opts_default(sketch=tk.TK_SKETCH_GAUSS, s=w["s"], seed=1, precision=prec)
        work = torch.empty(tk.workspace_size(tk.make_problem(prob.A, prob.b), len(lams), o), dtype=torch.uint8,
                           device="cuda")
        X = torch.empty((len(lams), prob.A.shape[1]), dtype=torch.float64, device="cuda")
        for _ in range(3):
            tk.tk_solve(prob.A, prob.b, lams, o, work=work, X=X, stream=stream)
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        l0 = tk.tk_launch_count()
        e0.record(stream)
        for _ in range(reps):
            r = tk.tk_solve(prob.A, prob.b, lams, o, work=work, X=X, stream=stream)
        e1.record(stream)
        barrier()
        t = e0.elapsed_time(e1) / reps
        launches = (tk.tk_launch_count() - l0) / reps
        tk.tk_profile_enable(True)  # one more call, profiled, for the phase split
        tk.tk_profile_collect()
        tk.tk_solve(prob.A, prob.b, lams, o, work=work, X=X, stream=stream)
        barrier()
        prof = tk.tk_profile_collect()
        tk.tk_profile_enable(False)
        out[key] = {"us_per_lambda_solve": t * 1e3 / len(lams), "ms_per_solve_call": t,
                    "launches_per_call": launches,
                    "iters_mean": float(np.mean([q["iters"] for q in r.info])),
                    "phase_ms": {k: round(v["ms"], 3) for k, v in prof.items() if v["launches"]},
                    "phase_launches": {k: v["launches"] for k, v in prof.items() if v["launches"]}}
    return out


def uneven_batch_step(tk, datagen, stream, barrier):
    """256 problems, m in [2000, 65536], n in [64, 1024], float32, 16 lambda each;
    odd problems have a small statistical dimension and take the low-rank
    preconditioner (sketch size 2 sd), the others the Cholesky one (s = 4n)."""
    import math
    import torch
    probs = datagen.uneven_batch(256, device="cuda", dtype=torch.float32)
    pairs, opts = [], []
    for p in probs:
        n = p.A.shape[1]
        lam_min = float(p.lambdas.min())
        if p.meta["lowrank"]:
            sd = float(np.sum(1.0 / (1.0 + lam_min / (p.sigma.numpy() ** 2))))
            opts.append(tk.opts_default(sketch=tk.TK_SKETCH_GAUSS, s=min(n, 2 * math.ceil(sd)), seed=1,
                                        precond=tk.TK_PRECOND_LOWRANK, alpha=2.0, precision=tk.TK_PREC_MIXED))
        else:
            opts.append(tk.opts_default(sketch=tk.TK_SKETCH_GAUSS, s=min(4 * n, p.A.shape[0]), seed=1,
                                        precision=tk.TK_PREC_MIXED))
        pairs.append((p.A, p.b))
    lams = np.stack([p.lambdas.numpy() for p in probs])
    need = tk.workspace_size_batched(pairs, lams.shape[1], opts)
    work = torch.empty(need, dtype=torch.uint8, device="cuda")
    tk.tk_solve_batched(pairs, lams, opts, work=work, stream=stream)  # warm-up
    barrier()
    tk.tk_profile_enable(True)
    tk.tk_profile_collect()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    _, infos, _ = tk.tk_solve_batched(pairs, lams, opts, work=work, stream=stream)
    e1.record(stream)
    barrier()
    prof = tk.tk_profile_collect()
    tk.tk_profile_enable(False)
    t = e0.elapsed_time(e1)
    solves = int(lams.size)
    a_bytes = sum(A.numel() * A.element_size() for A, _ in pairs)
    keys = ("A_times_W", "At_times_U", "refine_residual64", "refine_normal64")
    stream_ms = sum(prof[k]["ms"] for k in keys)
    stream_bytes = sum(prof[k]["bytes"] for k in keys)
    stream_impl = sum(prof[k]["impl_bytes"] for k in keys)
    return {"value": solves / (t / 1e3), "unit": "lambda-solves/s", "ms_per_step": t, "problems": len(pairs),
            "lambda_solves": solves, "a_bytes": a_bytes,
            "a_stream_gbs_summed_phases": stream_bytes / (stream_ms / 1e3) / 1e9 if stream_ms > 0 else None,
            "a_stream_impl_gbs_summed_phases": stream_impl / (stream_ms / 1e3) / 1e9 if stream_ms > 0 else None,
            "note": "phase times are summed over the concurrent host lanes of the build; the grouped LSQR and "
                    "refinement run on one stream",
            "iters_mean": float(np.mean([q["iters"] for inf in infos for q in inf])),
            "phase_ms_summed_over_lanes": {k: v["ms"] for k, v in prof.items() if v["launches"]}}


def roofline_of(prof, peaks, peak_src, a_elems, fp64=False):
    """Roofline line of the phase with the largest event time in `prof` (tk_profile_collect totals over
    the timed region), judged by that phase's bound; traffic scaled from an ncu capture when one exists.
    fp64: the plain float64 form, whose products and inverse run on the float64 pipe."""
    dom = max(prof.items(), key=lambda kv: kv[1]["ms"])
    name, st = dom
    bound = PHASE_BOUND.get(name, "fp32")
    if fp64 and name in ("A_times_W", "At_times_U", "precond_inverse"):
        bound = "fp64"
    per_launch_ms = st["ms"] / max(st["launches"], 1)
    secs = st["ms"] / 1e3
    if bound == "hbm":
        achieved = st["bytes"] / secs / 1e9 if secs > 0 else 0.0
        peak, unit = float(peaks["hbm_gbs"]), "GB/s"
        psrc = f"{peak_src}: MEASURED_PEAKS.json hbm_gbs (copy bandwidth)"
    elif bound == "tensor":
        achieved = EMULATED_PAIRS * st["flops"] / secs / 1e12 if secs > 0 else 0.0
        peak, unit = float(peaks["bf16_tflops_sustained"]), "TFLOP/s"
        psrc = f"{peak_src}: MEASURED_PEAKS.json bf16_tflops_sustained"
    else:
        achieved = st["flops"] / secs / 1e12 if secs > 0 else 0.0
        peak, unit = (PEAK_FP64_TFLOPS if bound == "fp64" else PEAK_FP32_TFLOPS), "TFLOP/s"
        psrc = "derived from unit counts and max clock (FP64 2 DFMA/clk/SM, FP32 128 FFMA/clk/SM)"
    # DRAM bytes (read + write) of one launch from an ncu capture of the same kernel on a smaller
    # case (profiles/), scaled by the elements of A it streams; None for kernels not captured
    traffic = None
    if name in MEASURED_TRAFFIC:
        case_elems, case_bytes = MEASURED_TRAFFIC[name]
        traffic = case_bytes * a_elems / case_elems
    roofline = {"bound": bound if bound in ("hbm", "tensor") else "alu", "kernel": name, "achieved": achieved,
                "peak": peak, "unit": unit, "frac": achieved / peak if peak else None, "traffic": traffic,
                "algorithmic_bytes_per_launch": st["bytes"] / max(st["launches"], 1),
                "impl_bytes_per_launch": st["impl_bytes"] / max(st["launches"], 1),
                "per_launch_ms": per_launch_ms, "launches": st["launches"], "peak_source": psrc}
    if bound == "hbm" and secs > 0:
        # what the kernel physically moves (digit planes, copies) beside the method's own bytes
        roofline["impl_achieved"] = st["impl_bytes"] / secs / 1e9
        roofline["impl_frac"] = roofline["impl_achieved"] / peak
    return roofline


STREAM_PHASES = ("A_times_W", "At_times_U", "A_times_W_digits", "At_times_U_digits", "lsqr_step_fused",
                 "refine_residual64", "refine_normal64")


def a_stream_of(prof):
    """(method GB/s, implementation GB/s) over the phases that stream A (LSQR products, refinement passes)."""
    ms = sum(prof[k]["ms"] for k in STREAM_PHASES if k in prof)
    if ms <= 0:
        return None, None
    by = sum(prof[k]["bytes"] for k in STREAM_PHASES if k in prof)
    ib = sum(prof[k]["impl_bytes"] for k in STREAM_PHASES if k in prof)
    return by / (ms / 1e3) / 1e9, ib / (ms / 1e3) / 1e9


def phase_table(prof, steps):
    return {k: {"ms_per_step": v["ms"] / steps, "launches_per_step": v["launches"] / steps,
                "tflops": (v["flops"] / (v["ms"] / 1e3) / 1e12) if v["ms"] > 0 else 0.0,
                "gbs": (v["bytes"] / (v["ms"] / 1e3) / 1e9) if v["ms"] > 0 else 0.0,
                "impl_gbs": (v["impl_bytes"] / (v["ms"] / 1e3) / 1e9) if v["ms"] > 0 else 0.0}
            for k, v in prof.items() if v["launches"]}


def workload_leg(tk, datagen, stream, barrier, name, make_opts, steps, warmup, peaks, peak_src, fp64=False):
    """One of the other full-size workloads, timed like the headline: inputs resident in HBM (larger than
    L2), `warmup` untimed solves, `steps` timed solves with live phase events."""
    import torch
    t_gen = time.perf_counter()
    prob, w = datagen.workload_problem(name, device="cuda")
    t_gen = time.perf_counter() - t_gen
    A, b = prob.A, prob.b
    lams = prob.lambdas.numpy()
    N = len(lams)
    o = make_opts(w)
    work = torch.empty(tk.workspace_size(tk.make_problem(A, b), N, o), dtype=torch.uint8, device="cuda")
    X = torch.empty((N, A.shape[1]), dtype=torch.float64, device="cuda")
    for _ in range(warmup):
        tk.tk_solve(A, b, lams, o, work=work, X=X, stream=stream)
    barrier()
    tk.tk_profile_enable(True)
    tk.tk_profile_collect()
    l0 = tk.tk_launch_count()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        r = tk.tk_solve(A, b, lams, o, work=work, X=X, stream=stream)
    e1.record(stream)
    barrier()
    prof = tk.tk_profile_collect()
    tk.tk_profile_enable(False)
    ms = e0.elapsed_time(e1) / steps
    gbs, igbs = a_stream_of(prof)
    out = {"value": N / (ms / 1e3), "unit": UNIT, "ms_per_step": ms, "steps": steps, "warmup": warmup,
           "m": int(A.shape[0]), "n": int(A.shape[1]), "N": N, "dtype": str(A.dtype).replace("torch.", ""),
           "a_bytes": int(A.numel() * A.element_size()), "workspace_bytes": int(work.numel()),
           "a_stream_gbs": gbs, "a_stream_impl_gbs": igbs,
           "roofline": roofline_of(prof, peaks, peak_src, A.shape[0] * A.shape[1], fp64=fp64),
           "phases": phase_table(prof, steps), "gpu_launches_per_step": (tk.tk_launch_count() - l0) / steps,
           "iters_mean": float(np.mean([q["iters"] for q in r.info])),
           "iters_max": int(max(q["iters"] for q in r.info)),
           "refine_steps_max": int(max(q["refine_steps"] for q in r.info)),
           "status_ok": all(q["status"] == 0 for q in r.info), "generate_s": round(t_gen, 1)}
    del work, X, A, b, prob
    torch.cuda.empty_cache()
    return out


def bp2_vs_cholesky(tk, datagen, stream, barrier):
    """Fig. 2 of the paper on this GPU: the same 15 lambda solved with the Cholesky preconditioner of
    Algorithm 1 and with BP2 (a QR of [XA; sqrt(l) I] per lambda), SRDCT sketch, float64, for sketch
    sizes s = 2n .. 20n; A 65536 x 512 with sigma log-spaced 1e5 .. 1e-5 (the figure's spectrum, the
    rows scaled down from 5e5)."""
    import torch
    m, n = 65536, 512
    sig = datagen.spectrum("log", n, hi=1e5, lo=1e-5)
    p = datagen.make_ridge_problem(m, n, sig, datagen.log_lambdas(15, 1e-6, 1e2), seed=20220321, device="cuda")
    lams = p.lambdas.numpy()
    out = {}
    for over in (2, 5, 10, 20):
        row = {}
        for name, pc in (("cholesky", tk.TK_PRECOND_CHOL), ("bp2_qr", tk.TK_PRECOND_QR)):
            o = tk.opts_default(sketch=tk.TK_SKETCH_SRDCT, s=over * n, seed=1, precond=pc)
            work = torch.empty(tk.workspace_size(tk.make_problem(p.A, p.b), len(lams), o), dtype=torch.uint8,
                               device="cuda")
            tk.tk_solve(p.A, p.b, lams, o, work=work, stream=stream)  # warm-up
            barrier()
            tk.tk_profile_enable(True)
            tk.tk_profile_collect()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            r = tk.tk_solve(p.A, p.b, lams, o, work=work, stream=stream)
            e1.record(stream)
            barrier()
            prof = tk.tk_profile_collect()
            tk.tk_profile_enable(False)
            row[name] = {"ms_15_lambda": e0.elapsed_time(e1), "factor_ms": prof["cholesky"]["ms"],
                         "gram_ms": prof["gram"]["ms"], "iters_mean": float(np.mean([q["iters"] for q in r.info])),
                         "status_ok": all(q["status"] == 0 for q in r.info)}
            del work
        out[f"s={over}n"] = row
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="tikhonov", choices=["tikhonov", "reference"])
    ap.add_argument("--m", type=int, default=262144)
    ap.add_argument("--n", type=int, default=2048)
    ap.add_argument("--no-fp64", action="store_true", help="skip the plain float64 comparison solves")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle sample")
    ap.add_argument("--no-tc", action="store_true", help="skip the tensor-core LSQR comparison step")
    ap.add_argument("--no-uneven", action="store_true", help="skip the 256 uneven problems batch")
    ap.add_argument("--no-small", action="store_true", help="skip the 4096 x 256 workload")
    ap.add_argument("--no-c3", action="store_true", help="skip the 2048 x 2^18 underdetermined workload")
    ap.add_argument("--no-lcurve", action="store_true", help="skip the L-curve sweep on the headline workload")
    ap.add_argument("--no-bp2", action="store_true", help="skip the BP2-versus-Cholesky comparison (Fig. 2)")
    ap.add_argument("--sketch", default="srht", choices=["srht", "gauss", "sparse", "srdct"],
                    help="embedding of the headline solve (the workload's own is the SRHT)")
    ap.add_argument("--no-c4", action="store_true", help="skip the 2^20 x 4096 float32 precision-form workload")
    ap.add_argument("--no-tune", action="store_true", help="keep the fixed tile rules (no tk_autotune)")
    ap.add_argument("--lsqr-tc", type=int, default=None, choices=[0, 1, 2, 3],
                    help="LSQR products of the timed mixed step: 0 SIMT float32, 1 TF32 x3, 2 4-digit slices "
                         "(default: the library's)")
    ap.add_argument("--gen-device", default="cuda", choices=["cuda", "cpu"],
                    help="where the synthetic problem is generated (cpu for profiler runs)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import torch.distributed as dist
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    from paper_2203_07329_gb300 import replicas
    dev = torch.device("cuda", local)

    def barrier():
        replicas.barrier(dev)

    from paper_2203_07329_gb300 import build, datagen
    build.build()
    from paper_2203_07329_gb300 import tikhonov as tk

    m, n = args.m, args.n
    prob, w = datagen.workload_problem(WORKLOAD, device=args.gen_device, m=m, n=n)
    A, b = prob.A.cuda(), prob.b.cuda()
    del prob.A
    lams = prob.lambdas.numpy()
    N = len(lams)
    s = w["s"]
    extra_opts = {} if args.lsqr_tc is None else {"lsqr_tc": args.lsqr_tc}
    sk = {"srht": tk.TK_SKETCH_SRHT, "gauss": tk.TK_SKETCH_GAUSS, "sparse": tk.TK_SKETCH_SPARSE,
          "srdct": tk.TK_SKETCH_SRDCT}[args.sketch]
    if args.sketch == "sparse":
        s = 4 * s  # the sparse embedding needs more rows for the same distortion (Theorem 3.5)
    o_mixed = tk.opts_default(sketch=sk, s=s, seed=1, precision=tk.TK_PREC_MIXED, **extra_opts)
    o_fp64 = tk.opts_default(sketch=sk, s=s, seed=1, tol=1e-14)
    o_fp64_one = tk.opts_default(sketch=sk, s=s, seed=1, tol=1e-14,
                                 schedule=tk.TK_SCHED_ONE_AT_A_TIME)
    stream = torch.cuda.current_stream()
    work = torch.empty(max(tk.workspace_size(tk.make_problem(A, b), N, o) for o in (o_mixed, o_fp64, o_fp64_one)),
                       dtype=torch.uint8, device="cuda")
    X = torch.empty((N, n), dtype=torch.float64, device="cuda")

    def step(o, Xo=X):
        return tk.tk_solve(A, b, lams, o, work=work, X=Xo, stream=stream)

    # measured tile shapes / split counts for this workload's products (outside the timed region)
    t_tune = time.perf_counter()
    tuned = 0
    if not args.no_tune:
        for o in (o_mixed, o_fp64):
            tuned = tk.tk_autotune(A, b, N, o, work=work, stream=stream)
    t_tune = time.perf_counter() - t_tune

    for _ in range(args.warmup):
        res = step(o_mixed)
    barrier()
    # ---- timed region: K batched mixed steps, inputs resident in HBM
    clocks = ClockSampler(local)
    clocks.start()
    tk.tk_profile_enable(True)
    tk.tk_profile_collect()
    launches0 = tk.tk_launch_count()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    ev0.record(stream)
    for _ in range(args.steps):
        res = step(o_mixed)
    ev1.record(stream)
    barrier()
    launches = tk.tk_launch_count() - launches0
    prof = tk.tk_profile_collect()
    tk.tk_profile_enable(False)
    clk = clocks.stop()
    ms = replicas.max_over_ranks(ev0.elapsed_time(ev1) / args.steps, dev)
    value = replicas.job_throughput(N, ms, ws)
    X_mixed = X.clone()
    info_mixed = res.info

    # ---- e2e: the same call with host buffers, copies inside the timed region
    A_host = A.cpu().pin_memory()
    b_host = b.cpu().pin_memory()
    X_host = torch.empty((N, n), dtype=torch.float64).pin_memory()
    A_dev = torch.empty_like(A)
    b_dev = torch.empty_like(b)

    def e2e_step():
        A_dev.copy_(A_host, non_blocking=True)
        b_dev.copy_(b_host, non_blocking=True)
        tk.tk_solve(A_dev, b_dev, lams, o_mixed, work=work, X=X, stream=stream)
        X_host.copy_(X, non_blocking=True)

    for _ in range(max(1, args.warmup)):  # untimed, like the device-resident steps (first use of the pinned pages)
        e2e_step()
    barrier()
    t0 = time.perf_counter()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        e2e_step()
    e1.record(stream)
    barrier()
    e2e_ms = replicas.max_over_ranks(e0.elapsed_time(e1) / args.steps, dev)
    del A_dev, A_host

    # ---- the mixed solve with the LSQR products on the tensor cores (one step)
    extra = {}
    if not args.no_tc:
        o_tc = tk.opts_default(sketch=tk.TK_SKETCH_SRHT, s=s, seed=1, precision=tk.TK_PREC_MIXED, lsqr_tc=1)
        need = tk.workspace_size(tk.make_problem(A, b), N, o_tc)
        work_tc = work if work.numel() >= need else torch.empty(need, dtype=torch.uint8, device="cuda")
        Xtc = torch.empty((N, n), dtype=torch.float64, device="cuda")
        tk.tk_solve(A, b, lams, o_tc, work=work_tc, X=Xtc, stream=stream)  # warm-up
        barrier()
        tk.tk_profile_enable(True)
        tk.tk_profile_collect()
        c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        c0.record(stream)
        rtc = tk.tk_solve(A, b, lams, o_tc, work=work_tc, X=Xtc, stream=stream)
        c1.record(stream)
        barrier()
        prof_tc = tk.tk_profile_collect()
        tk.tk_profile_enable(False)
        ttc = c0.elapsed_time(c1)
        dtc = (Xtc - X_mixed).norm(dim=1) / X_mixed.norm(dim=1)
        extra["mixed_tensor_core_lsqr"] = {
            "value": N / (ttc / 1e3), "ms_per_step": ttc,
            "iters_mean": float(np.mean([q["iters"] for q in rtc.info])),
            "refine_steps_max": int(max(q["refine_steps"] for q in rtc.info)),
            "max_rel_diff_vs_simt_mixed": float(dtc.max()),
            "phases": {k: {"ms": v["ms"], "launches": v["launches"],
                           "gbs": (v["bytes"] / (v["ms"] / 1e3) / 1e9) if v["ms"] > 0 else 0.0}
                       for k, v in prof_tc.items() if v["launches"]}}
        del work_tc, Xtc

    # ---- plain float64 comparisons on the same inputs (one step each)
    if not args.no_fp64:
        X64 = torch.empty((N, n), dtype=torch.float64, device="cuda")
        step(o_fp64, X64)  # warm-up of the float64 kernels (shared by both schedules)
        for key, o, reps in (("fp64_batched", o_fp64, 2), ("fp64_one_at_a_time", o_fp64_one, 1)):
            barrier()
            a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a0.record(stream)
            for _ in range(reps):
                r64 = step(o, X64)
            a1.record(stream)
            barrier()
            t64 = a0.elapsed_time(a1) / reps
            extra[key] = {"value": N / (t64 / 1e3), "ms_per_step": t64, "timed_steps_after_warmup": reps,
                          "iters_mean": float(np.mean([q["iters"] for q in r64.info]))}
            if key == "fp64_batched":
                d = (X_mixed - X64).norm(dim=1) / X64.norm(dim=1)
                extra["max_rel_diff_mixed_vs_fp64"] = float(d.max())
        extra["speedup_mixed_vs_fp64_one_at_a_time"] = value / ws / extra["fp64_one_at_a_time"]["value"]
        extra["speedup_mixed_vs_fp64_batched"] = value / ws / extra["fp64_batched"]["value"]

    # ---- the small 4096 x 256 workload (fits in L2: launch/latency-bound)
    if not args.no_small:
        extra["small_4096x256_f64"] = small_workload_step(tk, datagen, stream, barrier)

    # ---- many independent problems of uneven size in one batched call (one step)
    if not args.no_uneven:
        extra["uneven_256_mixed"] = uneven_batch_step(tk, datagen, stream, barrier)

    # ---- roofline of the dominant phase (live events over the timed region)
    peaks, peak_src = load_peaks()
    roofline = roofline_of(prof, peaks, peak_src, m * n)
    a_stream_gbs, a_stream_impl_gbs = a_stream_of(prof)
    phases = phase_table(prof, args.steps)

    # ---- CPU oracle sample (rank 0 only, N = 1 only)
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu:
        try:
            import oracle
            oracle.build()
            A_np = A.cpu().numpy()
            b_np = b.cpu().numpy()
            ips = oracle_iters_per_solve()
            ob = oracle_baseline(A_np, b_np, lams, ips)
            cpu = {"value": ob["all_cores"], "unit": UNIT, "cores": ob["cores"], "kind": "oracle",
                   "one_thread_value": ob["one_thread"],
                   "sample": f"oracle LSQR iterations on the full {m}x{n} float64 A (plain C loops): 2 timed "
                             f"iterations of one lambda on 1 thread, and 2 of {ob['cores']} lambdas at once on "
                             f"{ob['cores']} host threads; lambda-solve = {ips} iterations (the oracle's own count "
                             "on the same family); a lower bound on the oracle's time per lambda-solve: sketch, "
                             "Gram and Cholesky excluded"}
        except Exception as ex:  # the baseline is reported, never the target
            cpu = {"value": None, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": f"failed: {ex}"}

    # ---- the L-curve of Section 4.3 on the headline's A: 32 lambda in 1e-10..1, then 16 between the
    #      corner's neighbours with the sketch, Gram matrix and digit planes reused (one call)
    if not args.no_lcurve:
        lam_lc = np.logspace(-10, 0, 32)
        need = tk.lcurve_workspace_size(A, b, 32, 16, o_mixed)
        work_lc = torch.empty(need, dtype=torch.uint8, device="cuda")
        tk.tk_lcurve(A, b, lam_lc, 16, o_mixed, work=work_lc, stream=stream)  # warm-up
        barrier()
        tk.tk_profile_enable(True)
        tk.tk_profile_collect()
        c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        c0.record(stream)
        _, pts_lc, k_lc = tk.tk_lcurve(A, b, lam_lc, 16, o_mixed, work=work_lc, stream=stream)
        c1.record(stream)
        barrier()
        prof_lc = tk.tk_profile_collect()
        tk.tk_profile_enable(False)
        t_lc = c0.elapsed_time(c1)
        extra["lcurve_262144x2048_mixed"] = {
            "value": len(pts_lc) / (t_lc / 1e3), "unit": UNIT, "ms_per_call": t_lc,
            "lambdas": len(pts_lc), "sweeps": "32 log-spaced in 1e-10..1, then 16 between the corner's neighbours",
            "corner_lambda": pts_lc[k_lc]["lam"], "corner_curvature": pts_lc[k_lc]["curvature"],
            "status_ok": all(q["status"] == 0 for q in pts_lc),
            "phase_ms": {k2: round(v["ms"], 3) for k2, v in prof_lc.items() if v["launches"]}}
        del work_lc

    # ---- the other full-size workloads (the headline's buffers freed first)
    h2d_bytes = int(A.numel() * A.element_size() + b.numel() * 8)
    del work, X, A, b
    torch.cuda.empty_cache()
    if not args.no_c4:
        extra["precision_form_1048576x4096_f32"] = workload_leg(
            tk, datagen, stream, barrier, "ridge_over_1048576x4096_f32",
            lambda w: tk.opts_default(sketch=tk.TK_SKETCH_GAUSS, s=w["s"], seed=1, precision=tk.TK_PREC_MIXED),
            steps=2, warmup=1, peaks=peaks, peak_src=peak_src)
    if not args.no_bp2:
        extra["bp2_vs_cholesky_65536x512_srdct"] = bp2_vs_cholesky(tk, datagen, stream, barrier)
    if not args.no_c3:
        extra["under_2048x262144_f64"] = workload_leg(
            tk, datagen, stream, barrier, "ridge_under_2048x262144_f64",
            lambda w: tk.opts_default(sketch=tk.TK_SKETCH_SRHT, s=w["s"], seed=1, tol=1e-14),
            steps=2, warmup=1, peaks=peaks, peak_src=peak_src, fp64=True)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
                "config": {"workload": WORKLOAD, "m": m, "n": n, "N": N, "sketch": args.sketch, "s": s,
                           "precision": "mixed (float32 LSQR, float64 refinement, Gram and Cholesky)",
                           "schedule": "batched", "l2": "inputs larger than L2 (A is 4 GiB)",
                           "parallelism": f"{ws} independent replicas" if ws > 1 else "1 GPU"},
                "roofline": roofline, "a_stream_gbs": a_stream_gbs, "a_stream_impl_gbs": a_stream_impl_gbs,
                "phases": phases,
                "cpu_baseline": cpu,
                "e2e": {"value": ws * N / (e2e_ms / 1e3), "unit": UNIT,
                        "h2d_bytes_per_step": h2d_bytes,
                        "d2h_bytes_per_step": int(N * n * 8)},
                "gpu_launches": int(launches), "clocks": clk,
                "iters_mean": float(np.mean([q["iters"] for q in info_mixed])),
                "refine_steps_max": int(max(q["refine_steps"] for q in info_mixed)),
                "autotune": {"entries": tuned, "seconds": round(t_tune, 2)},
                "peaks_source": peak_src}
        line.update(extra)
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
