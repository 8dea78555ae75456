#!/usr/bin/env python3
"""Benchmark of the GB300 PPCG eigensolver: time-to-tolerance (max residual 1e-8) and PPCG iterations/s.

One step = one complete ppcg_solve (Algorithm 3: orthonormalisation, Rayleigh-Ritz steps, preconditioned
projected search directions, sub-block Rayleigh-Ritz, CholeskyQR2, locking) from the seeded starting block to
max residual 1e-8, on the 32^3-grid / k = 256 / sbsize = 4 / 8-well workload with V and X0 resident in HBM.

Prints one JSON line. Also reported:
  roofline      the dominant kernel (FP64 Gram X^T W, the FP64 pipe is the bound) timed live with CUDA events
  e2e           the same metric through the C ABI with host (pinned) buffers: V and X0 copied in and X,
                lambda, residuals copied out inside the timed region
  cpu_baseline  the CPU oracle (numpy/LAPACK Algorithm 3) on a bounded sample of the same workload
  clocks        nvidia-smi samples taken during the timed region
--impl reference times the CPU oracle alone (the reference arm of this method: there is no other code).
"""
from __future__ import annotations

import argparse
import ctypes
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

import workloads as wl  # noqa: E402

METRIC = "time-to-tol 1e-8 and PPCG iters/s, mixed vs FP64 form on 1 GB300; % roofline"
# FP64 FMA pipe of GB300: 2 FMA lanes per SM per clock (measured: a DFMA stream reaches 1.195 TFLOP/s at 1.97 GHz)
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12          # 1.2586, at the 2070 MHz maximum SM clock
# dram bytes (read + write) per launch of the roofline kernel, from one ncu capture of this shape
# (134.66 MB read + 9.42 MB written)
ROOFLINE_TRAFFIC_BYTES = 144.08e6
# DRAM bytes (read + write) of one tc_gram_kernel<256,2> launch, 32768 x 256 x 256, from one ncu capture
# (134.27 MB read + 3.62 MB written: the FP32 split-K partials stay mostly in L2)
TF32_GRAM_TRAFFIC_BYTES = 137.89e6
L2_BYTES = 129 * 2 ** 20
WORKLOADS = {"grid32_k256": wl.GRID32_K256, "grid16_k64": wl.GRID16_K64, "grid48_k1024": wl.GRID48_K1024,
             "grid32_k128_bloch": wl.GRID32_K128_BLOCH}


def _env_rank():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("LOCAL_RANK",
                                                                                                         "0"))


def max_over_ranks(value, dist, device):
    """The job's time is the slowest replica's: all-reduce MAX over the ranks (identity without a process group)."""
    if dist is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


class ClockSampler:
    """nvidia-smi clock/throttle samples every 200 ms while active."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index=0):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def _oracle_threads():
    try:
        import threadpoolctl
        info = threadpoolctl.threadpool_info()
        return max([i.get("num_threads", 0) for i in info if i.get("user_api") == "blas"] or [0]) or None
    except Exception:
        return None


def cpu_oracle_sample(w, iters):
    """Time the CPU oracle on a bounded sample: orth + initial Rayleigh-Ritz + `iters` iterations."""
    import oracle
    V, X0 = wl.make_inputs(w)
    t0 = time.perf_counter()
    r = oracle.ppcg(V, w.N, w.h, w.k, w.sbsize, w.rr_period, X0, tol=w.tol, maxiter=iters,
                    theta=w.theta if w.dtype == "c128" else None)
    el = time.perf_counter() - t0
    return el, r


def oracle_full_iters():
    """Iterations the oracle needed on the benchmark workload (stored by tests/golden/make_golden.py)."""
    path = os.path.join(ROOT, "tests", "golden", "grid32_k256_oracle_eigs.txt")
    if not os.path.exists(path):
        return None, None
    head = open(path).readline() + open(path).readlines()[1]
    lam = np.loadtxt(path)[:, 0]
    for tok in head.split():
        if tok.startswith("iters="):
            return int(tok.split("=")[1]), lam
    return None, lam


def cpu_baseline(w, sample_iters, gpu_iters, stored=True):
    el, r = cpu_oracle_sample(w, sample_iters)
    full_iters, _ = oracle_full_iters() if stored else (None, None)
    iters_target = full_iters or gpu_iters
    per_iter = el / max(1, r.iters)
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    return {"value": per_iter * iters_target, "unit": "s", "cores": _oracle_threads() or cores, "kind": "oracle",
            "sample": (f"oracle Algorithm 3 (numpy/LAPACK FP64) on {w.name}: orth + initial Rayleigh-Ritz + "
                       f"{r.iters} iterations took {el:.2f} s; time-to-tol extrapolated as {per_iter:.3f} s/iter x "
                       f"{iters_target} iterations ({'oracle full run' if full_iters else 'GPU iteration count'})"),
            "iters_per_s": 1.0 / per_iter, "host_cores": cores}


def run_reference(args, w):
    rank, world, _ = _env_rank()
    if rank != 0:
        return 0
    for _ in range(args.warmup):
        cpu_oracle_sample(w, args.ref_iters)
    times, iters = [], 0
    for _ in range(args.steps):
        el, r = cpu_oracle_sample(w, args.ref_iters)
        times.append(el)
        iters += r.iters
    full_iters, _ = oracle_full_iters()
    per_iter = sum(times) / max(1, iters)
    value = per_iter * (full_iters or 1000)
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times), "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w.name, "n": w.n, "k": w.k, "sbsize": w.sbsize, "rr_period": w.rr_period,
                       "tol": w.tol, "form": "fp64"},
            "iters_per_s": 1.0 / per_iter,
            "cpu_baseline": {"value": value, "unit": "s", "cores": _oracle_threads() or cores, "kind": "oracle",
                             "sample": f"each step: orth + initial Rayleigh-Ritz + {args.ref_iters} iterations of the "
                                       f"oracle; time-to-tol extrapolated x {full_iters or 1000} iterations"},
            "e2e": {"value": value, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# form name -> (precision, how the FP64 n x k GEMMs run, step-18 orthonormalisation)
FORMS = {
    "fp64": ("fp64", "fma", "cholqr2"),
    "mixed": ("mixed_tf32", "fma", "cholqr2"),
    "fp64_ozaki": ("fp64", "ozaki", "cholqr2"),
    "mixed_ozaki": ("mixed_tf32", "ozaki", "cholqr2"),
    "fp64_ozaki_polar": ("fp64", "ozaki", "polar"),
    "mixed_ozaki_polar": ("mixed_tf32", "ozaki", "polar"),
}
FORM_TEXT = {
    "fp64": "FP64 throughout (FP64 FMA pipe GEMMs), CholeskyQR2",
    "mixed": "TF32 tcgen05 projection GEMMs and first CholeskyQR Gram; everything else FP64",
    "fp64_ozaki": "FP64 with the n x k GEMMs emulated on BF16 tcgen05 (8 digit slices, Ozaki)",
    "mixed_ozaki": "mixed (TF32 projections) with the other FP64 n x k GEMMs emulated on BF16 tcgen05 (Ozaki)",
    "fp64_ozaki_polar": "fp64_ozaki with the polar-series orthonormalisation of Section 5.5",
    "mixed_ozaki_polar": "mixed_ozaki with the polar-series orthonormalisation of Section 5.5",
}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="grid32_k256", choices=list(WORKLOADS) + ["batch64"],
                    help="grid32_k256 (default), grid16_k64, grid48_k1024 (mixed-form size), "
                         "grid32_k128_bloch (the complex Bloch recipe), batch64 (64 uneven problems)")
    ap.add_argument("--maxiter", type=int, default=6000)
    ap.add_argument("--ref-iters", type=int, default=3, help="oracle iterations per reference-arm step")
    ap.add_argument("--cpu-iters", type=int, default=3, help="oracle iterations in the cpu_baseline sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--forms", default="fp64,mixed,fp64_ozaki,mixed_ozaki,mixed_ozaki_polar",
                    help="forms to time; the first is the headline value (" + ", ".join(FORMS) + ")")
    ap.add_argument("--batch-concurrency", type=int, default=16, help="concurrent solves of the batched workload")
    ap.add_argument("--batch-gemm", default="fma", choices=["fma", "ozaki"],
                    help="FP64 GEMMs of the batched workload: FP64 FMA pipe or Ozaki emulation on tcgen05")
    args = ap.parse_args()
    if args.workload == "batch64":
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "the batched workload has no oracle arm: 64 CPU "
                              "solves do not fit a bounded sample"}), flush=True)
            return 0
        return run_batched(args)
    w = WORKLOADS[args.workload]
    if args.impl == "reference":
        return run_reference(args, w)

    import torch
    import paper_1407_7506_gb300 as pk
    from paper_1407_7506_gb300 import build as _build

    rank, world, local = _env_rank()
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    if rank == 0:
        _build.build()
    if dist:
        dist.barrier()
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    V, X0 = wl.make_inputs(w)
    V_d = torch.from_numpy(V).to(dev)
    X0_d = torch.from_numpy(np.ascontiguousarray(X0.T)).to(dev)         # (k, n) rows = columns of X0
    _, gold = oracle_full_iters() if args.workload == "grid32_k256" else (None, None)
    cplx = w.dtype == "c128"
    sk = {"dtype": w.dtype, "theta": w.theta} if cplx else {}          # Solver arguments of the operator

    def run_form(precision, clk_sampler, fp64_gemm="fma", orth="cholqr2"):
        solver = pk.Solver(V_d, w.N, w.k, w.sbsize, rr_period=w.rr_period, maxiter=args.maxiter, device=dev,
                           stream=stream, precision=precision, fp64_gemm=fp64_gemm, orth=orth, **sk)
        X_out = torch.empty((w.k, w.n), dtype=solver.dtype, device=dev)
        for _ in range(args.warmup):
            solver.solve(X0_d, w.tol, out=X_out)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        iters, launches, stats = 0, 0, []
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        with clk_sampler:
            ev0.record(stream)
            t0 = time.perf_counter()
            for _ in range(args.steps):
                lam, _, res, st = solver.solve(X0_d, w.tol, out=X_out)
                iters += st["iters"]
                launches += st["kernel_launches"]
                stats.append(st)
            ev1.record(stream)
            torch.cuda.synchronize()
            wall = time.perf_counter() - t0
        if dist:
            dist.barrier()
        ms = max_over_ranks(ev0.elapsed_time(ev1), dist, dev)
        parity = {"max_residual": float(np.max(res)), "converged": all(s_["converged"] == 1 for s_ in stats)}
        if gold is not None:
            parity["max_rel_err_vs_oracle"] = float(np.max(np.abs(lam - gold) / np.maximum(np.abs(gold), 1.0)))
        solver.close()
        # one more solve with per-phase timers (the paper's profile categories), outside the timed region
        ps = pk.Solver(V_d, w.N, w.k, w.sbsize, rr_period=w.rr_period, maxiter=args.maxiter, device=dev,
                       stream=stream, timing=True, precision=precision, fp64_gemm=fp64_gemm, orth=orth, **sk)
        _, _, _, pst = ps.solve(X0_d, w.tol)
        ps.close()
        return {"ms_per_step": ms / args.steps, "iters": iters // args.steps, "iters_per_s": iters / (ms / 1e3),
                "wall_s_per_step": wall / args.steps, "launches": launches, "parity": parity,
                "phase_ms": {k_: round(v_, 2) for k_, v_ in pst["t_phase_ms"].items()},
                "jacobi_sweeps_max": pst["jacobi_sweeps_max"],
                "counts": {k_: stats[-1][k_] for k_ in ("n_rr", "n_drop_p", "n_cholqr_fallback", "n_polar",
                                                         "n_orth_skip", "n_eig_diagonal", "n_eig_refined")}}

    forms = [f.strip() for f in args.forms.split(",") if f.strip()]
    clk = ClockSampler(local)
    first = forms[0]
    results = {}
    for f in forms:
        prec, gm, orth = FORMS[f]
        results[f] = run_form(prec, clk if f == first else ClockSampler(local), fp64_gemm=gm, orth=orth)
    fp64 = results[first]
    ms_per_step = fp64["ms_per_step"]
    iters = fp64["iters"] * args.steps
    launches = fp64["launches"]
    parity = fp64["parity"]
    phases = fp64["phase_ms"]
    probe = pk.Solver(V_d, w.N, w.k, w.sbsize, rr_period=w.rr_period, maxiter=1, device=dev, stream=stream, **sk)
    roof = roofline(pk, probe, w, dev, stream)
    roof_stencil = roofline_stencil(pk, probe, w, dev, stream)
    probe.close()
    roof_mixed = None
    if any(FORMS[f][0] == "mixed_tf32" for f in results):
        probe = pk.Solver(V_d, w.N, w.k, w.sbsize, rr_period=w.rr_period, maxiter=1, device=dev, stream=stream,
                          precision="mixed_tf32", **sk)
        roof_mixed = roofline_tc(pk, probe, w, dev, stream)
        probe.close()
    roof_oz = None
    if any(FORMS[f][1] == "ozaki" for f in results):
        probe = pk.Solver(V_d, w.N, w.k, w.sbsize, rr_period=w.rr_period, maxiter=1, device=dev, stream=stream,
                          fp64_gemm="ozaki", **sk)
        roof_oz = roofline_ozaki(pk, probe, w, dev, stream)
        probe.close()
    e2e = None if args.no_e2e else run_e2e(pk, w, V, X0, max(1, args.steps // 2), stream)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(w, args.cpu_iters, iters // max(1, args.steps), stored=args.workload == "grid32_k256")
    if rank != 0:
        return 0
    line = {
        "metric": METRIC, "value": ms_per_step / 1e3, "unit": "s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": w.name, "n": w.n, "k": w.k, "sbsize": w.sbsize, "rr_period": w.rr_period,
                   "tol": w.tol, "form": first,
                   "potential": (f"{w.n_wells} Gaussian wells + U[0,0.1) noise" if w.potential == "wells"
                                 else "V ~ U[0,1)"),
                   "operator": (f"complex Bloch twist {w.theta}, solved in the real form of order 2n"
                                if w.dtype == "c128" else "real symmetric"),
                   "l2": f"no flush: working set {7 * w.n * w.k * 8 / 2**20:.0f} MiB > {L2_BYTES // 2**20} MiB L2"},
        "iters": fp64["iters"], "iters_per_s": fp64["iters_per_s"], "wall_s_per_step": fp64["wall_s_per_step"],
        "parity": parity, "roofline": roof, "phase_ms": phases, "jacobi_sweeps_max": fp64["jacobi_sweeps_max"],
        "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches, "clocks": clk.summary(),
        "counts": fp64["counts"],
        "forms": {
            name: {"form": FORM_TEXT[name], "value": f["ms_per_step"] / 1e3, "unit": "s", "iters": f["iters"],
                   "iters_per_s": f["iters_per_s"],
                   "speedup_vs_fp64": (results["fp64"]["ms_per_step"] / f["ms_per_step"]) if "fp64" in results else None,
                   "parity": f["parity"], "phase_ms": f["phase_ms"], "gpu_launches": f["launches"],
                   "counts": f["counts"]}
            for name, f in results.items()},
        "roofline_tf32_gram": roof_mixed,
        "roofline_stencil": roof_stencil,
        "roofline_ozaki_gram": roof_oz,
    }
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def run_batched(args):
    """The batched workload (64 independent problems, N in 12..28, k in 32..256): sbsize per k bucket from the
    library's autotuner, then every step solves all problems concurrently through ppcg_solve_batched."""
    import torch
    import paper_1407_7506_gb300 as pk
    from paper_1407_7506_gb300 import build as _build
    rank, world, local = _env_rank()
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    if rank == 0:
        _build.build()
    if dist:
        dist.barrier()
    dev = torch.device("cuda", local)
    ws = wl.batch()
    inputs = [wl.make_inputs(w) for w in ws]
    # autotune q on the median problem of each k bucket (outside the timed region)
    buckets = {"k<144": [i for i, w in enumerate(ws) if w.k < 144], "k>=144": [i for i, w in enumerate(ws) if w.k >= 144]}
    tuned, tune_info = {}, {}
    cands = [1, 2, 4, 8]
    t_tune = time.perf_counter()
    for name, idx in buckets.items():
        if not idx:
            continue
        i = sorted(idx, key=lambda j: ws[j].n * ws[j].k)[len(idx) // 2]
        w = ws[i]
        V, X0 = inputs[i]
        Vd = torch.from_numpy(V).to(dev)
        X0d = torch.from_numpy(np.ascontiguousarray(X0.T)).to(dev)
        op = pk.ppcg_operator(w.N, w.N, w.N, 1.0, Vd.data_ptr(), (ctypes.c_double * 3)(0.0, 0.0, 0.0), 0)
        opt = pk.ppcg_options()
        opt.maxiter = args.maxiter
        opt.fp64_gemm = 1 if args.batch_gemm == "ozaki" else 0
        best, times = pk.ppcg_autotune_sbsize(op, w.n, w.k, w.rr_period, opt, X0d.data_ptr(), w.tol, cands,
                                              torch.cuda.current_stream(dev).cuda_stream)
        tuned[name] = best
        tune_info[name] = {"problem": w.name, "candidates": cands, "ms": [round(t, 2) for t in times], "best": best}
    t_tune = time.perf_counter() - t_tune
    problems = []
    for w, (V, _) in zip(ws, inputs):
        q = tuned["k<144" if w.k < 144 else "k>=144"]
        problems.append({"V": V, "grid": w.N, "k": w.k, "sbsize": min(q, w.k), "rr_period": w.rr_period})
    X0s = [torch.from_numpy(np.ascontiguousarray(X0.T)).to(dev) for _, X0 in inputs]   # resident in HBM
    torch.cuda.synchronize()
    bs = pk.BatchSolver(problems, device=dev, maxiter=args.maxiter, fp64_gemm=args.batch_gemm)
    for _ in range(args.warmup):
        bs.solve(X0s, tol=1e-8, max_concurrent=args.batch_concurrency)
    clk = ClockSampler(local)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    launches0 = None
    with clk:
        ev0.record()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            results, status = bs.solve(X0s, tol=1e-8, max_concurrent=args.batch_concurrency)
        torch.cuda.synchronize()
        ev1.record()
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
    ms = max_over_ranks(ev0.elapsed_time(ev1), dist, dev) / args.steps
    # the same batch one problem at a time, for the concurrency gain (outside the timed region)
    t1 = time.perf_counter()
    bs.solve(X0s, tol=1e-8, max_concurrent=1)
    torch.cuda.synchronize()
    seq = time.perf_counter() - t1
    per = [r[3]["time_ms"] / 1e3 for r in results]
    iters = [r[3]["iters"] for r in results]
    launches = sum(r[3]["kernel_launches"] for r in results) * args.steps
    maxres = max(float(np.max(r[2])) for r in results)
    conv = all(r[3]["converged"] == 1 for r in results)
    bs.close()
    if rank != 0:
        return 0
    line = {
        "metric": "aggregate time-to-tol 1e-8 of 64 independent problems (batched), 1 GB300", "value": ms / 1e3,
        "unit": "s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "batch64_grid12-28_k32-256_uniform", "problems": len(ws),
                   "n_range": [min(w.n for w in ws), max(w.n for w in ws)],
                   "k_range": [min(w.k for w in ws), max(w.k for w in ws)], "sbsize": tuned,
                   "concurrency": args.batch_concurrency, "fp64_gemm": args.batch_gemm,
                   "l2": "per-problem working sets 2-45 MB; no flush"},
        "per_problem_s": {"min": min(per), "median": statistics.median(per), "max": max(per),
                          "all": [round(x, 4) for x in per]},
        "iters": {"min": min(iters), "median": statistics.median(iters), "max": max(iters)},
        "sequential_s": seq, "concurrency_speedup": seq / (ms / 1e3), "wall_s_per_step": wall / args.steps,
        "autotune": {"buckets": tune_info, "seconds": t_tune},
        "parity": {"converged": conv, "max_residual": maxres, "status": status},
        "gpu_launches": launches, "clocks": clk.summary(), "roofline": None, "cpu_baseline": None, "e2e": None,
    }
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def roofline(pk, solver, w, dev, stream):
    import torch
    f = 2 if w.dtype == "c128" else 1            # a complex handle's GEMMs run on the real form: 2n x 2k
    n, k = f * w.n, f * w.k
    g = torch.Generator(device="cpu").manual_seed(1)
    A = torch.randn((k, n), generator=g, dtype=torch.float64).to(dev)
    B = torch.randn((k, n), generator=g, dtype=torch.float64).to(dev)
    C = torch.empty((k, k), dtype=torch.float64, device=dev)
    for _ in range(3):
        pk.ppcg_gram(solver.handle, A.data_ptr(), n, B.data_ptr(), n, k, k, C.data_ptr())
    reps = 20
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(reps):
        pk.ppcg_gram(solver.handle, A.data_ptr(), n, B.data_ptr(), n, k, k, C.data_ptr())
    e1.record(stream)
    torch.cuda.synchronize()
    dur = e0.elapsed_time(e1) / reps / 1e3
    flops = 2.0 * n * k * k
    ach = flops / dur / 1e12
    return {"kernel": f"gram_tn_kernel (+ split-K reduce): FP64 X^T W, n={n}, {k}x{k}", "bound": "alu",
            "achieved": ach, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": ach / FP64_PEAK_TFLOPS,
            "traffic": ROOFLINE_TRAFFIC_BYTES, "algorithmic_flops_per_launch": flops, "launch_ms": dur * 1e3,
            "peak_note": "FP64 FMA pipe: 152 SMs x 2 FMA/clk x 2 flop x 2.07 GHz (nominal 1.25 TFLOP/s)"}


def _time_ms(fn, stream, reps):
    import torch
    for _ in range(3):
        fn()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(reps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def roofline_stencil(pk, solver, w, dev, stream):
    """The operator on a full n x k block: 7 FP64 instructions (6 additions and a multiply-add; 6 when h = 1) and
    16 bytes per output element plus 8 n bytes of diagonal. At 0.44 op/B it is bound by the FP64 pipe's
    instruction rate (152 SMs x 2 lanes x 2.07 GHz = 629 G lane-operations/s), not by HBM."""
    import torch
    f = 2 if w.dtype == "c128" else 1
    n, k = f * w.n, f * w.k
    g = torch.Generator(device="cpu").manual_seed(3)
    X = torch.randn((k, n), generator=g, dtype=torch.float64).to(dev)
    Y = torch.empty_like(X)
    ms = _time_ms(lambda: pk.ppcg_apply_operator(solver.handle, X.data_ptr(), n, Y.data_ptr(), n, k), stream, 20)
    per = (6.0 if w.h == 1.0 else 7.0) * (2.0 if w.dtype == "c128" else 1.0)     # per grid point and column
    ops = per * w.n * k
    nbytes = 16.0 * n * k + 8.0 * n
    ach = ops / (ms / 1e3) / 1e9
    peak = FP64_PEAK_TFLOPS * 1e3 / 2.0                                          # lane-operations per second (G)
    hbm, kind = hbm_peak()
    return {"kernel": f"stencil_kernel: A X on {n} x {k}", "bound": "alu", "achieved": ach, "peak": peak,
            "unit": "G FP64 ops/s", "frac": ach / peak, "traffic": None, "launch_ms": ms,
            "hbm_gbs": nbytes / (ms / 1e3) / 1e9, "hbm_frac": nbytes / (ms / 1e3) / 1e9 / hbm,
            "peak_note": f"FP64 pipe instruction rate (2 lanes per SM per clock); HBM against the {kind} copy "
                         "bandwidth"}


def roofline_ozaki(pk, solver, w, dev, stream):
    """FP64-accurate Gram X^T W on the BF16 tensor cores (8 digit slices, 36 products): FP64-equivalent TFLOP/s and
    the BF16 tensor work against the measured BF16 peak."""
    import torch
    f = 2 if w.dtype == "c128" else 1
    n, k = f * w.n, f * w.k
    g = torch.Generator(device="cpu").manual_seed(4)
    A = torch.randn((k, n), generator=g, dtype=torch.float64).to(dev)
    B = torch.randn((k, n), generator=g, dtype=torch.float64).to(dev)
    C = torch.empty((k, k), dtype=torch.float64, device=dev)
    ms = _time_ms(lambda: pk.ppcg_gram(solver.handle, A.data_ptr(), n, B.data_ptr(), n, k, k, C.data_ptr()),
                  stream, 20)
    fp64_eq = 2.0 * n * k * k / (ms / 1e3) / 1e12
    tensor = 36 * 2.0 * n * k * k / (ms / 1e3) / 1e12
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            bf16, kind = float(json.load(fh)["bf16_tflops"]), "measured"
    except (OSError, KeyError, ValueError):
        bf16, kind = 1900.0, "fallback"
    return {"kernel": f"Ozaki Gram (exponents + digit images + oz_img_kernel + reduce): X^T W, n={n}, {k}x{k}",
            "bound": "tensor", "achieved": tensor, "peak": bf16, "unit": "TFLOP/s", "frac": tensor / bf16,
            "traffic": None, "launch_ms": ms, "fp64_equivalent_tflops": fp64_eq,
            "fp64_equivalent_vs_fp64_peak": fp64_eq / FP64_PEAK_TFLOPS,
            "peak_note": f"{kind} dense BF16 burst peak; tensor work = 36 digit-pair products x 2 n k^2"}


def hbm_peak():
    """Measured HBM copy bandwidth (GB/s) from MEASURED_PEAKS.json, else the recipe's fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def roofline_tc(pk, solver, w, dev, stream):
    """Mixed form: the tcgen05 TF32 Gram X^T W reads FP64 inputs; HBM is its bound at k = 256."""
    import torch
    f = 2 if w.dtype == "c128" else 1
    n, k = f * w.n, f * w.k
    g = torch.Generator(device="cpu").manual_seed(2)
    A = torch.randn((k, n), generator=g, dtype=torch.float64).to(dev)
    B = torch.randn((k, n), generator=g, dtype=torch.float64).to(dev)
    C = torch.empty((k, k), dtype=torch.float64, device=dev)
    for _ in range(3):
        pk.ppcg_gram(solver.handle, A.data_ptr(), n, B.data_ptr(), n, k, k, C.data_ptr())
    reps = 50
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(reps):
        pk.ppcg_gram(solver.handle, A.data_ptr(), n, B.data_ptr(), n, k, k, C.data_ptr())
    e1.record(stream)
    torch.cuda.synchronize()
    dur = e0.elapsed_time(e1) / reps / 1e3
    nbytes = 8.0 * n * 2 * k
    peak, kind = hbm_peak()
    ach = nbytes / dur / 1e9
    return {"kernel": f"tc_gram_kernel (tcgen05 TF32, + split-K reduce): X^T W, n={n}, {k}x{k}", "bound": "hbm",
            "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
            "traffic": TF32_GRAM_TRAFFIC_BYTES if (n, k) == (32768, 256) else None,
            "algorithmic_bytes_per_launch": nbytes, "launch_ms": dur * 1e3, "tflops": 2.0 * n * k * k / dur / 1e12,
            "peak_note": f"{kind} HBM copy bandwidth"}


def run_e2e(pk, w, V, X0, steps, stream):
    """The same solve through the C ABI with host buffers: copies in/out are inside the timed region."""
    import torch
    n, k = w.n, w.k
    cplx = w.dtype == "c128"
    Vh = torch.from_numpy(V).pin_memory()
    X0h = torch.from_numpy(np.ascontiguousarray(X0.T)).pin_memory()
    Xh = torch.empty((k, n), dtype=torch.complex128 if cplx else torch.float64).pin_memory()
    lam = np.zeros(k)
    res = np.zeros(k)
    op = pk.ppcg_operator(w.N, w.N, w.N, w.h, Vh.data_ptr(), (ctypes.c_double * 3)(*w.theta), 1 if cplx else 0)
    opt = pk.ppcg_options()
    opt.maxiter = 6000
    h = pk.ppcg_create(op, n, k, w.sbsize, w.rr_period, opt, stream.cuda_stream)
    try:
        pk.ppcg_solve(h, X0h.data_ptr(), w.tol, lam.ctypes.data, Xh.data_ptr(), res.ctypes.data)   # warm
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(steps):
            pk.ppcg_set_potential(h, Vh.data_ptr())
            pk.ppcg_solve(h, X0h.data_ptr(), w.tol, lam.ctypes.data, Xh.data_ptr(), res.ctypes.data)
        el = (time.perf_counter() - t0) / steps
    finally:
        pk.ppcg_destroy(h)
    es = 16 if cplx else 8
    return {"value": el, "unit": "s", "h2d_bytes_per_step": 8 * n + es * n * k, "d2h_bytes_per_step": es * n * k + 16 * k,
            "steps": steps, "max_residual": float(np.max(res))}


if __name__ == "__main__":
    sys.exit(main())
