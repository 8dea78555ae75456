#!/usr/bin/env python3
"""Benchmark of the GB300 PPCG eigensolver: time-to-tolerance (max residual 1e-8) and PPCG iterations/s, mixed
form against the FP64 form, with the roofline of the dominant kernels.

One step = one complete ppcg_solve (Algorithm 3: orthonormalisation, Rayleigh-Ritz steps, preconditioned
projected search directions, sub-block Rayleigh-Ritz, CholeskyQR2, locking) from the seeded starting block to
max residual 1e-8, on the 48^3-grid / k = 1024 / sbsize = 8 / 32-well workload, with V and X0 resident in HBM.
The headline `value` is the mixed form (TF32 tensor-core projections, the other n x k GEMMs FP64-accurate on the
tensor cores); the FP64 forms are timed beside it.

Prints one JSON line. Also reported:
  forms         every form's time-to-tol, iterations, per-phase times and parity; forms too slow for a full solve
                per step (FP64 on the FMA pipe) are timed over their first iterations and extrapolated
  roofline      the dominant kernel (the FP64-accurate tensor-core Gram) timed live with CUDA events; roofline_*
                for the other hot kernels, and the k x k eigensolve times
  parity        residuals of the benchmarked solve, and the same solve on a separable potential of the same size
                against its exact spectrum (sums of three 1-D spectra)
  e2e           the same metric through the C ABI with host (pinned) buffers: V and X0 copied in and X,
                lambda, residuals copied out inside the timed region
  cpu_baseline  the CPU oracle (numpy/LAPACK Algorithm 3): its components timed on the workload's data, summed
                along the iteration's active-column trajectory (extrapolated time-to-tol)
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
L2_BYTES = 129 * 2 ** 20
WORKLOADS = {"grid48_k1024": wl.GRID48_K1024, "grid32_k256": wl.GRID32_K256, "grid16_k64": wl.GRID16_K64,
             "grid32_k128_bloch": wl.GRID32_K128_BLOCH, "grid48_k512_bloch": wl.GRID48_K512_BLOCH}


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


# ------------------------------------------------------------------------------------------------ CPU oracle
def _oracle_threads():
    try:
        import threadpoolctl
        info = threadpoolctl.threadpool_info()
        return max([i.get("num_threads", 0) for i in info if i.get("user_api") == "blas"] or [0]) or None
    except Exception:
        return None


def _host_cores():
    return len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()


ORACLE_COMPONENTS = ("orth", "rr", "H", "precond", "project", "blocks", "resid", "copy")


class OracleCost:
    """Time-to-tol of the CPU oracle (the plain Algorithm 3 of oracle/), predicted from its components timed on the
    workload's own data at full width (k_act = k) and summed along an iteration's active-column trajectory.

    Per iteration with k_a active of k_t columns (a = k_a / k_t) the oracle runs: precondition, the sub-block loop
    (three operator applications per block, the small generalised eigenproblem, the update) and the projections of
    W (and of P from iteration 2) against [X, X_lock], all proportional to a; a plain step adds CholeskyQR2 and
    M = X^T A X, W = A X - X M (proportional to a^2, their n k_a^2 GEMMs dominate) and one operator application (a); a
    Rayleigh-Ritz step adds the Rayleigh-Ritz on all k_t columns with its residuals (constant). The solve starts
    with CholeskyQR2 of X0 and one Rayleigh-Ritz step."""

    def __init__(self, w, V=None, X0=None):
        self.w = w
        if V is None:
            V, X0 = wl.make_inputs(w)
        self.V, self.X0 = V, X0
        self._X = None

    def _data(self):
        import oracle
        if self._X is None:
            w = self.w
            rng = np.random.default_rng(w.seed + 17)
            self._X = oracle.orth(np.asfortranarray(self.X0))
            shape = self._X.shape
            cplx = np.iscomplexobj(self._X)
            r = lambda: rng.standard_normal(shape) + (1j * rng.standard_normal(shape) if cplx else 0.0)
            # W and P in the memory order they have inside the oracle's loop (W = A X - X M and P = the block
            # update's output are row-major numpy results), so their column slices cost what they cost there
            self._W, self._P = np.ascontiguousarray(r()), np.ascontiguousarray(r())
        return self._X, self._W, self._P

    def time_component(self, name):
        """Seconds of one oracle component at full width on this workload, with the data layouts and copies of
        its loop (the sub-block loop over a slice of the sub-blocks, scaled to all of them)."""
        import oracle
        w = self.w
        theta = w.theta if w.dtype == "c128" else None
        N, h, q = w.N, w.h, w.sbsize
        Hop = lambda Y: oracle.apply_H(self.V, N, h, Y, theta)
        X, W, P = self._data()
        kt = X.shape[1]
        t0 = time.perf_counter()
        if name == "orth":
            oracle.orth(np.asfortranarray(self.X0))
        elif name == "rr":
            S = np.hstack([X, X[:, :0]])
            Xf, lam = oracle.rayleigh_ritz(S, Hop)
            Wf = oracle.residual(Xf, Hop(Xf), lam)
            np.linalg.norm(Wf, axis=0)
            Pfull = np.zeros(P.shape, dtype=P.dtype)
            Pfull[:, list(range(kt))] = P
            np.asfortranarray(Pfull[:, list(range(kt))])
        elif name == "H":
            Hop(X)
        elif name == "precond":
            oracle.precondition(W, self.V, N, h, 0.0, 0.1 / (h * h))
        elif name == "project":
            oracle.project(oracle.project(W, X), X[:, :0])
        elif name == "copy":
            X[:, list(range(kt))]
        elif name == "blocks":
            blocks = oracle.subblocks(kt, q)
            take = blocks[:max(1, len(blocks) // 8)]
            Xn, Pn = np.empty_like(X), np.empty_like(W)
            for (a, b) in take:
                Xj, Wj, Pj = X[:, a:b], W[:, a:b], P[:, a:b]
                if np.any(np.linalg.norm(Pj, axis=0) == 0.0):
                    Pj = None
                CX, CW, CP = oracle.block_coefficients(Xj, Wj, Pj, Hop(Xj), Hop(Wj), Hop(Pj))
                Xn[:, a:b], Pn[:, a:b] = oracle.block_update(Xj, Wj, Pj, CX, CW, CP)
            return (time.perf_counter() - t0) * len(blocks) / len(take)
        elif name == "resid":
            HX = Hop(X)
            t0 = time.perf_counter()
            M = X.conj().T @ HX
            oracle.residual(X, HX, M)
        else:
            raise ValueError(name)
        return time.perf_counter() - t0

    def measure(self, names=ORACLE_COMPONENTS):
        return {nm: self.time_component(nm) for nm in names}

    @staticmethod
    def predict(t, trajectory, kt):
        """trajectory: (iteration, kind, k_act) per iteration after the start (kind 0 plain, 1 Rayleigh-Ritz),
        iteration 0 being the initial Rayleigh-Ritz step."""
        total = t["orth"] + t["rr"]
        prev = None
        for it, kind, ka in trajectory:
            if it == 0 or it == prev:                             # the history repeats the final step's entry
                continue
            prev = it
            a = ka / kt
            total += (t["precond"] + t["blocks"]) * a + t["project"] * a * (1 if it == 1 else 2)
            total += t["copy"] * (kt - ka) / kt                   # X_lock = X[:, J_lock] at every iteration
            if kind == 0:
                total += (t["orth"] + t["resid"]) * a * a + t["H"] * a
            else:
                total += t["rr"]
        return total


def oracle_trajectory(history, kt):
    """(iteration, kind, k_act) from an oracle history (k_act from the lock count of the latest Rayleigh-Ritz
    step)."""
    out, ka = [], kt
    for h in history:
        out.append((h["iter"], 1 if h["rr"] else 0, ka))
        if h["rr"]:
            ka = kt - h["n_lock"]
    return out


# The iteration trajectory of the benchmarked 48^3 mixed-form solve (k = 1024 with 50 buffer vectors), for the
# reference arm (which runs no GPU code):
# runs of iterations [first, last] with the same number of active columns, and the Rayleigh-Ritz iterations, as the
# library's solve history recorded them (bench.py prints them as "trajectory"). The main arm uses the trajectory
# of its own timed solve instead.
TRAJECTORY_GRID48 = {
    "runs": [(1, 25, 1074), (26, 30, 1069), (31, 35, 929), (36, 40, 796), (41, 45, 683), (46, 50, 573),
             (51, 55, 479), (56, 60, 426), (61, 65, 369), (66, 70, 325), (71, 75, 294), (76, 80, 255), (81, 85, 231),
             (86, 90, 211), (91, 95, 189), (96, 100, 174), (101, 105, 161), (106, 110, 149), (111, 115, 140),
             (116, 120, 126), (121, 125, 117), (126, 130, 105), (131, 135, 97), (136, 140, 90), (141, 145, 82),
             (146, 150, 76), (151, 155, 73), (156, 160, 68), (161, 165, 64), (166, 170, 57), (171, 175, 55),
             (176, 182, 51), (182, 182, 51)],
    "rr": sorted(set(range(5, 181, 5)) | {182}),
}


def trajectory_summary(traj):
    """Compact form of a trajectory: runs of equal k_act and the list of Rayleigh-Ritz iterations."""
    runs, rr = [], []
    for it, kind, ka in traj:
        if it == 0:
            continue
        if kind == 1:
            rr.append(int(it))
        if runs and runs[-1][2] == ka and runs[-1][1] == it - 1:
            runs[-1][1] = int(it)
        else:
            runs.append([int(it), int(it), int(ka)])
    return {"runs": runs, "rr": rr}


def convergence_summary(history, samples=24):
    """Max Ritz residual, active columns and elapsed time at a spread of the solve's Rayleigh-Ritz steps (the
    residual-versus-time view of the paper's Figure "Liband")."""
    rr = [r for r in history if int(r[1]) == 1]
    if not rr:
        return []
    pick = sorted(set(np.linspace(0, len(rr) - 1, min(samples, len(rr))).round().astype(int).tolist()))
    return [{"iter": int(rr[i][0]), "t_ms": round(float(rr[i][5]), 1), "max_res": float(rr[i][2]),
             "k_act": int(rr[i][4])} for i in pick]


def trajectory_expand(summary, kt):
    rr = set(summary["rr"])
    out = [(0, 1, kt)]
    for i0, i1, ka in summary["runs"]:
        out.extend((it, 1 if it in rr else 0, ka) for it in range(i0, i1 + 1))
    return out


def cpu_baseline(w, trajectory, label, V=None, X0=None):
    model = OracleCost(w, V, X0)
    model.measure(("H",))                                      # warm the BLAS and the page cache
    t0 = time.perf_counter()
    t = model.measure()
    sampled = time.perf_counter() - t0
    kt = w.k + w.nbuf
    value = OracleCost.predict(t, trajectory, kt)
    iters = sum(1 for it, _, _ in trajectory if it > 0)
    cores = _host_cores()
    return {"value": value, "unit": "s", "cores": _oracle_threads() or cores, "kind": "oracle",
            "sample": (f"oracle Algorithm 3 (numpy/LAPACK FP64) on {w.name}: each component timed once at full "
                       f"width ({sampled:.1f} s of CPU work: " + ", ".join(f"{k_} {v_:.2f} s" for k_, v_ in t.items())
                       + f"); time-to-tol extrapolated along the {label} trajectory of {iters} iterations and "
                       "its active-column counts (the model is checked against a full oracle run at 32^3)"),
            "extrapolated": True, "components_s": t, "iters_per_s": iters / value, "host_cores": cores}


def run_reference(args, w):
    """The reference arm: the CPU oracle as it stands. Each step times one of its components on the workload's data
    (rotating through them); the value is the time-to-tol those component times predict along the benchmarked
    trajectory."""
    rank, world, _ = _env_rank()
    if rank != 0:
        return 0
    model = OracleCost(w)
    names = ORACLE_COMPONENTS
    for i in range(args.warmup):
        model.time_component(names[i % len(names)])
    samples = {nm: [] for nm in names}
    step_s = []
    for i in range(max(args.steps, len(names))):
        nm = names[i % len(names)]
        t0 = time.perf_counter()
        samples[nm].append(model.time_component(nm))
        step_s.append(time.perf_counter() - t0)
    t = {nm: statistics.median(v) for nm, v in samples.items()}
    traj = reference_trajectory(w)
    value = OracleCost.predict(t, traj, w.k + w.nbuf)
    iters = sum(1 for it, _, _ in traj if it > 0)
    cores = _host_cores()
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * sum(step_s) / len(step_s), "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(w, "oracle (numpy/LAPACK FP64)"),
            "iters_per_s": iters / value,
            "cpu_baseline": {"value": value, "unit": "s", "cores": _oracle_threads() or cores, "kind": "oracle",
                             "sample": ("each step times one component of the oracle's iteration at full width on "
                                        f"the workload's data ({', '.join(names)}, rotating; medians used); "
                                        f"time-to-tol extrapolated along a {iters}-iteration trajectory with its "
                                        "active-column counts"),
                             "extrapolated": True, "components_s": t},
            "e2e": {"value": value, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def reference_trajectory(w):
    """Trajectory for the reference arm: the stored run-length summary for the 48^3 workload, else (smaller
    workloads) the oracle's own full run, which finishes in minutes there."""
    if w.name == wl.GRID48_K1024.name and TRAJECTORY_GRID48:
        return trajectory_expand(TRAJECTORY_GRID48, w.k + w.nbuf)
    import oracle
    V, X0 = wl.make_inputs(w)
    r = oracle.ppcg(V, w.N, w.h, w.k, w.sbsize, w.rr_period, X0, tol=w.tol, maxiter=6000, nbuf=w.nbuf,
                    theta=w.theta if w.dtype == "c128" else None)
    return oracle_trajectory(r.history, w.k + w.nbuf)


def workload_config(w, form):
    return {"workload": w.name, "n": w.n, "k": w.k, "sbsize": w.sbsize, "rr_period": w.rr_period, "tol": w.tol,
            "nbuf": w.nbuf, "form": form,
            "potential": (f"{w.n_wells} Gaussian wells + U[0,0.1) noise" if w.potential == "wells"
                          else "V ~ U[0,1)"),
            "operator": (f"complex Bloch twist {w.theta}, solved in the real form of order 2n"
                         if w.dtype == "c128" else "real symmetric"),
            "l2": (f"no flush: working set {7 * w.n * w.k * 8 / 2**20:.0f} MiB > {L2_BYTES // 2**20} MiB L2"
                   if 7 * w.n * w.k * 8 > L2_BYTES else
                   f"no flush: working set {7 * w.n * w.k * 8 / 2**20:.0f} MiB fits the {L2_BYTES // 2**20} MiB L2; "
                   "every pass of the solve reuses it, as the method does")}


# form name -> (precision, how the FP64 n x k GEMMs run, step-18 orthonormalisation)
FORMS = {
    "fp64": ("fp64", "fma", "cholqr2"),
    "mixed": ("mixed_tf32", "fma", "cholqr2"),
    "fp64_ozaki": ("fp64", "ozaki", "cholqr2"),
    "mixed_ozaki": ("mixed_tf32", "ozaki", "cholqr2"),
    "fp64_ozaki_polar": ("fp64", "ozaki", "polar"),
    "mixed_ozaki_polar": ("mixed_tf32", "ozaki", "polar"),
    "mixed_bf16_ozaki": ("mixed_bf16", "ozaki", "cholqr2"),
    "mixed_ozaki_nbuf0": ("mixed_tf32", "ozaki", "cholqr2"),
}
# forms that override the workload's number of buffer vectors
FORM_NBUF = {"mixed_ozaki_nbuf0": 0}
FORM_TEXT = {
    "fp64": "FP64 throughout (FP64 FMA pipe GEMMs), CholeskyQR2",
    "mixed": "TF32 tcgen05 projection GEMMs and first CholeskyQR Gram; the other GEMMs on the FP64 FMA pipe",
    "fp64_ozaki": "FP64 with the n x k GEMMs emulated on BF16 tcgen05 (8 digit slices, Ozaki)",
    "mixed_ozaki": "mixed: TF32 tcgen05 projections and first CholeskyQR Gram, the other FP64 n x k GEMMs emulated "
                   "on BF16 tcgen05 (Ozaki)",
    "fp64_ozaki_polar": "fp64_ozaki with the polar-series orthonormalisation of Section 5.5",
    "mixed_ozaki_polar": "mixed_ozaki with the polar-series orthonormalisation of Section 5.5",
    "mixed_bf16_ozaki": "mixed with BF16 tcgen05 projections and first CholeskyQR Gram (FP32 accumulation), the "
                        "other FP64 n x k GEMMs emulated on BF16 tcgen05 (Ozaki)",
    "mixed_ozaki_nbuf0": "mixed_ozaki without buffer vectors (X has exactly k columns)",
}
# the FP64-accurate tensor-core form whose full solve stands in for each windowed form's iteration count
WINDOW_PARTNER = {"fp64": "fp64_ozaki", "mixed": "mixed_ozaki"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="grid48_k1024", choices=list(WORKLOADS) + ["batch64"],
                    help="grid48_k1024 (default: the mixed-form workload), grid32_k256, grid16_k64, "
                         "grid48_k512_bloch, grid32_k128_bloch (the complex Bloch recipe), batch64 (64 uneven "
                         "problems)")
    ap.add_argument("--maxiter", type=int, default=6000)
    ap.add_argument("--forms", default="mixed_ozaki,fp64_ozaki,mixed_bf16_ozaki,mixed_ozaki_nbuf0",
                    help="forms solved to tolerance; the first is the headline value (" + ", ".join(FORMS) + ")")
    ap.add_argument("--form-repeats", type=int, default=2, help="timed solves of each non-headline form")
    ap.add_argument("--window-forms", default="fp64,mixed",
                    help="forms too slow for full solves: timed over their first --window-iters iterations")
    ap.add_argument("--window-iters", type=int, default=10)
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-separable", action="store_true")
    ap.add_argument("--kernels-only", action="store_true",
                    help="only the roofline timings of the hot kernels at the workload's shape (for profiling)")
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
    X0_d = torch.from_numpy(np.ascontiguousarray(X0.T)).to(dev)         # (k + nbuf, n) rows = columns of X0
    X0_by_nbuf = {w.nbuf: X0_d}

    def start(form):
        nb = FORM_NBUF.get(form, w.nbuf)
        if nb not in X0_by_nbuf:
            X0_by_nbuf[nb] = torch.from_numpy(np.ascontiguousarray(wl.make_inputs(w, ncols=w.k + nb)[1].T)).to(dev)
        return X0_by_nbuf[nb]
    gold = stored_eigs(w)
    cplx = w.dtype == "c128"
    sk = {"dtype": w.dtype, "theta": w.theta} if cplx else {}          # Solver arguments of the operator
    if args.kernels_only:
        print(json.dumps(rooflines(pk, w, dev, stream, V_d, sk)), flush=True)
        return 0

    def solver(form, **kw):
        prec, gm, orth = FORMS[form]
        return pk.Solver(V_d, w.N, w.k, w.sbsize, rr_period=w.rr_period, device=dev, stream=stream, precision=prec,
                         fp64_gemm=gm, orth=orth, nbuf=FORM_NBUF.get(form, w.nbuf), **sk, **kw)

    def run_form(form, steps, warmup, clk_sampler):
        s = solver(form, maxiter=args.maxiter, history=args.maxiter + 8)
        X_out = torch.empty((w.k, w.n), dtype=s.dtype, device=dev)
        X0_f = start(form)
        for _ in range(warmup):
            s.solve(X0_f, w.tol, out=X_out)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        iters, launches, stats = 0, 0, []
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        with clk_sampler:
            ev0.record(stream)
            t0 = time.perf_counter()
            for _ in range(steps):
                lam, _, res, st = s.solve(X0_f, w.tol, out=X_out)
                iters += st["iters"]
                launches += st["kernel_launches"]
                stats.append(st)
            ev1.record(stream)
            torch.cuda.synchronize()
            wall = time.perf_counter() - t0
        if dist:
            dist.barrier()
        ms = max_over_ranks(ev0.elapsed_time(ev1), dist, dev)
        s.close()
        return {"ms_per_step": ms / steps, "iters": iters // steps, "iters_per_s": iters / (ms / 1e3),
                "wall_s_per_step": wall / steps, "launches": launches, "steps": steps,
                "parity": parity_of(lam, res, stats, gold), "history": stats[-1]["history"],
                "counts": {k_: stats[-1][k_] for k_ in ("n_rr", "n_drop_p", "n_cholqr_fallback", "n_polar",
                                                         "n_orth_skip", "n_eig_diagonal", "n_eig_refined",
                                                         "n_eig_mixed", "n_rr_unit", "n_locked")}}

    def phase_solve(form, maxiter):
        s = solver(form, maxiter=maxiter, timing=True)
        _, _, _, st = s.solve(start(form), w.tol)
        s.close()
        return {k_: round(v_, 2) for k_, v_ in st["t_phase_ms"].items()}, st

    forms = [f.strip() for f in args.forms.split(",") if f.strip()]
    first = forms[0]
    clk = ClockSampler(local)
    results = {}
    for f in forms:
        if f == first:
            results[f] = run_form(f, args.steps, args.warmup, clk)
        else:
            results[f] = run_form(f, max(1, min(args.steps, args.form_repeats)), 1 if args.warmup else 0,
                                  ClockSampler(local))
        results[f]["phase_ms"] = phase_solve(f, args.maxiter)[0]
    # forms too slow to solve to tolerance every step: their first iterations against the same window of the
    # FP64-accurate tensor-core form whose full solve they would repeat (same arithmetic accuracy, same iterates)
    windows = {}
    for f in [x.strip() for x in args.window_forms.split(",") if x.strip()]:
        partner = WINDOW_PARTNER[f]
        tw = {}
        for g in (f, partner):
            s = solver(g, maxiter=args.window_iters)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            _, _, _, st = s.solve(start(g), w.tol)
            e1.record(stream)
            torch.cuda.synchronize()
            s.close()
            tw[g] = (e0.elapsed_time(e1) / 1e3, st["iters"])
        ratio = tw[f][0] / tw[partner][0]
        est = results[partner]["ms_per_step"] / 1e3 * ratio if partner in results else None
        windows[f] = {"form": FORM_TEXT[f], "window_iters": tw[f][1], "window_s": tw[f][0],
                      "iters_per_s_window": tw[f][1] / tw[f][0], "partner": partner, "partner_window_s": tw[partner][0],
                      "time_to_tol_s_extrapolated": est,
                      "basis": (f"not solved to tolerance each step: orthonormalisation, the initial Rayleigh-Ritz "
                                f"step and the first {tw[f][1]} iterations timed once with CUDA events; time-to-tol "
                                f"= {partner}'s measured time-to-tol x the ratio of the two windows")}
    head = results[first]
    traj = [(int(r[0]), int(r[1]), int(r[4])) for r in head["history"]]
    roofs = rooflines(pk, w, dev, stream, V_d, sk)
    sep = None if (args.no_separable or cplx) else separable_parity(pk, w, dev, stream, first, args.maxiter)
    e2e = None if args.no_e2e else run_e2e(pk, w, V, X0, max(1, args.e2e_steps), stream, FORMS[first])
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(w, traj, f"benchmarked {first} solve's", V, X0)
    if rank != 0:
        return 0
    ref_form = "fp64_ozaki" if "fp64_ozaki" in results else None
    line = {
        "metric": METRIC, "value": head["ms_per_step"] / 1e3, "unit": "s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": head["ms_per_step"], "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(w, first),
        "iters": head["iters"], "iters_per_s": head["iters_per_s"], "wall_s_per_step": head["wall_s_per_step"],
        "parity": dict(head["parity"], separable_same_size=sep),
        "roofline": roofs.pop("roofline"), **roofs,
        "phase_ms": head["phase_ms"], "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": head["launches"],
        "clocks": clk.summary(), "counts": head["counts"],
        "forms": {
            name: {"form": FORM_TEXT[name], "value": f["ms_per_step"] / 1e3, "unit": "s", "iters": f["iters"],
                   "iters_per_s": f["iters_per_s"], "timed_solves": f["steps"],
                   "speedup_vs_fp64_ozaki": (results[ref_form]["ms_per_step"] / f["ms_per_step"]) if ref_form else None,
                   "parity": f["parity"], "phase_ms": f["phase_ms"], "gpu_launches": f["launches"],
                   "counts": f["counts"]}
            for name, f in results.items()},
        "window_forms": windows,
        "convergence": convergence_summary(head["history"]),
        "trajectory": trajectory_summary(traj),
    }
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def stored_eigs(w):
    """Stored oracle eigenvalues of a workload, where the oracle finishes (tests/golden/, written by oracle/ only)."""
    path = {wl.GRID32_K256.name: "grid32_k256_oracle_eigs.txt",
            wl.GRID16_K64.name: "grid16_k64_dense_eigs.txt"}.get(w.name)
    if not path:
        return None
    return np.loadtxt(os.path.join(ROOT, "tests", "golden", path))[:w.k] if path.endswith("dense_eigs.txt") else \
        np.loadtxt(os.path.join(ROOT, "tests", "golden", path))[:, 0]


def parity_of(lam, res, stats, gold):
    p = {"max_residual": float(np.max(res)), "converged": all(s_["converged"] == 1 for s_ in stats)}
    if gold is not None:
        p["max_rel_err_vs_oracle"] = float(np.max(np.abs(lam - gold) / np.maximum(np.abs(gold), 1.0)))
    return p


def separable_exact(V1, V2, V3, N, k):
    """The k smallest eigenvalues of -Laplacian + diag(V1(i) + V2(j) + V3(l)) on the periodic N^3 grid: sums of the
    three 1-D spectra (each a dense N x N eigh)."""
    L = 2.0 * np.eye(N) - np.eye(N, k=1) - np.eye(N, k=-1)
    L[0, -1] = L[-1, 0] = -1.0
    e = [np.linalg.eigvalsh(L + np.diag(v)) for v in (V1, V2, V3)]
    return np.sort((e[0][:, None, None] + e[1][None, :, None] + e[2][None, None, :]).ravel())[:k]


def separable_parity(pk, w, dev, stream, form, maxiter):
    """The benchmarked form on a separable potential of the same grid, k and sbsize: eigenvalues against the exact
    spectrum (the wells workload has no independent reference at this size)."""
    import torch
    sw = wl.Workload(w.name.replace(f"wells{w.n_wells}", "separable"), N=w.N, k=w.k, sbsize=w.sbsize,
                     rr_period=w.rr_period, potential="separable", seed=w.seed + 100, nbuf=w.nbuf)
    V, X0 = wl.make_inputs(sw)
    N = w.N
    Vg = V.reshape((N, N, N), order="F")
    exact = separable_exact(Vg[:, 0, 0], Vg[0, :, 0] - Vg[0, 0, 0], Vg[0, 0, :] - Vg[0, 0, 0],
                            N, w.k)
    prec, gm, orth = FORMS[form]
    s = pk.Solver(torch.from_numpy(V).to(dev), N, w.k, w.sbsize, rr_period=w.rr_period, device=dev, stream=stream,
                  precision=prec, fp64_gemm=gm, orth=orth, maxiter=maxiter, nbuf=sw.nbuf)
    t0 = time.perf_counter()
    lam, _, res, st = s.solve(torch.from_numpy(np.ascontiguousarray(X0.T)).to(dev), w.tol)
    el = time.perf_counter() - t0
    s.close()
    return {"workload": sw.name, "form": form, "converged": st["converged"] == 1, "iters": st["iters"],
            "seconds": el, "max_rel_err_vs_exact": float(np.max(np.abs(lam - exact) / np.maximum(np.abs(exact), 1))),
            "max_residual": float(np.max(res))}


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


def _time_ms(fn, stream, reps):
    """Mean device time of fn() in ms: CUDA events on the launching stream, after warm-up."""
    import torch
    for _ in range(2):
        fn()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(reps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), float(d["bf16_tflops"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, 1900.0, "fallback"


# DRAM bytes (read + write) per launch of the Ozaki image kernel (one 1024 x 1024 Gram over n = 110592), from one ncu
# capture of that shape with the current kernel: 4.169 GB read + 43.7 MB written (profiles/oz_img_kernel_grid48_k1024.md)
OZ_IMG_TRAFFIC_BYTES = 4.213e9


def rooflines(pk, w, dev, stream, V_d, sk):
    """Live CUDA-event timings of the hot kernels at the workload's shape (n x k blocks), each against its bound.
    The dominant kernel of the mixed form at this size is the FP64-accurate tensor-core Gram/update (Ozaki digit
    products on BF16 tcgen05), bound by the tensor pipe."""
    import torch
    f = 2 if w.dtype == "c128" else 1            # a complex handle's GEMMs run on the real form: 2n x 2k
    n, k = f * w.n, f * w.k
    hbm, bf16, kind = _peaks()
    g = torch.Generator(device="cpu").manual_seed(1)
    A = torch.randn((k, n), generator=g, dtype=torch.float64).to(dev)
    B = torch.randn((k, n), generator=g, dtype=torch.float64).to(dev)
    C = torch.empty((k, k), dtype=torch.float64, device=dev)
    out = {}

    def handle(**kw):
        return pk.Solver(V_d, w.N, w.k, w.sbsize, rr_period=w.rr_period, device=dev, stream=stream, maxiter=1,
                         **sk, **kw)

    gemm_flops = 2.0 * n * k * k
    # FP64-accurate Gram on the tensor cores: 36 BF16 digit-pair products per FP64 product
    hz = handle(fp64_gemm="ozaki")
    ms = _time_ms(lambda: pk.ppcg_gram(hz.handle, A.data_ptr(), n, B.data_ptr(), n, k, k, C.data_ptr()), stream, 5)
    tens = 36 * gemm_flops / (ms / 1e3) / 1e12
    out["roofline"] = {
        "kernel": f"Ozaki Gram X^T W (exponents + digit images + oz_img_kernel + split-K reduce), n={n}, {k}x{k}",
        "bound": "tensor", "achieved": tens, "peak": bf16, "unit": "TFLOP/s", "frac": tens / bf16,
        "traffic": OZ_IMG_TRAFFIC_BYTES if (n, k) == (110592, 1024) else None,
        "traffic_note": "DRAM bytes of oz_img_kernel<0> alone (the call's main kernel), from one ncu capture",
        "launch_ms": ms, "algorithmic_flops_per_launch": 36 * gemm_flops,
        "fp64_equivalent_tflops": gemm_flops / (ms / 1e3) / 1e12,
        "fp64_equivalent_vs_fp64_peak": gemm_flops / (ms / 1e3) / 1e12 / FP64_PEAK_TFLOPS,
        "peak_note": f"{kind} dense BF16 burst peak; tensor work = 36 digit-pair products x 2 n k^2"}
    Y = B.clone()
    ms_p = _time_ms(lambda: pk.ppcg_project(hz.handle, A.data_ptr(), n, k, Y.data_ptr(), n, k), stream, 3)
    ms_u = max(ms_p - ms, 1e-6)
    out["roofline_ozaki_update"] = {
        "kernel": f"Ozaki update Y -= X G (row digit images + oz_img_kernel), n={n}, {k}x{k} (projection minus Gram)",
        "bound": "tensor", "achieved": 36 * gemm_flops / (ms_u / 1e3) / 1e12, "peak": bf16, "unit": "TFLOP/s",
        "frac": 36 * gemm_flops / (ms_u / 1e3) / 1e12 / bf16, "traffic": None, "launch_ms": ms_u}
    # the k x k eigensolve of the Rayleigh-Ritz step on its three routes, FP64-accurate products on the tensor cores
    rng = np.random.default_rng(5)
    m = k
    R = rng.standard_normal((m, m))
    mats = {"random (FP32 Jacobi + refinement)": R + R.T,
            "nearly diagonal, off-diagonal 1e-5 (refinement from I)":
                np.diag(np.sort(rng.standard_normal(m)) * 10) + 1e-5 * (R + R.T),
            "nearly diagonal, off-diagonal 1e-3 (FP32 Jacobi + refinement)":
                np.diag(np.sort(rng.standard_normal(m)) * 10) + 1e-3 * (R + R.T)}
    lam = torch.empty(m, dtype=torch.float64, device=dev)
    Cm = torch.empty((m, m), dtype=torch.float64, device=dev)
    eig = {}
    for name, Mh in mats.items():
        Md = torch.from_numpy(np.ascontiguousarray(Mh)).to(dev)
        eig[name] = _time_ms(lambda: pk.ppcg_dense_eigh(hz.handle, Md.data_ptr(), m, lam.data_ptr(), Cm.data_ptr()),
                             stream, 3)
    out["dense_eigh_ms"] = {"m": m, **eig,
                            "bound": "latency: grid barriers of the FP32 Jacobi rounds and the m x m products"}
    Xq = A.clone()
    out["cholqr2_ms"] = {"m": k, "n": n, "ms": _time_ms(lambda: (Xq.copy_(A), pk.ppcg_cholqr2(hz.handle, Xq.data_ptr(),
                                                                                             n, k)), stream, 3),
                         "note": "two passes of Ozaki Gram + blocked Cholesky/inverse + Ozaki update, incl. a copy"}
    hz.close()
    # TF32 Gram of the mixed form's projections
    ht = handle(precision="mixed_tf32")
    ms = _time_ms(lambda: pk.ppcg_gram(ht.handle, A.data_ptr(), n, B.data_ptr(), n, k, k, C.data_ptr()), stream, 10)
    nbytes = 8.0 * n * 2 * k
    ach = nbytes / (ms / 1e3) / 1e9
    out["roofline_tf32_gram"] = {
        "kernel": f"tc_gram_kernel (tcgen05 TF32, + split-K reduce): X^T W, n={n}, {k}x{k}", "bound": "hbm",
        "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
        "traffic": None,                  # the launch grid changed since the last capture (K split for whole waves)
        "algorithmic_bytes_per_launch": nbytes, "launch_ms": ms, "tflops": gemm_flops / (ms / 1e3) / 1e12,
        "peak_note": f"{kind} HBM copy bandwidth (FP64 operands read once); at k = {k} the TF32 tensor work "
                     f"({gemm_flops / 1e9:.0f} GFLOP) is within a factor of two of the byte bound"}
    ht.close()
    hb = handle(precision="mixed_bf16")
    ms = _time_ms(lambda: pk.ppcg_gram(hb.handle, A.data_ptr(), n, B.data_ptr(), n, k, k, C.data_ptr()), stream, 10)
    ach = nbytes / (ms / 1e3) / 1e9
    out["roofline_bf16_gram"] = {
        "kernel": f"tc_gram_kernel (tcgen05 kind::f16, BF16 operands, + split-K reduce): X^T W, n={n}, {k}x{k}",
        "bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm, "traffic": None,
        "algorithmic_bytes_per_launch": nbytes, "launch_ms": ms, "tflops": gemm_flops / (ms / 1e3) / 1e12,
        "tensor_frac": gemm_flops / (ms / 1e3) / 1e12 / bf16,
        "peak_note": f"{kind} HBM copy bandwidth (FP64 operands read once); tensor_frac against the {kind} BF16 peak"}
    hb.close()
    hf = handle()
    # the stencil: 6 FP64 additions and one multiply-add (h = 1: 6 operations) per output, 16 B per output
    X = A
    Yo = torch.empty_like(X)
    ms = _time_ms(lambda: pk.ppcg_apply_operator(hf.handle, X.data_ptr(), n, Yo.data_ptr(), n, k), stream, 10)
    per = (6.0 if w.h == 1.0 else 7.0) * (2.0 if w.dtype == "c128" else 1.0)
    ops = per * w.n * k
    sbytes = 16.0 * n * k + 8.0 * n
    peak_ops = FP64_PEAK_TFLOPS * 1e3 / 2.0
    out["roofline_stencil"] = {
        "kernel": f"stencil_kernel: A X on {n} x {k}", "bound": "alu", "achieved": ops / (ms / 1e3) / 1e9,
        "peak": peak_ops, "unit": "G FP64 ops/s", "frac": ops / (ms / 1e3) / 1e9 / peak_ops, "traffic": None,
        "launch_ms": ms, "hbm_gbs": sbytes / (ms / 1e3) / 1e9, "hbm_frac": sbytes / (ms / 1e3) / 1e9 / hbm,
        "peak_note": f"FP64 pipe instruction rate (152 SMs x 2 lanes x 2.07 GHz); HBM against the {kind} copy "
                     "bandwidth"}
    # sub-block Grams + small eigensolves (steps 11-13) and the block update (steps 14-15), FP64 pipe
    q = w.sbsize * f
    Wb, Pb = B, B.clone()
    HX, HW, HP = torch.empty_like(X), torch.empty_like(X), torch.empty_like(X)
    s_blocks = -(-k // q)
    coef = torch.zeros(s_blocks * 3 * q * q, dtype=torch.float64, device=dev)
    flags = torch.zeros(s_blocks, dtype=torch.int32, device=dev)
    ms_b = _time_ms(lambda: pk.ppcg_block_coefficients(hf.handle, X.data_ptr(), Wb.data_ptr(), Pb.data_ptr(),
                                                       HX.data_ptr(), HW.data_ptr(), HP.data_ptr(), n, k, 1,
                                                       coef.data_ptr(), flags.data_ptr()), stream, 5)
    bflops = 18.0 * q * n * k              # per row and sub-block, both 3q x 3q Gram triangles: ~9 q^2 FMAs
    out["roofline_block_gram"] = {
        "kernel": f"block_gram_kernel + block_solve_kernel: 2 x (3q x 3q) Grams per sub-block, q={q}, {n} x {k}",
        "bound": "alu", "achieved": bflops / (ms_b / 1e3) / 1e12, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
        "frac": bflops / (ms_b / 1e3) / 1e12 / FP64_PEAK_TFLOPS, "traffic": None, "launch_ms": ms_b,
        "hbm_gbs": 48.0 * n * k / (ms_b / 1e3) / 1e9}
    Xu, Pu = X.clone(), Pb.clone()
    ms_u = _time_ms(lambda: pk.ppcg_block_update(hf.handle, Xu.data_ptr(), Wb.data_ptr(), Pu.data_ptr(), n, k, 1,
                                                 coef.data_ptr()), stream, 5)
    uflops = 2.0 * 3 * q * n * k
    ubytes = 40.0 * n * k
    out["roofline_block_update"] = {
        "kernel": f"block_update_kernel: P <- W C_W + P C_P; X <- X C_X + P, q={q}, {n} x {k}",
        "bound": "alu" if q >= 2 else "hbm", "achieved": uflops / (ms_u / 1e3) / 1e12, "peak": FP64_PEAK_TFLOPS,
        "unit": "TFLOP/s", "frac": uflops / (ms_u / 1e3) / 1e12 / FP64_PEAK_TFLOPS, "traffic": None,
        "launch_ms": ms_u, "hbm_gbs": ubytes / (ms_u / 1e3) / 1e9, "hbm_frac": ubytes / (ms_u / 1e3) / 1e9 / hbm}
    hf.close()
    return out


def run_e2e(pk, w, V, X0, steps, stream, form):
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
    opt.nbuf = w.nbuf
    prec, gm, orth = form
    opt.precision = {"fp64": 0, "mixed_tf32": 1, "mixed_bf16": 2}[prec]
    opt.fp64_gemm = {"fma": 0, "ozaki": 1}[gm]
    opt.orth = {"cholqr2": 0, "polar": 1}[orth]
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
    return {"value": el, "unit": "s", "h2d_bytes_per_step": 8 * n + es * n * (k + w.nbuf),
            "d2h_bytes_per_step": es * n * k + 16 * k,
            "steps": steps, "max_residual": float(np.max(res))}


if __name__ == "__main__":
    sys.exit(main())
