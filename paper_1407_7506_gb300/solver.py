"""Convenience wrapper: a PPCG solver handle whose memory and stream come from PyTorch.

Arguments are marshalled to the C ABI; all computation happens in libppcg.so.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import (PPCG_ERR_NOT_CONVERGED, PPCG_OK, ppcg_batch_item, ppcg_create, ppcg_destroy, ppcg_operator,
               ppcg_options, ppcg_solve, ppcg_solve_batched, ppcg_stats, ppcg_workspace_bytes, ppcg_set_potential)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


class Solver:
    """k smallest eigenpairs of A = -Laplacian_h + diag(V) on an N^3 (or nx x ny x nz) periodic grid.

    dtype "c128" with a Bloch twist theta gives the complex Hermitian operator (start blocks and vectors complex).
    V: torch tensor (any device) or numpy array of n doubles. The workspace is a torch uint8 CUDA tensor owned
    by this object; the stream is torch's current stream unless one is given.
    """

    def __init__(self, V, grid, k, sbsize, rr_period=5, h=1.0, nbuf=0, maxiter=0, lock=True, timing=False,
                 sigma_floor=0.0, device="cuda", stream=None, history=0, precision="fp64", fp64_gemm="fma",
                 orth="cholqr2", orth_skip_tol=0.0, dtype="f64", theta=(0.0, 0.0, 0.0)):
        if not torch.cuda.is_available():
            raise RuntimeError("the PPCG library needs a CUDA GPU; no CPU fallback exists")
        nx, ny, nz = (grid, grid, grid) if np.isscalar(grid) else tuple(grid)
        self.n = nx * ny * nz
        self.k, self.nbuf, self.sbsize, self.rr_period = k, nbuf, sbsize, rr_period
        self.device = torch.device(device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self._V = torch.as_tensor(np.asarray(V) if not torch.is_tensor(V) else V, dtype=torch.float64)
        self._V = self._V.to(self.device).contiguous()
        self.cplx = {"f64": False, "c128": True}[dtype]
        self.dtype = torch.complex128 if self.cplx else torch.float64
        self.op = ppcg_operator(nx, ny, nz, h, self._V.data_ptr(), (ctypes.c_double * 3)(*theta), 1 if self.cplx else 0)
        self.opt = ppcg_options()
        self.opt.maxiter = maxiter
        self.opt.nbuf = nbuf
        self.opt.no_lock = 0 if lock else 1
        self.opt.timing = 1 if timing else 0
        self.opt.sigma_floor = sigma_floor
        self.opt.precision = {"fp64": 0, "mixed_tf32": 1, "mixed": 1, "mixed_bf16": 2}[precision]
        self.opt.fp64_gemm = {"fma": 0, "ozaki": 1}[fp64_gemm]
        self.opt.orth = {"cholqr2": 0, "polar": 1}[orth]
        self.opt.orth_skip_tol = orth_skip_tol
        self._hist = np.zeros(6 * max(history, 1))
        if history:
            self.opt.history_cap = history
            self.opt.history = self._hist.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        nbytes = ppcg_workspace_bytes(self.op, self.n, k, sbsize, self.opt)
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        self.handle = ppcg_create(self.op, self.n, k, sbsize, rr_period, self.opt, self.stream.cuda_stream,
                                  self.workspace.data_ptr(), nbytes)

    def set_potential(self, V):
        V = torch.as_tensor(V, dtype=torch.float64).contiguous()
        self._V = V                      # keep alive across the (synchronous) copy
        ppcg_set_potential(self.handle, V.data_ptr())

    def solve(self, X0, tol=1e-8, out=None):
        """X0: n x (k + nbuf) column-major (torch tensor of shape (k+nbuf, n) row-major, or numpy Fortran
        array (n, k+nbuf)). Returns (lam numpy, X torch (k, n) row-major = columns, res numpy, stats dict)."""
        if isinstance(X0, np.ndarray):
            X0t = torch.from_numpy(np.ascontiguousarray(X0.T)).to(self.device)
        else:
            X0t = X0
        assert X0t.shape == (self.k + self.nbuf, self.n) and X0t.dtype == self.dtype and X0t.is_contiguous()
        X = out if out is not None else torch.empty((self.k, self.n), dtype=self.dtype, device=self.device)
        lam = np.zeros(self.k)
        res = np.zeros(self.k)
        st = ppcg_stats()
        status = ppcg_solve(self.handle, X0t.data_ptr(), tol, lam.ctypes.data, X.data_ptr(), res.ctypes.data, st)
        d = st.as_dict()
        d["status"] = "ok" if status == PPCG_OK else ("not_converged" if status == PPCG_ERR_NOT_CONVERGED else status)
        d["history"] = self._hist[:6 * d["history_len"]].reshape(-1, 6).copy()
        return lam, X, res, d

    def close(self):
        if getattr(self, "handle", None):
            ppcg_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _status_name(status):
    return "ok" if status == PPCG_OK else ("not_converged" if status == PPCG_ERR_NOT_CONVERGED else status)


class BatchSolver:
    """Independent problems of uneven size solved concurrently through ppcg_solve_batched.

    problems: list of dicts with keys V, grid, k, sbsize and optionally rr_period. Each problem gets its own
    Solver (handle, workspace) on its own CUDA stream; solver_kw are passed to every Solver.
    """

    def __init__(self, problems, device="cuda", **solver_kw):
        self.device = torch.device(device)
        self.solvers = []
        for p in problems:
            st = torch.cuda.Stream(device=self.device)
            with torch.cuda.stream(st):
                self.solvers.append(Solver(p["V"], p["grid"], p["k"], p["sbsize"], rr_period=p.get("rr_period", 5),
                                           device=device, stream=st, **solver_kw))

    def solve(self, X0s, tol=1e-8, max_concurrent=0):
        """X0s: one start block per problem (as for Solver.solve). Returns (results, batch_status): results is a
        list of (lam, X, res, stats) with stats["time_ms"] the problem's own wall time."""
        n = len(self.solvers)
        items = (ppcg_batch_item * n)()
        keep = []
        for i, (s, X0) in enumerate(zip(self.solvers, X0s)):
            with torch.cuda.stream(s.stream):
                if isinstance(X0, np.ndarray):
                    X0t = torch.from_numpy(np.ascontiguousarray(X0.T)).to(self.device)
                else:
                    X0t = X0
                X = torch.empty((s.k, s.n), dtype=s.dtype, device=self.device)
            assert X0t.shape == (s.k + s.nbuf, s.n) and X0t.dtype == s.dtype and X0t.is_contiguous()
            lam, res, st = np.zeros(s.k), np.zeros(s.k), ppcg_stats()
            items[i].h = s.handle
            items[i].X0 = X0t.data_ptr()
            items[i].tol = tol
            items[i].lam = lam.ctypes.data
            items[i].X = X.data_ptr()
            items[i].resnorm = res.ctypes.data
            items[i].stats = ctypes.pointer(st)
            keep.append((X0t, X, lam, res, st))
        for s in self.solvers:
            s.stream.synchronize()                       # start blocks are on the device before the solves run
        status = ppcg_solve_batched(items, max_concurrent)
        out = []
        for i, (X0t, X, lam, res, st) in enumerate(keep):
            d = st.as_dict()
            d["status"] = _status_name(items[i].status)
            d["time_ms"] = items[i].time_ms
            out.append((lam, X, res, d))
        return out, _status_name(status)

    def close(self):
        for s in self.solvers:
            s.close()
