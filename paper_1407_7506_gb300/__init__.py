"""GB300 PPCG eigensolver (Vecharynski, Yang, Pask, arXiv 1407.7506) — Python binding of libppcg.so.

The binding only marshals arguments: every step of the solver runs in the library's sm_103a CUDA kernels
(C ABI in include/ppcg.h and include/ppcg_steps.h). PyTorch is used for device memory and streams only.
There is no CPU fallback: if libppcg.so is missing or no GPU is present the calls raise.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libppcg.so")

# status codes (ppcg_status)
PPCG_OK = 0
PPCG_ERR_ARG = 1
PPCG_ERR_CUDA = 2
PPCG_ERR_OOM = 3
PPCG_ERR_NOT_CONVERGED = 4
PPCG_ERR_BREAKDOWN = 5
PPCG_ERR_NUMERIC = 6
PPCG_ERR_TIMEOUT = 7
PPCG_ERR_UNSUPPORTED = 8
PHASES = ("AX", "GEMM", "BlockRR", "CholQR", "RR", "Precond", "Lock", "Other")

EXPORTS = ("ppcg_status_string", "ppcg_workspace_bytes", "ppcg_create", "ppcg_set_potential", "ppcg_solve",
           "ppcg_destroy", "ppcg_apply_operator", "ppcg_gram", "ppcg_project", "ppcg_cholqr2", "ppcg_dense_eigh",
           "ppcg_block_coefficients", "ppcg_block_update", "ppcg_residual", "ppcg_gram_noalloc",
           "ppcg_energy_gradient", "ppcg_solve_batched", "ppcg_autotune_sbsize", "ppcg_barrier_timeout_check")


class ppcg_operator(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32), ("h", ctypes.c_double),
                ("V", ctypes.c_void_p), ("theta", ctypes.c_double * 3), ("dtype", ctypes.c_int32)]


class ppcg_options(ctypes.Structure):
    _fields_ = [("maxiter", ctypes.c_int32), ("nbuf", ctypes.c_int32), ("no_lock", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("sigma_floor", ctypes.c_double), ("timing", ctypes.c_int32),
                ("history_cap", ctypes.c_int32), ("history", ctypes.POINTER(ctypes.c_double)),
                ("fp64_gemm", ctypes.c_int32), ("orth", ctypes.c_int32), ("orth_skip_tol", ctypes.c_double),
                ("reserved", ctypes.c_int32 * 2)]


class ppcg_stats(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32), ("n_rr", ctypes.c_int32), ("n_locked", ctypes.c_int32),
                ("n_drop_p", ctypes.c_int32), ("n_stall", ctypes.c_int32), ("n_cholqr_fallback", ctypes.c_int32),
                ("n_early_rr", ctypes.c_int32), ("converged", ctypes.c_int32), ("history_len", ctypes.c_int32),
                ("jacobi_sweeps_max", ctypes.c_int32), ("kernel_launches", ctypes.c_int64), ("t_phase_ms", ctypes.c_double * 8),
                ("max_res", ctypes.c_double), ("n_orth_skip", ctypes.c_int32), ("n_polar", ctypes.c_int32),
                ("n_eig_diagonal", ctypes.c_int32), ("n_eig_refined", ctypes.c_int32), ("n_eig_mixed", ctypes.c_int32),
                ("n_rr_unit", ctypes.c_int32)]

    def as_dict(self):
        d = {f: getattr(self, f) for f, _ in self._fields_ if f != "t_phase_ms"}
        d["t_phase_ms"] = dict(zip(PHASES, list(self.t_phase_ms)))
        return d


class ppcg_batch_item(ctypes.Structure):
    _fields_ = [("h", ctypes.c_void_p), ("X0", ctypes.c_void_p), ("tol", ctypes.c_double),
                ("lam", ctypes.c_void_p), ("X", ctypes.c_void_p), ("resnorm", ctypes.c_void_p),
                ("stats", ctypes.POINTER(ppcg_stats)), ("status", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("time_ms", ctypes.c_double)]


class PPCGError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        super().__init__(f"{where}: {ppcg_status_string(status)}")


_lib = None
_vp, _i32, _i64, _d, _sz = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_size_t


def lib():
    """Load libppcg.so (built in-tree by paper_1407_7506_gb300.build); raise if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is not built; run `python -m paper_1407_7506_gb300.build`")
        L = ctypes.CDLL(LIB_PATH)
        P = ctypes.POINTER
        sig = {
            "ppcg_status_string": (ctypes.c_char_p, [_i32]),
            "ppcg_workspace_bytes": (_i32, [P(ppcg_operator), _i64, _i32, _i32, P(ppcg_options), P(_sz)]),
            "ppcg_create": (_i32, [P(ppcg_operator), _i64, _i32, _i32, _i32, P(ppcg_options), _vp, _vp, _sz,
                                   P(_vp)]),
            "ppcg_set_potential": (_i32, [_vp, _vp]),
            "ppcg_solve": (_i32, [_vp, _vp, _d, _vp, _vp, _vp, P(ppcg_stats)]),
            "ppcg_destroy": (_i32, [_vp]),
            "ppcg_apply_operator": (_i32, [_vp, _vp, _i64, _vp, _i64, _i32]),
            "ppcg_gram": (_i32, [_vp, _vp, _i64, _vp, _i64, _i32, _i32, _vp]),
            "ppcg_project": (_i32, [_vp, _vp, _i64, _i32, _vp, _i64, _i32]),
            "ppcg_cholqr2": (_i32, [_vp, _vp, _i64, _i32, P(_i32)]),
            "ppcg_dense_eigh": (_i32, [_vp, _vp, _i32, _vp, _vp]),
            "ppcg_block_coefficients": (_i32, [_vp, _vp, _vp, _vp, _vp, _vp, _vp, _i64, _i32, _i32, _vp, _vp]),
            "ppcg_block_update": (_i32, [_vp, _vp, _vp, _vp, _i64, _i32, _i32, _vp]),
            "ppcg_residual": (_i32, [_vp, _vp, _vp, _i64, _i32, _vp, _vp, _d, _vp, _vp]),
            "ppcg_gram_noalloc": (_i32, [_vp, _i64, _vp, _i64, _i64, _i32, _i32, _vp, _vp]),
            "ppcg_energy_gradient": (_i32, [_vp, _vp, _i64, _i32, _d, _vp]),
            "ppcg_solve_batched": (_i32, [P(ppcg_batch_item), _i32, _i32]),
            "ppcg_autotune_sbsize": (_i32, [P(ppcg_operator), _i64, _i32, _i32, P(ppcg_options), _vp, _d,
                                            P(_i32), _i32, _vp, P(_i32), P(_d)]),
            "ppcg_barrier_timeout_check": (_i32, [_vp, _i32]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(status, where):
    if status != PPCG_OK:
        raise PPCGError(status, where)


# ------------------------------------------------------------------------------ thin wrappers, same names
def ppcg_status_string(status: int) -> str:
    return lib().ppcg_status_string(int(status)).decode()


def ppcg_workspace_bytes(op, n, k, sbsize, opt=None) -> int:
    out = _sz(0)
    _check(lib().ppcg_workspace_bytes(ctypes.byref(op), n, k, sbsize, ctypes.byref(opt) if opt else None,
                                      ctypes.byref(out)), "ppcg_workspace_bytes")
    return out.value


def ppcg_create(op, n, k, sbsize, rr_period, opt=None, stream=0, workspace=0, workspace_bytes=0):
    h = _vp(0)
    _check(lib().ppcg_create(ctypes.byref(op), n, k, sbsize, rr_period, ctypes.byref(opt) if opt else None,
                             stream, workspace, workspace_bytes, ctypes.byref(h)), "ppcg_create")
    return h.value


def ppcg_set_potential(h, V_ptr):
    _check(lib().ppcg_set_potential(h, V_ptr), "ppcg_set_potential")


def ppcg_solve(h, X0_ptr, tol, lam_ptr, X_ptr, res_ptr, stats=None):
    """Returns the status (PPCG_OK or PPCG_ERR_NOT_CONVERGED); other statuses raise."""
    st = lib().ppcg_solve(h, X0_ptr, tol, lam_ptr, X_ptr, res_ptr, ctypes.byref(stats) if stats else None)
    if st not in (PPCG_OK, PPCG_ERR_NOT_CONVERGED):
        raise PPCGError(st, "ppcg_solve")
    return st


def ppcg_destroy(h):
    _check(lib().ppcg_destroy(h), "ppcg_destroy")


def ppcg_apply_operator(h, X, ldx, Y, ldy, m):
    _check(lib().ppcg_apply_operator(h, X, ldx, Y, ldy, m), "ppcg_apply_operator")


def ppcg_gram(h, A, lda, B, ldb, ma, mb, C):
    _check(lib().ppcg_gram(h, A, lda, B, ldb, ma, mb, C), "ppcg_gram")


def ppcg_project(h, X, ldx, mx, Y, ldy, my):
    _check(lib().ppcg_project(h, X, ldx, mx, Y, ldy, my), "ppcg_project")


def ppcg_cholqr2(h, X, ldx, m):
    fb = _i32(0)
    _check(lib().ppcg_cholqr2(h, X, ldx, m, ctypes.byref(fb)), "ppcg_cholqr2")
    return fb.value


def ppcg_dense_eigh(h, M, m, lam, C):
    _check(lib().ppcg_dense_eigh(h, M, m, lam, C), "ppcg_dense_eigh")


def ppcg_block_coefficients(h, X, W, P, HX, HW, HP, ld, k_act, has_p, coef, flags):
    _check(lib().ppcg_block_coefficients(h, X, W, P, HX, HW, HP, ld, k_act, has_p, coef, flags),
           "ppcg_block_coefficients")


def ppcg_block_update(h, X, W, P, ld, k_act, has_p, coef):
    _check(lib().ppcg_block_update(h, X, W, P, ld, k_act, has_p, coef), "ppcg_block_update")


def ppcg_residual(h, X, HX, ld, m, M, lam, sigma, W, colnorm2):
    _check(lib().ppcg_residual(h, X, HX, ld, m, M, lam, sigma, W, colnorm2), "ppcg_residual")


def ppcg_energy_gradient(h, X, ld, k, scale, grad_V):
    _check(lib().ppcg_energy_gradient(h, X, ld, k, scale, grad_V), "ppcg_energy_gradient")


def ppcg_barrier_timeout_check(h, spin_polls):
    """Returns the status (PPCG_ERR_TIMEOUT when the bounded barrier wait gave up as designed)."""
    return lib().ppcg_barrier_timeout_check(h, spin_polls)


def ppcg_gram_noalloc(A, lda, B, ldb, n, ma, mb, C, stream=0):
    """C = A^T B without a handle and without device allocation (static scratch; ma * mb <= 2**20)."""
    _check(lib().ppcg_gram_noalloc(A, lda, B, ldb, n, ma, mb, C, stream), "ppcg_gram_noalloc")




def ppcg_solve_batched(items, max_concurrent=0):
    """items: a ctypes array of ppcg_batch_item. Returns the batch status (PPCG_OK or PPCG_ERR_NOT_CONVERGED);
    other statuses raise. Per-item status and time_ms are written into the items."""
    st = lib().ppcg_solve_batched(items, len(items), max_concurrent)
    if st not in (PPCG_OK, PPCG_ERR_NOT_CONVERGED):
        raise PPCGError(st, "ppcg_solve_batched")
    return st


def ppcg_autotune_sbsize(op, n, k, rr_period, opt, X0_ptr, tol, candidates, stream=0):
    """Returns (best sbsize, list of per-candidate times in ms, negative where invalid or not converged)."""
    cand = (_i32 * len(candidates))(*candidates)
    times = (_d * len(candidates))()
    best = _i32(0)
    _check(lib().ppcg_autotune_sbsize(ctypes.byref(op), n, k, rr_period, ctypes.byref(opt) if opt else None, X0_ptr,
                                      tol, cand, len(candidates), stream, ctypes.byref(best), times),
           "ppcg_autotune_sbsize")
    return best.value, list(times)


from .solver import Solver, BatchSolver  # noqa: E402,F401
from .autograd import smallest_eigsum  # noqa: E402,F401
