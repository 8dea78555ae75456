/*
 * ppcg.h — C ABI of the GB300 PPCG eigensolver.
 *
 * Computes the k algebraically smallest eigenpairs of A = -Laplacian_h + diag(V) (7-point stencil on a periodic
 * nx x ny x nz grid) with the Projected Preconditioned Conjugate Gradient method of Vecharynski, Yang and Pask
 * (arXiv 1407.7506): the trace-minimisation problem of Section 2 (eq. tracemin), iterated as Algorithm 3
 * (Appendix A) with sub-block size sbsize (Section 5.1), Rayleigh-Ritz every rr_period iterations (Section 5.6),
 * soft locking (Section 5.7), buffer vectors (Section 5.3) and Cholesky QR orthonormalisation (Section 5.5).
 *
 * Conventions
 *   - A grid function is n = nx*ny*nz doubles, linear index p = i + nx*j + nx*ny*l (x fastest).
 *   - A block of m vectors is column-major with leading dimension ld >= n (column c starts at c*ld).
 *   - Every call runs on the handle's CUDA stream. ppcg_solve is synchronous (it reads two scalars per iteration
 *     to steer the loop); a handle is not thread-safe.
 *   - All functions return a ppcg_status; no function aborts the process or prints.
 *   - Device work is done by the library's own sm_103a kernels; there is no CPU fallback. If the library was
 *     built without a usable GPU the calls return PPCG_ERR_CUDA.
 */
#ifndef PPCG_H
#define PPCG_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define PPCG_API __attribute__((visibility("default")))
#else
#define PPCG_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  PPCG_OK = 0,
  PPCG_ERR_ARG = 1,            /* invalid argument (sizes, null pointers, n != nx*ny*nz, ...) */
  PPCG_ERR_CUDA = 2,           /* a CUDA runtime call failed (no device, launch failure, ...) */
  PPCG_ERR_OOM = 3,            /* workspace allocation failed or the caller's workspace is too small */
  PPCG_ERR_NOT_CONVERGED = 4,  /* maxiter reached; outputs hold the last Ritz pairs (Alg. 3 step 32) */
  PPCG_ERR_BREAKDOWN = 5,      /* orthonormalisation failed even with shifted CholeskyQR3 */
  PPCG_ERR_NUMERIC = 6,        /* a NaN/Inf appeared in a residual norm */
  PPCG_ERR_TIMEOUT = 7,        /* a bounded device-side wait (grid barrier) gave up */
  PPCG_ERR_UNSUPPORTED = 8     /* option valid in the paper but not provided by this library */
} ppcg_status;

typedef enum { PPCG_R64 = 0, PPCG_C128 = 1 } ppcg_dtype;

/* Arithmetic of the GEMMs whose rounding only perturbs search directions: the projections of W and P (Alg. 3
 * steps 9-10) and the Gram of the first CholeskyQR pass (step 18). PPCG_FP64: FP64. PPCG_MIXED_TF32 /
 * PPCG_MIXED_BF16: tcgen05 tensor cores with TF32 / BF16 operands (converted from the FP64 blocks, round to nearest)
 * and FP32 accumulation. Everything else (the sub-block Grams, step 20, the second CholeskyQR pass, the stencil, the
 * small eigensolves and the Rayleigh-Ritz step) stays FP64 in every form. */
typedef enum { PPCG_FP64 = 0, PPCG_MIXED_TF32 = 1, PPCG_MIXED_BF16 = 2 } ppcg_precision;

/* The operator A = -Laplacian_h + diag(V). V may be a host or a device pointer; it is copied at create time
 * (ppcg_set_potential replaces it). theta is the Bloch twist per axis (0 = periodic). */
typedef struct {
  int32_t nx, ny, nz;
  double h;
  const double* V;
  double theta[3];
  int32_t dtype; /* ppcg_dtype: PPCG_R64 (theta must be 0) or PPCG_C128 (complex Hermitian, Bloch twist theta);
                    a C128 problem is solved in its real form [[Re A, -Im A], [Im A, Re A]] of order 2n, whose
                    eigenvalues are those of A, each twice; X0 and X are then complex (interleaved re/im), and
                    the step entry points of ppcg_steps.h work on real-form blocks of 2n rows */
} ppcg_operator;

/* Options; a zero-initialised struct gives the defaults in brackets. */
typedef struct {
  int32_t maxiter;      /* [0 -> 500] iterations of the loop of Algorithm 3 */
  int32_t nbuf;         /* [0] buffer vectors (Section 5.3); X0 then has k + nbuf columns */
  int32_t no_lock;      /* [0] 1 disables soft locking (Section 5.7) */
  int32_t precision;    /* [PPCG_FP64] ppcg_precision */
  double sigma_floor;   /* [0 -> 0.1/h^2] floor delta of the preconditioner diagonal, see ppcg_solve */
  int32_t timing;       /* [0] 1 records per-phase device times into ppcg_stats.t_phase_ms */
  int32_t history_cap;  /* [0] capacity (entries) of history */
  double* history;      /* [NULL] host array of 6 * history_cap doubles; entry i = {iteration, kind,
                           value, trace, k_act, t_ms}: kind 0 = plain step (value = ||W||_F over the wanted
                           columns), kind 1 = Rayleigh-Ritz step (value = max_i r_i, trace = sum of the k Ritz
                           values); k_act = active (unlocked) columns the iteration worked on (k + nbuf for
                           iteration 0); t_ms = milliseconds since the solve began, taken when the step's norms
                           reached the host */
  int32_t fp64_gemm;    /* [0] how the FP64 n x k GEMMs run: 0 = FP64 FMA pipe, 1 = FP64-accurate emulation on
                           the BF16 tensor cores (error-free splitting into 8 digit slices, Ozaki scheme) */
  int32_t orth;         /* [0] step 18 (Section 5.5): 0 = CholeskyQR2; 1 = polar X <- X (X^T X)^{-1/2} by the
                           series of (I + Y)^{-1/2}, Y = X^T X - I, with the fewest terms (at most 8) whose first
                           omitted term nu^{t+1} |c_{t+1}| is below the FP64 unit roundoff, nu = ||Y||_F; when no
                           such t exists CholeskyQR2 runs instead */
  double orth_skip_tol; /* [0] skip step 18 when ||X^T X - I||_F <= orth_skip_tol (Section 5.5); 0 never skips */
  int32_t reserved[2];
} ppcg_options;

/* Phases of the per-phase times, after the paper's profile categories (Tables Li318prof, Siprof) */
enum { PPCG_T_AX = 0, PPCG_T_GEMM = 1, PPCG_T_BLOCKRR = 2, PPCG_T_CHOLQR = 3, PPCG_T_RR = 4, PPCG_T_PRECOND = 5,
       PPCG_T_LOCK = 6, PPCG_T_OTHER = 7 };

typedef struct {
  int32_t iters;              /* iterations of the main loop */
  int32_t n_rr;               /* Rayleigh-Ritz steps (including the initial one and the final one) */
  int32_t n_locked;           /* locked columns at exit */
  int32_t n_drop_p;           /* sub-blocks redone without P (Theorem 1 / Theorem 2 back-track, Section 3) */
  int32_t n_stall;            /* sub-blocks that kept X_j because even the [X_j, W_j] problem broke down */
  int32_t n_cholqr_fallback;  /* shifted CholeskyQR3 fallbacks */
  int32_t n_early_rr;         /* Rayleigh-Ritz steps forced by ||W||_F <= tol */
  int32_t converged;          /* 1 if max residual <= tol */
  int32_t history_len;        /* entries written to options.history */
  int32_t jacobi_sweeps_max;  /* most Jacobi sweeps one Rayleigh-Ritz eigensolve needed */
  int64_t kernel_launches;    /* device kernels this solve launched */
  double t_phase_ms[8];       /* per-phase device time (ms) when options.timing = 1 */
  double max_res;             /* max_i ||A x_i - lambda_i x_i|| over the k returned pairs */
  int32_t n_orth_skip;        /* plain steps whose orthonormalisation was skipped (options.orth_skip_tol) */
  int32_t n_polar;            /* plain steps orthonormalised by the polar series (options.orth = 1) */
  int32_t n_eig_diagonal;     /* Rayleigh-Ritz eigensolves whose matrix was already diagonal (no rotation needed) */
  int32_t n_eig_refined;      /* Rayleigh-Ritz eigensolves finished by eigenvector refinement from the identity */
  int32_t n_eig_mixed;        /* Rayleigh-Ritz eigensolves by single-precision Jacobi + FP64 eigenvector refinement
                                 (the others that are not diagonal, refined or mixed took FP64 Jacobi) */
  int32_t n_rr_unit;          /* Rayleigh-Ritz steps with locked columns whose eigenvectors were unit vectors: the
                                 locked columns and H applied to them were copied, only the active ones computed */
} ppcg_stats;

typedef struct ppcg_ctx* ppcg_handle;

/* Human-readable name of a status code (static storage). */
PPCG_API const char* ppcg_status_string(ppcg_status s);

/* Bytes of device workspace that ppcg_create needs for these sizes (so a caller can provide it). */
PPCG_API ppcg_status ppcg_workspace_bytes(const ppcg_operator* op, int64_t n, int32_t k, int32_t sbsize,
                                 const ppcg_options* opt, size_t* bytes);

/*
 * Create a solver for the k smallest eigenpairs of op (Algorithm 3 inputs: A, T, rr_period, sbsize, nbuf).
 *   n           must equal nx*ny*nz
 *   k           1 <= k, k + nbuf <= n/2
 *   sbsize      sub-block size q of Section 5.1, 1 <= sbsize <= min(k + nbuf, 16) (8 for PPCG_C128)
 *   rr_period   Rayleigh-Ritz period (Section 5.6), >= 1
 *   opt         may be NULL (defaults)
 *   cuda_stream a cudaStream_t (NULL = legacy default stream)
 *   workspace   device memory of at least ppcg_workspace_bytes, owned by the caller and kept alive until
 *               ppcg_destroy; NULL lets the library allocate (and free) it.
 * On success *out holds a handle that the caller releases with ppcg_destroy.
 */
PPCG_API ppcg_status ppcg_create(const ppcg_operator* op, int64_t n, int32_t k, int32_t sbsize, int32_t rr_period,
                        const ppcg_options* opt, void* cuda_stream, void* workspace, size_t workspace_bytes,
                        ppcg_handle* out);

/* Replace V (n doubles, host or device) without reallocating (e.g. successive SCF steps, Section 6.2). */
PPCG_API ppcg_status ppcg_set_potential(ppcg_handle h, const double* V);

/*
 * Run Algorithm 3 from the starting block X0 until every one of the first k Ritz pairs has residual
 * ||A x_i - lambda_i x_i||_2 <= tol at a Rayleigh-Ritz step, or maxiter iterations.
 *   X0      n x (k + nbuf), ld = n, host or device memory (need not be orthonormal; it is orthonormalised);
 *           complex (interleaved re/im) for a PPCG_C128 operator, and so is X
 *   lambda  host, k doubles: Ritz values, ascending
 *   X       n x k, ld = n, host or device memory (may alias X0): Ritz vectors, unit norm, with the entry of
 *           largest modulus (lowest index on ties) real positive
 *   resnorm host, k doubles: ||A x_i - lambda_i x_i||_2 recomputed on the returned pairs (may be NULL)
 *   stats   may be NULL
 * The preconditioner is T = diag(1 / max(6/h^2 + V_p - sigma, delta)), sigma the smallest Ritz value of the
 * latest Rayleigh-Ritz step (one is taken on orth(X0) before the first iteration).
 * Returns PPCG_OK, or PPCG_ERR_NOT_CONVERGED with the last Ritz pairs in the outputs.
 */
PPCG_API ppcg_status ppcg_solve(ppcg_handle h, const double* X0, double tol, double* lambda, double* X, double* resnorm,
                       ppcg_stats* stats);

/* Release the handle (and the workspace if the library allocated it). NULL is accepted. */
PPCG_API ppcg_status ppcg_destroy(ppcg_handle h);

/*
 * Many independent eigenproblems (uneven n and k, each with its own handle) solved concurrently, for workloads
 * of many small Hamiltonians such as the per-k-point or per-system solves around Section 6. Each item is one
 * ppcg_solve call; the library runs up to max_concurrent of them at once on native threads, each on its own
 * handle's stream (give every handle its own stream, or they serialise). Cooperative grid-barrier kernels of
 * different items are ordered one after another on the device; everything else overlaps.
 *   items           count entries; h, X0, tol, lambda, X, resnorm, stats as in ppcg_solve (stats may be NULL);
 *                   status and time_ms are written per item (time_ms: host wall time of that solve)
 *   max_concurrent  <= 0 means min(count, 16)
 * Returns PPCG_OK when every item returned PPCG_OK, otherwise the first non-OK item status in item order
 * (PPCG_ERR_ARG for a NULL items array, a NULL handle or count < 0). Items must use distinct handles.
 */
typedef struct {
  ppcg_handle h;
  const double* X0;
  double tol;
  double* lambda;
  double* X;
  double* resnorm;
  ppcg_stats* stats;
  int32_t status;     /* out: ppcg_status of this item's solve */
  int32_t reserved;
  double time_ms;     /* out */
} ppcg_batch_item;

PPCG_API ppcg_status ppcg_solve_batched(ppcg_batch_item* items, int32_t count, int32_t max_concurrent);

/*
 * Autotuner for the sub-block size q (Section 5.1; the paper's sbsize experiments in Section 6.1 show that the
 * best q depends on the problem). For each candidate q in candidates[0..ncand) with 1 <= q <= min(k + nbuf, 16)
 * it creates a solver (library-allocated workspace), solves from X0 to tol on cuda_stream and times the solve
 * with CUDA events; time_ms[i] receives the time (a negative value for a candidate that was invalid or did not
 * converge) and *best the fastest converged q. Returns PPCG_OK if at least one candidate converged, else the
 * status of the last candidate tried.
 */
PPCG_API ppcg_status ppcg_autotune_sbsize(const ppcg_operator* op, int64_t n, int32_t k, int32_t rr_period,
                                          const ppcg_options* opt, const double* X0, double tol,
                                          const int32_t* candidates, int32_t ncand, void* cuda_stream,
                                          int32_t* best, double* time_ms);

#ifdef __cplusplus
}
#endif

#endif /* PPCG_H */
