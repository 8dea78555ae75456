/*
 * ppcg_steps.h — the individual steps of Algorithm 3 (arXiv 1407.7506, Appendix A) as C-ABI calls.
 *
 * ppcg_solve strings these steps together; they are exported so that each step can be checked on its own
 * and reused (for instance inside an outer self-consistent-field loop, Section 6.2).
 *
 * Every call takes a handle from ppcg_create (it supplies the operator, the stream and the workspace), works on
 * DEVICE pointers only, enqueues its kernels on the handle's stream and returns without synchronising unless
 * stated. Blocks are column-major with the given leading dimension (>= n). Column counts are bounded by
 * kt = k + nbuf of the handle. Arguments out of range return PPCG_ERR_ARG and enqueue nothing.
 */
#ifndef PPCG_STEPS_H
#define PPCG_STEPS_H

#include "ppcg.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Operator application Y = A X (the "AX" kernel of Section 6; A = -Laplacian_h + diag(V), periodic),
 * m columns. X and Y must not overlap. */
PPCG_API ppcg_status ppcg_apply_operator(ppcg_handle h, const double* X, int64_t ldx, double* Y, int64_t ldy, int32_t m);

/* Gram matrix C = A^T B (the DGEMM + global sum of Section 6, used by steps 9, 10, 18, 20, 23):
 * A is n x ma, B is n x mb, C is ma x mb column-major with leading dimension ma. ma, mb <= kt. */
PPCG_API ppcg_status ppcg_gram(ppcg_handle h, const double* A, int64_t lda, const double* B, int64_t ldb, int32_t ma,
                      int32_t mb, double* C);

/* Steps 9-10: Y <- (I - X X^T) Y with X n x mx, Y n x my (mx, my <= kt). */
PPCG_API ppcg_status ppcg_project(ppcg_handle h, const double* X, int64_t ldx, int32_t mx, double* Y, int64_t ldy,
                         int32_t my);

/* Steps 18-19 (Section 5.5), applied twice (CholeskyQR2): X <- X R^{-1} with X^T X = R^T R, R upper triangular
 * with positive diagonal; in place on n x m (m <= kt). A relative pivot R_ii / sqrt(G_ii) < 1e-7 counts as a
 * breakdown and the shifted CholeskyQR3 of Fukaya et al. (2020) is used instead. Synchronises the stream.
 * *fallback (may be NULL) is set to 1 when the fallback ran. Returns PPCG_ERR_BREAKDOWN if that failed too. */
PPCG_API ppcg_status ppcg_cholqr2(ppcg_handle h, double* X, int64_t ldx, int32_t m, int32_t* fallback);

/* Symmetric eigensolver of the Rayleigh-Ritz step (steps 23-24, Section 5.6): M is m x m (leading dimension m,
 * the upper triangle is read), lambda receives the m eigenvalues ascending and C (m x m) the orthonormal
 * eigenvectors as columns. M, lambda and C are device buffers owned by the caller; C must not overlap M.
 * Routes, cheapest first: if no off-diagonal entry exceeds 1e-14 ||M||_F, the sorted diagonal and unit vectors.
 * If none exceeds 1e-4 ||M||_F, eigenvector refinement from the identity (Ogita and Aishima 2018), with clusters of
 * close eigenvalues solved as small eigenproblems; otherwise (or if that does not settle within 4 steps) the same
 * refinement started from the eigenvectors of a single-precision parallel Jacobi. A refinement is accepted once
 * every correction is <= 1e-8 and no cluster pair couples above 1e-14 ||M||_F; its eigenvalues are the Rayleigh
 * quotients of the final vectors. Parallel FP64 Jacobi is the fallback. The m x m products run on the FP64
 * tensor-core emulation when the handle was created with fp64_gemm = 1. Synchronises the stream; returns
 * PPCG_ERR_TIMEOUT if a bounded device wait gave up. */
PPCG_API ppcg_status ppcg_dense_eigh(ppcg_handle h, const double* M, int32_t m, double* lambda, double* C);

/* Steps 11-13 (eq. projev on S_j = [X_j, W_j, P_j], Section 5.1): for each of the s = ceil(k_act/q) sub-blocks
 * the q_j smallest eigenpairs of (S_j^T A S_j) c = theta (S_j^T S_j) c. X, W, P, HX = A X, HW = A W, HP = A P are
 * n x k_act (ld); has_p = 0 means P = [] (first iteration). coef receives, per sub-block j, a 3q x q
 * column-major matrix [C_X; C_W; C_P] at offset j*3q*q (C_P = 0 when P was dropped or absent); flags[j] is
 * 0 (ok), 1 (P dropped: Theorem 1 / Theorem 2 back-track) or 2 (kept X_j). coef and flags are device arrays. */
PPCG_API ppcg_status ppcg_block_coefficients(ppcg_handle h, const double* X, const double* W, const double* P,
                                    const double* HX, const double* HW, const double* HP, int64_t ld,
                                    int32_t k_act, int32_t has_p, double* coef, int32_t* flags);

/* Steps 14-15 for every sub-block: P_j <- W_j C_W + P_j C_P; X_j <- X_j C_X + P_j, in place, with coef as
 * produced by ppcg_block_coefficients. */
PPCG_API ppcg_status ppcg_block_update(ppcg_handle h, double* X, const double* W, double* P, int64_t ld, int32_t k_act,
                              int32_t has_p, const double* coef);

/* Steps 20/25 fused with step 8: R = HX - X M (M m x m, leading dimension m) or, when M is NULL,
 * R = HX - X diag(lam) (lam: device, m); then W = T R with T = diag(1/max(6/h^2 + V_p - sigma, delta)) and
 * colnorm2[c] = ||R[:, c]||^2 (device, m). X, HX, W are n x m (ld). */
PPCG_API ppcg_status ppcg_residual(ppcg_handle h, const double* X, const double* HX, int64_t ld, int32_t m, const double* M,
                          const double* lam, double sigma, double* W, double* colnorm2);

/* Adjoint of the solve with respect to the potential (Hellmann-Feynman): for E = sum_{i<k} lambda_i and
 * unit-norm eigenvectors x_i of A = -Laplacian_h + diag(V), dE/dV_p = sum_{i<k} x_i(p)^2 (the density), valid
 * when lambda_k < lambda_{k+1}. grad_V[p] = scale * sum_{c<k} |X[p, c]|^2 for X n x k (ld), as returned by
 * ppcg_solve (complex, interleaved re/im with ld counted in complex entries, for a PPCG_C128 handle); scale is
 * the upstream gradient of E. Device pointers; grad_V has n entries. */
PPCG_API ppcg_status ppcg_energy_gradient(ppcg_handle h, const double* X, int64_t ld, int32_t k, double scale,
                                          double* grad_V);

/* Check of the bounded device-side waits (the paper has no counterpart; failure handling of this library): runs a
 * cooperative kernel on the handle's stream in which one CTA never reaches the grid barrier that the others wait
 * at, with the wait bounded by spin_polls polls (>= 32; the solver's own barriers allow 2^22). The waiting CTAs
 * give up and return, so the call returns PPCG_ERR_TIMEOUT, the status a solve reports when one of its grid
 * barriers gives up, and the handle stays usable. Returns PPCG_OK only if the wait unexpectedly completed, and
 * PPCG_ERR_ARG for a NULL handle or spin_polls < 32. Synchronises the stream. */
PPCG_API ppcg_status ppcg_barrier_timeout_check(ppcg_handle h, int32_t spin_polls);

/* Gram matrix C = A^T B without a handle and without allocating any device memory. The paper has no
 * counterpart: this entry point exists for callers that cannot allocate (a fixed device-memory budget, an
 * application memory pool that forbids cudaMalloc, no ppcg handle). A is n x ma (lda >= n), B is n x mb
 * (ldb >= n), C is ma x mb with leading dimension ma; all device pointers. Runs on cuda_stream (NULL = legacy
 * default stream) and returns without synchronising.
 * Limit: ma * mb <= 1,048,576 (the partial sums use a static 8 MiB device array that every GPU loading this
 * library holds until the process exits); larger sizes return PPCG_ERR_ARG and enqueue nothing.
 * The first call on a device looks the array's device address up (cudaGetSymbolAddress), so make that first
 * call before any stream capture. All calls share the one array and nothing in it needs to start at zero, but
 * calls that overlap on the GPU (other streams, other threads) race on it: serialise them. */
PPCG_API ppcg_status ppcg_gram_noalloc(const double* A, int64_t lda, const double* B, int64_t ldb, int64_t n,
                                       int32_t ma, int32_t mb, double* C, void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* PPCG_STEPS_H */
