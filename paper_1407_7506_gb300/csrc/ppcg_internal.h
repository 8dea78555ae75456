// Internal declarations shared by the CUDA translation units of the PPCG library.
#pragma once

#include <cuda_runtime.h>
#include <cstddef>
#include <cstdint>

namespace ppcg {

// ---------------------------------------------------------------------------------------------- constants
// Numerical thresholds of the method (shared by every kernel that takes the decision).
constexpr double kPivotTol = 1e-7;      // sub-block problems: smallest Cholesky diagonal of unit-diagonal S*S
constexpr double kAlphaTol = 1e-12;     // Theorem 1: smallest singular value of C_X
constexpr double kCholPivotTol = 1e-7;  // CholQR: smallest relative pivot R_ii / sqrt(G_ii)
constexpr double kJacobiTol = 1e-14;    // k x k Jacobi: rotate while |a_pq| > kJacobiTol * ||A||_F; an off-diagonal
                                        // left below that adds < ~1e-12 to a Ritz residual (tol is 1e-8)
constexpr double kJacobiTolSmall = 1e-16;  // sub-block warp Jacobi
constexpr int kJacobiMaxSweeps = 60;
constexpr double kRefineTau = 1e-4;      // refine from the identity when max |M_ij| (i != j) <= kRefineTau ||M||_F
constexpr int kRefineSteps = 8;          // refinement steps before falling back to Jacobi (the correction roughly
                                         // squares per step: from an FP32 Jacobi start, 1e-1 .. 1e-2 takes 5-6)
constexpr double kRefineAccept = 1e-8;   // accept a refinement step whose largest |E_ij| (i != j) is at most this
constexpr double kJacobiTol32 = 3e-7;    // single-precision Jacobi (start of the refinement): rotate while
                                         // |a_pq| > kJacobiTol32 ||A||_F
constexpr int kJacobiMaxSweeps32 = 8;     // then the refinement takes over (a random 1074 x 1074 matrix is the
                                          // slowest case: 8 sweeps leave corrections the refinement settles)
constexpr double kClusterGap = 4.0;      // refinement: eigenvalues closer than kClusterGap x the largest coupling
                                         // |S_ij + lam_j R_ij| form a cluster, solved as one small eigenproblem
constexpr double kClusterFloor = 1e-7;   // ... and always those closer than kClusterFloor ||M||_F: there rounding in
                                         // S (~1e-16 ||M|| sqrt(m)) would give first-order coefficients above
                                         // kRefineAccept although the pair's vectors are determined only up to it
constexpr int kMaxCluster = 48;          // largest cluster solved in shared memory (beyond it: FP64 Jacobi)
constexpr int kPolarMaxTerms = 8;        // most series terms of the polar orthonormalisation
constexpr int kMaxSbsize = 16;          // 3q <= 48 fits the warp-level sub-block solver

// Error-flag bits written by kernels into the handle's device flag word.
enum : int { kFlagCholBreakdown = 1, kFlagTimeout = 2, kFlagJacobiNoConv = 4 };

__host__ __device__ inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

// Process-wide count of kernels launched by this library (reported per solve in ppcg_stats).
void count_launch(int n = 1);
long long launch_count();

// ---------------------------------------------------------------------------------------------- operator
struct Grid {
  int nx, ny, nz;
  double inv_h2;
  int cplx;          // 1: complex Bloch operator applied in the real form [u; v] (columns of 2 nx ny nz)
  double ct[3], st[3];   // cos and sin of the Bloch twist per axis
};

// Y[:, c] = A X[:, c] for c < m; dg = 6/h^2 + V (n doubles).
cudaError_t stencil_apply(const Grid& g, const double* dg, const double* X, int64_t ldx, double* Y, int64_t ldy,
                          int m, cudaStream_t s);

// ---------------------------------------------------------------------------------------------- FP64 GEMMs
// Number of doubles of split-K partial storage used by gram() for these sizes.
int gram_splits(int64_t n, int ma, int mb, size_t part_capacity);
// C (ma x mb, ldc) = A^T B, reduction over n rows; symmetric = (A == B, ma == mb): only upper tiles computed
// and mirrored so that C is exactly symmetric.
cudaError_t gram(const double* A, int64_t lda, const double* B, int64_t ldb, int64_t n, int ma, int mb, double* C,
                 int ldc, bool symmetric, double* part, size_t part_capacity, cudaStream_t s);

enum class Epi : int { Store = 0, Sub = 1, Residual = 2 };

// C = op(A) B (m x p, K = kdim; op(A) = A^T when trans_a) for small square-ish operands, split over K with a
// deterministic reduction; part holds the split partials (part_capacity doubles).
cudaError_t small_gemm(bool trans_a, const double* A, int64_t lda, const double* B, int64_t ldb, int m, int p,
                       int kdim, double* C, int ldc, double* part, size_t part_capacity, cudaStream_t s);
struct ResidualArgs {
  const double* dg;     // 6/h^2 + V
  double sigma;         // preconditioner shift
  double delta;         // preconditioner floor
  double* norm_part;    // [row tiles][p] partial column norms^2
  const double* tinv;   // 1 / max(dg - sigma, delta) per row, precomputed (may be NULL: formed in the kernel)
};
// tinv[r] = 1 / max(dg[r] - sigma, delta): the preconditioner diagonal, formed once per shift
cudaError_t precond_diag(const double* dg, double sigma, double delta, int64_t n, double* tinv, cudaStream_t s);
// Store:    Y = A G
// Sub:      Y = Y - A G                       (in place)
// Residual: R = Yin - A G; Y = T R; norm_part = per-tile column sums of R^2
// A: n x m (lda), G: m x p (ldg), Y: n x p (ldy). g_upper: G is upper triangular (K loop trimmed).
cudaError_t gemm_nn(const double* A, int64_t lda, const double* G, int ldg, int64_t n, int m, int p, double* Y,
                    int64_t ldy, const double* Yin, int64_t ldyin, Epi epi, bool g_upper, const ResidualArgs* ra,
                    cudaStream_t s);
int64_t norm_row_tiles(int64_t n);   // row tiles of gemm_nn / residual_diag (norm_part has this many rows)
// sum FP64 split-K partials part[split][i + j*ma] into C (mirrored when symmetric)
cudaError_t gram_reduce_partials(const double* part, int nsplit, int ma, int mb, double* C, int ldc, bool symmetric,
                                 cudaStream_t s);

// ---------------------------------------------------------------------------------------------- tcgen05 (TF32/BF16)
// Same contracts as gram / gemm_nn (Sub or Store), with TF32 (bf16 = false) or BF16 (bf16 = true) inputs and FP32
// accumulation on the tensor cores. *flag receives kFlagTimeout if a bounded mbarrier wait gave up.
cudaError_t tc_gram(const double* A, int64_t lda, const double* B, int64_t ldb, int64_t n, int ma, int mb, double* C,
                    int ldc, bool symmetric, double* part, size_t part_capacity, int* flag, cudaStream_t s,
                    bool bf16 = false);
cudaError_t tc_update(const double* A, int64_t lda, const double* G, int ldg, int64_t n, int m, int p, double* Y,
                      int64_t ldy, bool subtract, int* flag, cudaStream_t s, bool bf16 = false);

// ---------------------------------------------------------------------------------------------- Ozaki (FP64)
// FP64-accurate versions of gram / gemm_nn (Store or Sub) on the BF16 tensor cores by error-free splitting.
// exps: int workspace of oz_exp_elems(n, max columns) entries.
size_t oz_exp_elems(int64_t n, int cols);
// img (img_bytes, may be NULL): workspace for the operands' digit images (oz_img_bytes(n, ma) + oz_img_bytes(n, mb));
// with enough of it the Gram slices each operand once and feeds the tensor cores by bulk copies.
size_t oz_img_bytes(int64_t n, int cols);
cudaError_t oz_gram(const double* A, int64_t lda, const double* B, int64_t ldb, int64_t n, int ma, int mb, double* C,
                    int ldc, bool symmetric, double* part, size_t part_capacity, int* exps, uint8_t* img,
                    size_t img_bytes, int* flag, cudaStream_t s);
// g_upper: G is upper triangular with exact zeros below the diagonal (each column tile then reads only the rows
// of G up to its last column; the result is the same)
cudaError_t oz_update(const double* A, int64_t lda, const double* G, int ldg, int64_t n, int m, int p, double* Y,
                      int64_t ldy, Epi mode, int* exps, uint8_t* img, size_t img_bytes, int* flag, cudaStream_t s,
                      bool g_upper = false);

// ---------------------------------------------------------------------------------------------- vectors
// R = HX - X diag(lam); W = T R; norm_part per row tile.
cudaError_t residual_diag(const double* X, const double* HX, int64_t ld, int64_t n, int m, const double* lam,
                          const ResidualArgs& ra, double* W, cudaStream_t s);
// W (holding R) <- T R in place; norm_part per row tile gets the column sums of R^2
cudaError_t precond_norms(double* W, int64_t ld, int64_t n, int m, const ResidualArgs& ra, cudaStream_t s);
// out[c] = sum over row tiles of norm_part[t * m + c]
cudaError_t reduce_colnorms(const double* norm_part, int64_t tiles, int m, double* out, cudaStream_t s);
// out[:, j] = idx[j] >= 0 ? in[:, idx[j]] : 0 for j < m
cudaError_t gather_cols(const double* in, int64_t ldi, double* out, int64_t ldo, int64_t n, const int* idx, int m,
                        cudaStream_t s);
// rows[j] = row of the nonzero entry of column j of the m x m matrix C (column-major), whose columns are unit vectors
cudaError_t unit_column_rows(const double* C, int m, int* rows, cudaStream_t s);
// Unit norm and largest-modulus entry (lowest index on ties) positive, in place on n x m.
cudaError_t normalize_phase(double* X, int64_t ld, int64_t n, int m, double* scratch, cudaStream_t s);
// rho[p] = scale * sum_{c < k} X[p, c]^2
cudaError_t density(const double* X, int64_t ld, int64_t n, int k, double scale, double* rho, cudaStream_t s);
// dg = 6 * inv_h2 + V
cudaError_t make_diag(const double* V, double inv_h2, int64_t n, double* dg, cudaStream_t s);
// count non-finite entries of v[0..m) into *bad (device int)
cudaError_t check_finite(const double* v, int m, int* bad, cudaStream_t s);
// Complex (Bloch) problems in the real form: start block conversion, output extraction with the phase convention,
// and the density sum_c |z_c|^2 of a complex block (interleaved re/im, leading dimensions in complex entries).
cudaError_t cplx_to_realform(const double* Z, int64_t ldz, int64_t n, int kt, double* X, int64_t ldx, cudaStream_t s);
cudaError_t realform_to_cplx(const double* Y, int64_t ldy, int64_t n, int k, double* Z, int64_t ldz, cudaStream_t s);
cudaError_t density_c(const double* Z, int64_t ldz, int64_t n, int k, double scale, double* rho, cudaStream_t s);
// Polar orthonormalisation helpers (m x m, leading dimension m): Y = G - I in place with fro2[0] = ||Y||_F^2;
// Z = a Y + b I; Z += b I.
// Rayleigh-Ritz Grams with kl locked leading columns: G[0:kl, 0:kl] = I, M[0:kl, 0:kl] = diag(lam_lock), and the
// lower-left blocks G[kl:, 0:kl], M[kl:, 0:kl] mirrored from the computed upper-right ones (m x m, ld m).
cudaError_t locked_gram_fill(double* G, double* M, int m, int kl, const double* lam_lock, cudaStream_t s);
// Cholesky of a Gram with kl locked leading columns, G = [[I, G_la], [G_la^T, G_aa]]: the Schur complement
// Gs = G_aa - T (T = G_la^T G_la, ka x ka) with a breakdown flag for a pivot below pivot_tol^2 G_aa,ii, and
// R^{-1} = [[I, -U], [0, Ra^{-1}]] assembled from U = G_la Ra^{-1} (kl x ka) and Ra^{-1} (ka x ka, upper).
cudaError_t locked_schur(const double* G, int kt, int kl, const double* T, double pivot_tol, double* Gs, int* flag,
                         cudaStream_t s);
cudaError_t locked_rinv_fill(double* Rinv, int kt, int kl, const double* U, const double* Rainv, cudaStream_t s);
cudaError_t eye_residual(double* G, int m, double* fro2, cudaStream_t s);
cudaError_t scaled_plus_identity(const double* Y, int m, double a, double b, double* Z, cudaStream_t s);
cudaError_t add_diag(double* Z, int m, double b, cudaStream_t s);

// ---------------------------------------------------------------------------------------------- sub-blocks
struct BlockArgs {
  const double *X, *W, *P, *HX, *HW, *HP;
  int64_t ld, n;
  int k_act, q, has_p;
};
size_t block_gram_part_elems(int64_t n, int k_act, int q);
cudaError_t block_gram(const BlockArgs& a, double* part, size_t part_capacity, int* nchunk_out, cudaStream_t s);
cudaError_t block_solve(const BlockArgs& a, const double* part, int nchunk, double* coef, int* flags,
                        int* counters, cudaStream_t s);
cudaError_t block_update(double* X, const double* W, double* P, int64_t ld, int64_t n, int k_act, int q,
                         int has_p, const double* coef, cudaStream_t s);

// ---------------------------------------------------------------------------------------------- dense k x k
// How the dense k x k products of the Rayleigh-Ritz step (reduction, back-transformation, eigenvector refinement)
// and of the polar series run: FP64 split-K products on the FMA pipe, or, when ozaki is set and the product is
// large enough to fill the GPU, the FP64-accurate Ozaki emulation on the BF16 tensor cores.
struct KxK {
  double* part;         // split partials (>= m * p doubles)
  size_t part_cap;
  bool ozaki;
  int* exps;            // Ozaki exponent workspace (oz_exp_elems of the largest operand)
  uint8_t* img;         // Ozaki digit images (may be NULL)
  size_t img_bytes;
  int* flag;            // tensor-core timeout flag
};
// C (m x p, ldc) = op(A) B: op(A) = A^T with A kdim x m when trans_a, else A with A m x kdim; B is kdim x p.
// C must not overlap A or B. With trans_a and A == B (m == p) the result is exactly symmetric.
cudaError_t kxk_gemm(const KxK& g, bool trans_a, const double* A, int64_t lda, const double* B, int64_t ldb, int m,
                     int p, int kdim, double* C, int ldc, cudaStream_t s);

size_t chol_ws_elems(int m);
// Rinv (m x m, ldr = m, upper) = R^{-1} for G + shift I = R^T R (G m x m, ldg = m). Sets kFlagCholBreakdown in
// *flag on a relative pivot below kCholPivotTol.
cudaError_t chol_inv(const double* G, int m, double shift, double* Rinv, double* ws, int* flag, unsigned* bar,
                     cudaStream_t s);
size_t jacobi_ws_elems(int m);
// lambda ascending (m), C (m x m) eigenvectors of symmetric M (m x m, upper read).
cudaError_t jacobi_eigh(const double* M, int m, double* lambda, double* C, double* ws, int* flag, unsigned* bar,
                        int* sweeps_out_dev, cudaStream_t s);
// The same decomposition, cheapest route first: a diagonal M is sorted; a nearly diagonal M has its eigenvectors
// refined from the identity; otherwise a single-precision Jacobi gives the start of the refinement; FP64 Jacobi
// (jacobi_eigh) is the fallback. ws: jacobi_ws_elems(m); msym: m x m scratch; g: how the m x m products run.
// Synchronises the stream. path_out: 0 FP64 Jacobi, 1 diagonal, 2 refined from the identity, 3 refined from the
// single-precision Jacobi.
cudaError_t dense_eigh_auto(const double* M, int m, double* lambda, double* C, double* ws, double* msym,
                            const KxK& g, int* flag, unsigned* bar, int* sweeps_out_dev, int* path_out,
                            cudaStream_t s);
size_t barrier_words();
// Runs a cooperative kernel whose grid barrier can never complete (one CTA never arrives) with the given bound on
// the wait: the waiting CTAs give up, set kFlagTimeout in *flag and return.
cudaError_t barrier_timeout_probe(long long spin_limit, int* flag, unsigned* bar, cudaStream_t s);

}  // namespace ppcg
