// C ABI and host driver of the PPCG eigensolver (Algorithm 3 of arXiv 1407.7506, Appendix A).
//
// The driver keeps every block on the device and enqueues the library's own kernels on the caller's stream.
// It reads back two things to steer the loop: ||W||_F after each plain iteration (early Rayleigh-Ritz trigger)
// and the k_t Ritz residual norms after each Rayleigh-Ritz step (stop test and locking), plus the CholQR
// breakdown flag.
//
// Device layout (column-major, leading dimension ld = n rounded up to 32 doubles):
//   X  n x kt   [X_lock | X_act]: locked Ritz vectors first (ascending), then the active columns
//   HX n x kt   A X for the same columns
//   W, HW, P, HP  n x k_act  (active columns only, aligned with X_act)
//   Xs n x kt   scratch for out-of-place GEMMs and column gathers (roles are swapped, never copied)
#include "ppcg_internal.h"
#include "../../include/ppcg.h"
#include "../../include/ppcg_steps.h"

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstring>
#include <new>
#include <thread>
#include <vector>

using namespace ppcg;

struct ppcg_ctx {
  Grid grid{};
  double h = 1.0;
  int64_t n = 0, ld = 0;
  int k = 0, nbuf = 0, kt = 0, q = 1, rr_period = 1;
  ppcg_options opt{};
  double delta = 0.1;
  cudaStream_t stream = nullptr;
  void* ws = nullptr;
  size_t ws_bytes = 0;
  bool own_ws = false;
  // device
  double *V = nullptr, *dg = nullptr;
  double* blk[7] = {};
  double *X = nullptr, *Xs = nullptr, *HX = nullptr, *W = nullptr, *HW = nullptr, *P = nullptr, *HP = nullptr;
  double *G = nullptr, *M = nullptr, *C = nullptr, *Rinv = nullptr, *lam = nullptr, *norms = nullptr;
  double* lamlk = nullptr;    // Ritz values of the locked columns (their Rayleigh-Ritz step), leading kl entries
  double* tinv = nullptr;     // preconditioner diagonal 1 / max(dg - sigma, delta) for tinv_sigma
  double tinv_sigma = 0.0;
  bool tinv_valid = false;
  double *normpart = nullptr, *gpart = nullptr, *bpart = nullptr, *coef = nullptr, *cholws = nullptr,
         *jacws = nullptr;
  size_t gpart_cap = 0, bpart_cap = 0;
  int *iflag = nullptr, *icnt = nullptr, *jinfo = nullptr, *idx = nullptr, *bflags = nullptr;
  unsigned* bar = nullptr;
  // host mirrors
  std::vector<double> lam_h, nrm_h;
  int counters_h[4] = {0, 0, 0, 0};
  // phase timing
  std::vector<cudaEvent_t> evpool;
  std::vector<int> evphase;
  size_t evused = 0;
  double t_ms[8] = {};
  int last_sweeps = 0;
  int eig_path = 0;           // route of the last dense_eigh: 0 Jacobi, 1 diagonal, 2 refined, 3 FP32 + refined
  int eig_count[4] = {0, 0, 0, 0};   // dense_eigh calls of the current solve per route
  bool mixed = false;      // PPCG_MIXED_TF32 / _BF16: projections and the first CholQR Gram on tcgen05
  bool bf16 = false;       // PPCG_MIXED_BF16: those GEMMs take BF16 operands (else TF32)
  bool ozaki = false;      // FP64 n x k GEMMs emulated on the BF16 tensor cores (error-free splitting)
  int* ozexps = nullptr;   // exponent workspace of the emulated GEMMs
  uint8_t* ozimg = nullptr;   // digit images of the emulated Grams' operands
  size_t ozimg_bytes = 0;
  int* tcflag = nullptr;   // timeout flag of the tensor-core kernels
  bool cplx = false;       // complex Hermitian (Bloch) problem, solved in the real form of order 2 ng
  int64_t ng = 0;          // grid points (the complex order); n = 2 ng for a complex handle
  int kc = 0;              // wanted complex pairs (k = 2 kc internally)
  std::chrono::steady_clock::time_point t_solve0;   // start of the current solve (history time stamps)
};

namespace {

constexpr size_t kAlign = 256;

struct Layout {
  size_t bytes = 0;
  size_t off(size_t elems, size_t esize) {
    const size_t o = (bytes + kAlign - 1) / kAlign * kAlign;
    bytes = o + elems * esize;
    return o;
  }
};

struct Sizes {
  int64_t n, ld;
  int kt, q, smax;
  size_t gpart_cap, bpart_cap;
  size_t ozimg_bytes;   // digit images of the Ozaki Grams (0 unless the FP64 GEMMs are emulated)
};

Sizes make_sizes(int64_t n, int kt, int q, bool ozaki) {
  Sizes s{};
  s.n = n;
  s.ld = ceil_div(n, 32) * 32;
  s.kt = kt;
  s.q = q;
  s.smax = (int)ceil_div(kt, q);
  size_t kk = (size_t)kt * kt;
  size_t cap = kk * 64;
  const size_t lim = (size_t)32 << 20;
  if (cap > lim) cap = lim;
  if (cap < kk) cap = kk;
  s.gpart_cap = cap;
  s.bpart_cap = block_gram_part_elems(n, kt, q);
  s.ozimg_bytes = ozaki ? oz_img_bytes(n, kt) : 0;
  return s;
}

// Offsets of every region; returns the total byte count.
struct Offsets {
  size_t V, dg, tinv, blk[7], G, M, C, Rinv, lam, lamlk, norms, normpart, gpart, bpart, coef, cholws, jacws;
  size_t iflag, icnt, jinfo, idx, bflags, bar, ozexps, ozimg;
  size_t total;
};

Offsets layout(const Sizes& s) {
  Layout L;
  Offsets o{};
  const size_t blk = (size_t)s.ld * s.kt;
  o.V = L.off(s.ld, 8);
  o.dg = L.off(s.ld, 8);
  o.tinv = L.off(s.ld, 8);
  for (int i = 0; i < 7; ++i) o.blk[i] = L.off(blk, 8);
  const size_t kk = (size_t)s.kt * s.kt;
  o.G = L.off(kk, 8);
  o.M = L.off(kk, 8);
  o.C = L.off(kk, 8);
  o.Rinv = L.off(kk, 8);
  o.lam = L.off(s.kt, 8);
  o.lamlk = L.off(s.kt, 8);
  o.norms = L.off(s.kt, 8);
  o.normpart = L.off((size_t)norm_row_tiles(s.n) * s.kt, 8);
  o.gpart = L.off(s.gpart_cap, 8);
  o.bpart = L.off(s.bpart_cap, 8);
  o.coef = L.off((size_t)s.smax * 3 * s.q * s.q, 8);
  o.cholws = L.off(chol_ws_elems(s.kt), 8);
  o.jacws = L.off(jacobi_ws_elems(s.kt), 8);
  o.iflag = L.off(4, 4);
  o.icnt = L.off(4, 4);
  o.jinfo = L.off(4, 4);
  o.idx = L.off(s.kt, 4);
  o.bflags = L.off(s.smax, 4);
  o.bar = L.off(barrier_words(), 4);
  o.ozexps = L.off(oz_exp_elems(s.n, s.kt), 4);
  o.ozimg = L.off(s.ozimg_bytes, 1);
  o.total = L.bytes + kAlign;
  return o;
}

ppcg_status check_args(const ppcg_operator* op, int64_t n, int32_t k, int32_t sbsize, int32_t rr_period,
                       const ppcg_options* opt) {
  if (!op) return PPCG_ERR_ARG;
  if (op->nx < 1 || op->ny < 1 || op->nz < 1 || op->nz > 65535) return PPCG_ERR_ARG;
  if ((int64_t)op->nx * op->ny * op->nz != n) return PPCG_ERR_ARG;
  if (!(op->h > 0.0) || !std::isfinite(op->h)) return PPCG_ERR_ARG;
  if (op->dtype != PPCG_R64 && op->dtype != PPCG_C128) return PPCG_ERR_UNSUPPORTED;
  for (int d = 0; d < 3; ++d)
    if (!std::isfinite(op->theta[d])) return PPCG_ERR_ARG;
  const bool cplx = op->dtype == PPCG_C128;
  if (!cplx && (op->theta[0] != 0.0 || op->theta[1] != 0.0 || op->theta[2] != 0.0)) return PPCG_ERR_UNSUPPORTED;
  const int nbuf = opt ? opt->nbuf : 0;
  if (k < 1 || nbuf < 0 || rr_period < 1) return PPCG_ERR_ARG;
  const int64_t kt = (int64_t)k + nbuf;
  const int f = cplx ? 2 : 1;                    // a complex column is a pair of real-form columns
  if (2 * kt > n || f * kt > 65535) return PPCG_ERR_ARG;
  if (sbsize < 1 || f * sbsize > kMaxSbsize || sbsize > kt) return PPCG_ERR_ARG;
  if (opt && (opt->maxiter < 0 || opt->sigma_floor < 0.0)) return PPCG_ERR_ARG;
  if (opt && opt->precision != PPCG_FP64 && opt->precision != PPCG_MIXED_TF32 && opt->precision != PPCG_MIXED_BF16)
    return PPCG_ERR_UNSUPPORTED;
  if (opt && (opt->fp64_gemm < 0 || opt->fp64_gemm > 1)) return PPCG_ERR_ARG;
  if (opt && (opt->orth < 0 || opt->orth > 1)) return PPCG_ERR_ARG;
  if (opt && !(opt->orth_skip_tol >= 0.0 && std::isfinite(opt->orth_skip_tol))) return PPCG_ERR_ARG;
  return PPCG_OK;
}

thread_local cudaError_t g_last_cuda = cudaSuccess;
std::atomic<long long> g_launches{0};

#define CK(x)                                 \
  do {                                        \
    cudaError_t e_ = (x);                     \
    if (e_ != cudaSuccess) {                  \
      g_last_cuda = e_;                       \
      return PPCG_ERR_CUDA;                   \
    }                                         \
  } while (0)

#define PS(x)                                 \
  do {                                        \
    ppcg_status s_ = (x);                     \
    if (s_ != PPCG_OK) return s_;             \
  } while (0)

// ------------------------------------------------------------------------------------------ phase timing
void phase_mark(ppcg_ctx* c, int phase) {
  if (!c->opt.timing) return;
  if (c->evused == c->evpool.size()) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return;
    c->evpool.push_back(e);
    c->evphase.push_back(0);
  }
  cudaEventRecord(c->evpool[c->evused], c->stream);
  c->evphase[c->evused] = phase;
  ++c->evused;
}

void phase_flush(ppcg_ctx* c) {
  if (!c->opt.timing || c->evused < 2) {
    c->evused = 0;
    return;
  }
  cudaStreamSynchronize(c->stream);
  // event i closes the interval started by event i-1, attributed to the phase of event i-1
  for (size_t i = 1; i < c->evused; ++i) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, c->evpool[i - 1], c->evpool[i]) == cudaSuccess) c->t_ms[c->evphase[i - 1]] += ms;
  }
  c->evused = 0;
}

// ------------------------------------------------------------------------------------------ building blocks
ppcg_status apply_H(ppcg_ctx* c, const double* X, int64_t ldx, double* Y, int64_t ldy, int m) {
  CK(stencil_apply(c->grid, c->dg, X, ldx, Y, ldy, m, c->stream));
  return PPCG_OK;
}

constexpr int kProjectFuse = 128;   // W and P are projected as one block while together they have at most this many
                                    // columns (there the projections are bound by reading X, not by arithmetic)

// FP64 Gram over the n grid rows: FP64 pipe, or the FP64-accurate tensor-core emulation when selected.
// sym_result: A^T B is symmetric in exact arithmetic (X^T (H X) with H symmetric): only its upper tiles are formed
// and the lower triangle mirrors them, as for A^T A.
ppcg_status gram(ppcg_ctx* c, const double* A, int64_t lda, const double* B, int64_t ldb, int ma, int mb,
                 double* Cm, int ldc, bool sym_result = false) {
  const bool sym = ma == mb && ((A == B && lda == ldb) || sym_result);
  if (c->ozaki)
    CK(oz_gram(A, lda, B, ldb, c->n, ma, mb, Cm, ldc, sym, c->gpart, c->gpart_cap, c->ozexps, c->ozimg,
               c->ozimg_bytes, c->tcflag, c->stream));
  else
    CK(ppcg::gram(A, lda, B, ldb, c->n, ma, mb, Cm, ldc, sym, c->gpart, c->gpart_cap, c->stream));
  return PPCG_OK;
}

// FP64 update Y = A G (Store) or Y = Y - A G (Sub) over the n grid rows; g_upper trims the FP64-pipe K loop
ppcg_status update(ppcg_ctx* c, const double* A, int64_t lda, const double* G, int ldg, int m, int p, double* Y,
                   int64_t ldy, Epi mode, bool g_upper) {
  if (c->ozaki)
    CK(oz_update(A, lda, G, ldg, c->n, m, p, Y, ldy, mode, c->ozexps, c->ozimg, c->ozimg_bytes, c->tcflag,
                 c->stream, g_upper));
  else
    CK(gemm_nn(A, lda, G, ldg, c->n, m, p, Y, ldy, nullptr, 0, mode, g_upper, nullptr, c->stream));
  return PPCG_OK;
}

// Steps 20 / 8 fused: W = T (HX - X M) with column norms of HX - X M in norm_part
ppcg_status residual_m(ppcg_ctx* c, const double* X, const double* HX, int64_t ld, int m, const double* Mm,
                       const ResidualArgs& ra, double* W) {
  if (c->ozaki) {
    CK(cudaMemcpy2DAsync(W, ld * sizeof(double), HX, ld * sizeof(double), c->n * sizeof(double), m,
                         cudaMemcpyDeviceToDevice, c->stream));
    PS(update(c, X, ld, Mm, m, m, m, W, ld, Epi::Sub, false));
    CK(precond_norms(W, ld, c->n, m, ra, c->stream));
  } else {
    CK(gemm_nn(X, ld, Mm, m, c->n, m, m, W, ld, HX, ld, Epi::Residual, false, &ra, c->stream));
  }
  return PPCG_OK;
}

// Gram on the tensor cores (TF32 inputs, FP32 accumulation)
ppcg_status gram_tc(ppcg_ctx* c, const double* A, int64_t lda, const double* B, int64_t ldb, int ma, int mb,
                    double* Cm, int ldc) {
  const bool sym = (A == B && lda == ldb && ma == mb);
  CK(ppcg::tc_gram(A, lda, B, ldb, c->n, ma, mb, Cm, ldc, sym, c->gpart, c->gpart_cap, c->tcflag, c->stream,
                   c->bf16));
  return PPCG_OK;
}

// Steps 9-10: Y <- Y - X (X^T Y); on the tensor cores in the mixed form (the error only perturbs the search
// direction, whose coefficients the sub-block Rayleigh-Ritz then chooses in FP64)
ppcg_status project(ppcg_ctx* c, const double* X, int64_t ldx, int mx, double* Y, int64_t ldy, int my) {
  if (mx <= 0 || my <= 0) return PPCG_OK;
  if (c->mixed) {
    PS(gram_tc(c, X, ldx, Y, ldy, mx, my, c->G, mx));
    CK(tc_update(X, ldx, c->G, mx, c->n, mx, my, Y, ldy, true, c->tcflag, c->stream, c->bf16));
    return PPCG_OK;
  }
  PS(gram(c, X, ldx, Y, ldy, mx, my, c->G, mx));
  PS(update(c, X, ldx, c->G, mx, mx, my, Y, ldy, Epi::Sub, false));
  return PPCG_OK;
}

// One CholQR pass: Xout = Xin R^{-1}, Xin^T Xin + shift I = R^T R. lowprec: the Gram on the tensor cores (first
// pass of the mixed form); X R^{-1} is always applied in FP64, so span(X) is kept to FP64 accuracy.
ppcg_status cholqr_pass(ppcg_ctx* c, const double* Xin, int64_t ldi, double* Xout, int64_t ldo, int m,
                        double shift, bool lowprec = false) {
  if (lowprec) PS(gram_tc(c, Xin, ldi, Xin, ldi, m, m, c->G, m));
  else PS(gram(c, Xin, ldi, Xin, ldi, m, m, c->G, m));
  CK(chol_inv(c->G, m, shift, c->Rinv, c->cholws, c->iflag, c->bar, c->stream));
  PS(update(c, Xin, ldi, c->Rinv, m, m, m, Xout, ldo, Epi::Store, true));
  return PPCG_OK;
}

int read_flag(ppcg_ctx* c) {
  int f = 0;
  if (cudaMemcpyAsync(&f, c->iflag, sizeof(int), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess) return -1;
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) return -1;
  return f;
}

// CholeskyQR2 in place on X (n x m, ldx) with scratch Xs (ldxs); shifted CholeskyQR3 on breakdown.
ppcg_status cholqr2(ppcg_ctx* c, double* X, int64_t ldx, double* Xs, int64_t ldxs, int m, int* fell_back) {
  if (fell_back) *fell_back = 0;
  if (m <= 0) return PPCG_OK;
  CK(cudaMemsetAsync(c->iflag, 0, sizeof(int), c->stream));
  PS(cholqr_pass(c, X, ldx, Xs, ldxs, m, 0.0, c->mixed));
  int f = read_flag(c);
  if (f < 0) return PPCG_ERR_CUDA;
  if (f & kFlagTimeout) return PPCG_ERR_TIMEOUT;
  if (!(f & kFlagCholBreakdown)) {
    PS(cholqr_pass(c, Xs, ldxs, X, ldx, m, 0.0));
    f = read_flag(c);
    if (f < 0) return PPCG_ERR_CUDA;
    if (f & kFlagTimeout) return PPCG_ERR_TIMEOUT;
    if (!(f & kFlagCholBreakdown)) return PPCG_OK;
  }
  // shifted CholeskyQR3 (Fukaya, Kannan, Nakatsukasa, Yamamoto, Yamamoto 2020): shift from ||X||_F^2
  if (fell_back) *fell_back = 1;
  PS(gram(c, X, ldx, X, ldx, m, m, c->G, m));
  std::vector<double> g((size_t)m * m);
  CK(cudaMemcpyAsync(g.data(), c->G, sizeof(double) * g.size(), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  double fro2 = 0.0;
  for (int i = 0; i < m; ++i) fro2 += g[(size_t)i * m + i];
  const double u = 1.1102230246251565e-16;
  const double shift = 11.0 * ((double)c->n * m + (double)m * (m + 1)) * u * fro2;
  CK(cudaMemsetAsync(c->iflag, 0, sizeof(int), c->stream));
  PS(cholqr_pass(c, X, ldx, Xs, ldxs, m, shift));
  PS(cholqr_pass(c, Xs, ldxs, X, ldx, m, 0.0));
  PS(cholqr_pass(c, X, ldx, Xs, ldxs, m, 0.0));
  CK(cudaMemcpy2DAsync(X, ldx * sizeof(double), Xs, ldxs * sizeof(double), c->n * sizeof(double), m,
                       cudaMemcpyDeviceToDevice, c->stream));
  const int f2 = read_flag(c);
  if (f2 < 0) return PPCG_ERR_CUDA;
  if (f2 & kFlagTimeout) return PPCG_ERR_TIMEOUT;
  if (f2 & kFlagCholBreakdown) return PPCG_ERR_BREAKDOWN;
  return PPCG_OK;
}

// how the k x k products run: on the tensor cores (Ozaki) whenever the n x k GEMMs do
KxK kxk(ppcg_ctx* c) {
  return KxK{c->gpart, c->gpart_cap, c->ozaki, c->ozexps, c->ozimg, c->ozimg_bytes, c->tcflag};
}

// Mm must not alias c->G (the symmetrisation scratch) or Cm
ppcg_status dense_eigh(ppcg_ctx* c, const double* Mm, int m, double* lam, double* Cm) {
  CK(cudaMemsetAsync(c->iflag, 0, sizeof(int), c->stream));
  CK(cudaMemsetAsync(c->jinfo, 0, 2 * sizeof(int), c->stream));
  int path = 0;
  CK(dense_eigh_auto(Mm, m, lam, Cm, c->jacws, c->G, kxk(c), c->iflag, c->bar, c->jinfo, &path, c->stream));
  c->eig_path = path;
  if (path >= 0 && path < 4) c->eig_count[path]++;
  return PPCG_OK;
}

// sweeps used by the last dense_eigh (synchronises)
int last_sweeps(ppcg_ctx* c) {
  int info[2] = {0, 0};
  if (cudaMemcpyAsync(info, c->jinfo, sizeof(info), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess) return -1;
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) return -1;
  return info[0];
}

// Terms of the polar series: the fewest t >= 1 with |c_{t+1}| nu^{t+1} <= u (FP64 unit roundoff), 0 if none
// within kPolarMaxTerms. c_j = binom(-1/2, j) by c_j = c_{j-1} (-(2j - 1) / (2j)).
int polar_terms(double nu, double* coef) {
  coef[0] = 1.0;
  for (int j = 1; j <= kPolarMaxTerms + 1; ++j) coef[j] = coef[j - 1] * (-(2.0 * j - 1.0) / (2.0 * j));
  const double u = 1.1102230246251565e-16;
  for (int t = 1; t <= kPolarMaxTerms; ++t)
    if (std::fabs(coef[t + 1]) * std::pow(nu, t + 1) <= u) return t;
  return 0;
}

// Step 18 with the variants of Section 5.5: CholeskyQR2, the polar series X (I + Y)^{-1/2} (Y = X^T X - I, FP64
// Gram in every form), or no orthonormalisation when ||Y||_F <= orth_skip_tol.
ppcg_status orthonormalize(ppcg_ctx* c, double* X, int64_t ldx, double* Xs, int64_t ldxs, int m, ppcg_stats* S) {
  const bool variant = c->opt.orth != 0 || c->opt.orth_skip_tol > 0.0;
  if (variant && m > 0) {
    PS(gram(c, X, ldx, X, ldx, m, m, c->G, m));
    CK(eye_residual(c->G, m, c->C, c->stream));                  // Y = G - I in G, ||Y||_F^2 in C[0]
    double nu2 = 0.0;
    CK(cudaMemcpyAsync(&nu2, c->C, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (!std::isfinite(nu2)) return PPCG_ERR_NUMERIC;
    const double nu = std::sqrt(nu2);
    if (nu <= c->opt.orth_skip_tol) {
      S->n_orth_skip++;
      return PPCG_OK;
    }
    double coef[kPolarMaxTerms + 2];
    const int t = c->opt.orth == 1 ? polar_terms(nu, coef) : 0;
    if (t > 0) {
      // Horner: Z = c_t Y + c_{t-1} I; Z <- Y Z + c_j I for j = t-2 .. 0 (Y in G; Z alternates M / Rinv)
      double* Z = c->M;
      double* Zn = c->Rinv;
      CK(scaled_plus_identity(c->G, m, coef[t], coef[t - 1], Z, c->stream));
      for (int j = t - 2; j >= 0; --j) {
        CK(kxk_gemm(kxk(c), false, c->G, m, Z, m, m, m, m, Zn, m, c->stream));
        CK(add_diag(Zn, m, coef[j], c->stream));
        std::swap(Z, Zn);
      }
      PS(update(c, X, ldx, Z, m, m, m, Xs, ldxs, Epi::Store, false));
      CK(cudaMemcpy2DAsync(X, ldx * sizeof(double), Xs, ldxs * sizeof(double), c->n * sizeof(double), m,
                           cudaMemcpyDeviceToDevice, c->stream));
      S->n_polar++;
      return PPCG_OK;
    }
  }
  int fb = 0;
  PS(cholqr2(c, X, ldx, Xs, ldxs, m, &fb));
  if (fb) S->n_cholqr_fallback++;
  return PPCG_OK;
}

ResidualArgs resid_args(ppcg_ctx* c, double sigma) {
  ResidualArgs ra{};
  ra.dg = c->dg;
  ra.sigma = sigma;
  ra.delta = c->delta;
  ra.norm_part = c->normpart;
  // the preconditioner diagonal changes only with sigma (once per Rayleigh-Ritz step): form it once
  if (!(c->tinv_valid && c->tinv_sigma == sigma) &&
      precond_diag(c->dg, sigma, c->delta, c->n, c->tinv, c->stream) == cudaSuccess) {
    c->tinv_valid = true;
    c->tinv_sigma = sigma;
  }
  ra.tinv = (c->tinv_valid && c->tinv_sigma == sigma) ? c->tinv : nullptr;
  return ra;
}

void swap(double*& a, double*& b) {
  double* t = a;
  a = b;
  b = t;
}

struct SolveState {
  int k_lock = 0, k_act = 0;
  std::vector<int> pos_act;    // positions (sorted Ritz order at the last RR) of the active columns
  std::vector<int> pos_lock;
  bool has_p = false;
  double sigma = 0.0;
  bool done = false;
  double max_res = 0.0;
};

// Steps 22-31: Rayleigh-Ritz on S = [X_lock, X_act], residuals, stop test, locking and compaction.
// Step 23 solves eq. projev on S as written: with S^T S = R^T R (Cholesky), K = R^{-T} (S^T A S) R^{-1} is
// diagonalised, K Z = Z Omega, and X = S (R^{-1} Z). If that Cholesky breaks down (relative pivot below
// kCholPivotTol), S is orthonormalised by CholeskyQR2 first and the standard problem Q^T A Q is solved instead.
// The locked columns are orthonormal Ritz vectors of the previous Rayleigh-Ritz step that no step has touched
// since (steps 9-20 act on the active columns only), so the locked block of S^T S is I and that of S^T A S is
// diag(Lambda_lock) in exact arithmetic: only S^T X_act and S^T (A X_act) are formed, n k_t k_act work instead of
// the full Grams' n k_t^2 (most columns are locked late in a solve).
ppcg_status rr_step(ppcg_ctx* c, SolveState& st, bool allow_compact, ppcg_stats* stats, double tol) {
  const int kt = c->kt;
  cudaStream_t s = c->stream;
  int* rrflag = c->icnt + 3;
  const int kl = st.k_lock < kt ? st.k_lock : 0;
  phase_mark(c, PPCG_T_AX);
  if (kl > 0) PS(apply_H(c, c->X + (int64_t)kl * c->ld, c->ld, c->HX + (int64_t)kl * c->ld, c->ld, kt - kl));
  else PS(apply_H(c, c->X, c->ld, c->HX, c->ld, kt));
  phase_mark(c, PPCG_T_RR);
  if (kl > 0) {
    const double* Xa = c->X + (int64_t)kl * c->ld;
    const double* HXa = c->HX + (int64_t)kl * c->ld;
    PS(gram(c, c->X, c->ld, Xa, c->ld, kt, kt - kl, c->G + (int64_t)kl * kt, kt));    // S^T X_act
    PS(gram(c, c->X, c->ld, HXa, c->ld, kt, kt - kl, c->M + (int64_t)kl * kt, kt));   // S^T A X_act
    CK(locked_gram_fill(c->G, c->M, kt, kl, c->lamlk, s));
  } else {
    PS(gram(c, c->X, c->ld, c->X, c->ld, kt, kt, c->G, kt));            // S^T S
    PS(gram(c, c->X, c->ld, c->HX, c->ld, kt, kt, c->M, kt, true));     // S^T A S
  }
  CK(cudaMemsetAsync(rrflag, 0, sizeof(int), s));
  if (kl > 0) {
    // S^T S = [[I, G_la], [G_la^T, G_aa]] = R^T R with R = [[I, G_la], [0, Ra]], Ra^T Ra = G_aa - G_la^T G_la:
    // only the k_act x k_act Schur complement is factorised
    const int ka = kt - kl;
    const double* Gla = c->G + (int64_t)kl * kt;
    double* Gs = c->jacws;                                   // scratch until the eigensolve
    double* Rainv = c->jacws + (int64_t)ka * ka;
    CK(kxk_gemm(kxk(c), true, Gla, kt, Gla, kt, ka, ka, kl, c->C, ka, s));          // G_la^T G_la
    CK(locked_schur(c->G, kt, kl, c->C, kCholPivotTol, Gs, rrflag, s));
    CK(chol_inv(Gs, ka, 0.0, Rainv, c->cholws, rrflag, c->bar, s));
    CK(kxk_gemm(kxk(c), false, Gla, kt, Rainv, ka, kl, ka, ka, c->C, kl, s));       // U = G_la Ra^{-1}
    CK(locked_rinv_fill(c->Rinv, kt, kl, c->C, Rainv, s));
  } else {
    CK(chol_inv(c->G, kt, 0.0, c->Rinv, c->cholws, rrflag, c->bar, s));  // R^{-1}
  }
  // K = R^{-T} (S^T A S) R^{-1}: T = (S^T A S) R^{-1} (R^{-1} upper: trimmed K loop), K = (R^{-1})^T T
  CK(kxk_gemm(kxk(c), false, c->M, kt, c->Rinv, kt, kt, kt, kt, c->G, kt, s));
  CK(kxk_gemm(kxk(c), true, c->Rinv, kt, c->G, kt, kt, kt, kt, c->M, kt, s));
  PS(dense_eigh(c, c->M, kt, c->lam, c->C));
  // sigma = smallest Ritz value of this step: the host needs it for the preconditioner
  CK(cudaMemcpyAsync(c->lam_h.data(), c->lam, sizeof(double) * kt, cudaMemcpyDeviceToHost, s));
  int fl[3] = {0, 0, 0};
  bool diag_shortcut = false;
  CK(cudaMemcpyAsync(&fl[0], c->iflag, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(&fl[1], c->tcflag, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(&fl[2], rrflag, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if ((fl[0] | fl[1] | fl[2]) & kFlagTimeout) return PPCG_ERR_TIMEOUT;
  if (fl[2] & kFlagCholBreakdown) {
    // S^T S too ill-conditioned for the reduction: orthonormalise S and solve the standard problem
    if (stats) stats->n_cholqr_fallback++;
    int fb = 0;
    PS(cholqr2(c, c->X, c->ld, c->Xs, c->ld, kt, &fb));
    PS(apply_H(c, c->X, c->ld, c->HX, c->ld, kt));
    PS(gram(c, c->X, c->ld, c->HX, c->ld, kt, kt, c->M, kt, true));
    PS(dense_eigh(c, c->M, kt, c->lam, c->C));
    CK(cudaMemcpyAsync(c->G, c->C, sizeof(double) * (size_t)kt * kt, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(c->lam_h.data(), c->lam, sizeof(double) * kt, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(&fl[0], c->iflag, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (fl[0] & kFlagTimeout) return PPCG_ERR_TIMEOUT;
  } else if (kl > 0 && c->eig_path == 1) {
    // The eigenvectors are unit vectors (K was diagonal to the eigensolver's tolerance) and so are the locked
    // columns of R^{-1} = [[I, -U], [0, Ra^{-1}]]: the new block S R^{-1} Z is [X_lock, S R^{-1}[:, kl:]] with its
    // columns permuted by Z. The locked columns, and H applied to them, are copied instead of recomputed.
    const int ka = kt - kl;
    PS(update(c, c->X, c->ld, c->Rinv + (int64_t)kl * kt, kt, kt, ka, c->Xs + (int64_t)kl * c->ld, c->ld, Epi::Store,
              false));
    CK(cudaMemcpy2DAsync(c->Xs, c->ld * sizeof(double), c->X, c->ld * sizeof(double), c->n * sizeof(double), kl,
                         cudaMemcpyDeviceToDevice, s));
    phase_mark(c, PPCG_T_AX);
    PS(apply_H(c, c->Xs + (int64_t)kl * c->ld, c->ld, c->HX + (int64_t)kl * c->ld, c->ld, ka));
    phase_mark(c, PPCG_T_RR);
    CK(unit_column_rows(c->C, kt, c->idx, s));
    CK(gather_cols(c->Xs, c->ld, c->X, c->ld, c->n, c->idx, kt, s));
    CK(gather_cols(c->HX, c->ld, c->Xs, c->ld, c->n, c->idx, kt, s));
    swap(c->HX, c->Xs);
    diag_shortcut = true;
    if (stats) stats->n_rr_unit++;
  } else {
    // coefficients R^{-1} Z (R^{-1} is upper triangular)
    CK(kxk_gemm(kxk(c), false, c->Rinv, kt, c->C, kt, kt, kt, kt, c->G, kt, s));
  }
  if (!diag_shortcut) {
    PS(update(c, c->X, c->ld, c->G, kt, kt, kt, c->Xs, c->ld, Epi::Store, false));
    swap(c->X, c->Xs);
    phase_mark(c, PPCG_T_AX);
    PS(apply_H(c, c->X, c->ld, c->HX, c->ld, kt));
  }
  phase_mark(c, PPCG_T_PRECOND);
  st.sigma = c->lam_h[0];
  if (stats) {
    const int sw = last_sweeps(c);
    if (sw > stats->jacobi_sweeps_max) stats->jacobi_sweeps_max = sw;
  }
  ResidualArgs ra = resid_args(c, st.sigma);
  CK(residual_diag(c->X, c->HX, c->ld, c->n, kt, c->lam, ra, c->W, c->stream));
  CK(reduce_colnorms(c->normpart, norm_row_tiles(c->n), kt, c->norms, c->stream));
  CK(cudaMemcpyAsync(c->nrm_h.data(), c->norms, sizeof(double) * kt, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  phase_mark(c, PPCG_T_LOCK);
  double mx = 0.0;
  for (int i = 0; i < kt; ++i) {
    if (!std::isfinite(c->nrm_h[i]) || !std::isfinite(c->lam_h[i])) return PPCG_ERR_NUMERIC;
    if (i < c->k) mx = std::max(mx, std::sqrt(c->nrm_h[i]));
  }
  st.max_res = mx;
  st.done = mx <= tol;
  if (stats) stats->n_rr++;
  if (st.done || !allow_compact) return PPCG_OK;
  // locking (soft): J_lock = {i < k : r_i <= tol}; layout [locked ascending | active ascending]
  std::vector<int> lock, act;
  for (int i = 0; i < kt; ++i) {
    if (!c->opt.no_lock && i < c->k && std::sqrt(c->nrm_h[i]) <= tol) lock.push_back(i);
    else act.push_back(i);
  }
  std::vector<int> order(lock);
  order.insert(order.end(), act.begin(), act.end());
  const int nl = (int)lock.size(), na = (int)act.size();
  // P remap: new active column j takes the direction that belonged to position act[j] (zero if none)
  std::vector<int> pidx(na, -1);
  if (st.has_p) {
    for (int j = 0; j < na; ++j) {
      auto it = std::find(st.pos_act.begin(), st.pos_act.end(), act[j]);
      if (it != st.pos_act.end()) pidx[j] = (int)(it - st.pos_act.begin());
    }
  }
  std::vector<double> lam_lock(nl > 0 ? nl : 1);
  for (int i = 0; i < nl; ++i) lam_lock[i] = c->lam_h[lock[i]];
  if (nl > 0)
    CK(cudaMemcpyAsync(c->lamlk, lam_lock.data(), sizeof(double) * nl, cudaMemcpyHostToDevice, c->stream));
  int* d_order = c->idx;
  CK(cudaMemcpyAsync(d_order, order.data(), sizeof(int) * kt, cudaMemcpyHostToDevice, c->stream));
  CK(gather_cols(c->X, c->ld, c->Xs, c->ld, c->n, d_order, kt, c->stream));
  swap(c->X, c->Xs);
  CK(gather_cols(c->HX, c->ld, c->Xs, c->ld, c->n, d_order, kt, c->stream));
  swap(c->HX, c->Xs);
  // W: active columns (positions act) in order
  CK(cudaMemcpyAsync(d_order, act.data(), sizeof(int) * na, cudaMemcpyHostToDevice, c->stream));
  CK(gather_cols(c->W, c->ld, c->Xs, c->ld, c->n, d_order, na, c->stream));
  swap(c->W, c->Xs);
  if (st.has_p) {
    CK(cudaMemcpyAsync(d_order, pidx.data(), sizeof(int) * na, cudaMemcpyHostToDevice, c->stream));
    CK(gather_cols(c->P, c->ld, c->Xs, c->ld, c->n, d_order, na, c->stream));
    swap(c->P, c->Xs);
  }
  CK(cudaStreamSynchronize(c->stream));   // host vectors above must outlive the uploads
  st.k_lock = nl;
  st.k_act = na;
  st.pos_act = act;
  st.pos_lock = lock;
  return PPCG_OK;
}

void record(ppcg_ctx* c, ppcg_stats* S, int it, int kind, double value, double trace, int k_act) {
  if (!c->opt.history || S->history_len >= c->opt.history_cap) return;
  double* e = c->opt.history + 6 * (size_t)S->history_len;
  e[0] = it;
  e[1] = kind;
  e[2] = value;
  e[3] = trace;
  e[4] = k_act;
  // every entry is recorded right after the stream was synchronised to read the step's norms: host time since the
  // solve began is the device's progress (the residual-versus-time view of the paper's Figure "Liband")
  e[5] = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - c->t_solve0).count();
  S->history_len++;
}

double ritz_trace(const ppcg_ctx* c) {
  double t = 0.0;
  for (int i = 0; i < c->k; ++i) t += c->lam_h[i];
  return c->cplx ? 0.5 * t : t;            // the real form holds every complex Ritz value twice
}

}  // namespace

namespace ppcg {
void count_launch(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
long long launch_count() { return g_launches.load(std::memory_order_relaxed); }
}  // namespace ppcg

// ============================================================================================== C ABI
extern "C" {

const char* ppcg_status_string(ppcg_status s) {
  switch (s) {
    case PPCG_OK: return "PPCG_OK";
    case PPCG_ERR_ARG: return "PPCG_ERR_ARG: invalid argument";
    case PPCG_ERR_CUDA: return "PPCG_ERR_CUDA: a CUDA runtime call failed";
    case PPCG_ERR_OOM: return "PPCG_ERR_OOM: workspace allocation failed or too small";
    case PPCG_ERR_NOT_CONVERGED: return "PPCG_ERR_NOT_CONVERGED: maxiter reached";
    case PPCG_ERR_BREAKDOWN: return "PPCG_ERR_BREAKDOWN: orthonormalisation failed";
    case PPCG_ERR_NUMERIC: return "PPCG_ERR_NUMERIC: non-finite residual";
    case PPCG_ERR_TIMEOUT: return "PPCG_ERR_TIMEOUT: a bounded device wait gave up";
    case PPCG_ERR_UNSUPPORTED: return "PPCG_ERR_UNSUPPORTED: option not provided by this library";
  }
  return "PPCG: unknown status";
}

ppcg_status ppcg_workspace_bytes(const ppcg_operator* op, int64_t n, int32_t k, int32_t sbsize,
                                 const ppcg_options* opt, size_t* bytes) {
  if (!bytes) return PPCG_ERR_ARG;
  PS(check_args(op, n, k, sbsize, 1, opt));
  const int kt = k + (opt ? opt->nbuf : 0);
  const int f = op->dtype == PPCG_C128 ? 2 : 1;
  *bytes = layout(make_sizes(f * n, f * kt, f * sbsize, opt && opt->fp64_gemm == 1)).total;
  return PPCG_OK;
}

ppcg_status ppcg_create(const ppcg_operator* op, int64_t n, int32_t k, int32_t sbsize, int32_t rr_period,
                        const ppcg_options* opt, void* cuda_stream, void* workspace, size_t workspace_bytes,
                        ppcg_handle* out) {
  if (!out) return PPCG_ERR_ARG;
  *out = nullptr;
  PS(check_args(op, n, k, sbsize, rr_period, opt));
  if (!op->V) return PPCG_ERR_ARG;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) return PPCG_ERR_CUDA;
  ppcg_ctx* c = new (std::nothrow) ppcg_ctx();
  if (!c) return PPCG_ERR_OOM;
  c->grid.nx = op->nx;
  c->grid.ny = op->ny;
  c->grid.nz = op->nz;
  c->h = op->h;
  c->grid.inv_h2 = 1.0 / (op->h * op->h);
  if (opt) c->opt = *opt;
  if (c->opt.maxiter == 0) c->opt.maxiter = 500;
  c->delta = c->opt.sigma_floor > 0.0 ? c->opt.sigma_floor : 0.1 / (op->h * op->h);
  c->cplx = op->dtype == PPCG_C128;
  const int f = c->cplx ? 2 : 1;
  c->ng = n;
  c->kc = k;
  c->n = f * n;
  c->k = f * k;
  c->nbuf = f * c->opt.nbuf;
  c->kt = c->k + c->nbuf;
  c->q = f * sbsize;
  c->grid.cplx = c->cplx ? 1 : 0;
  for (int d = 0; d < 3; ++d) {
    c->grid.ct[d] = std::cos(op->theta[d]);
    c->grid.st[d] = std::sin(op->theta[d]);
  }
  c->rr_period = rr_period;
  c->stream = (cudaStream_t)cuda_stream;
  const Sizes sz = make_sizes(c->n, c->kt, c->q, c->opt.fp64_gemm == 1);
  const Offsets o = layout(sz);
  c->ld = sz.ld;
  c->gpart_cap = sz.gpart_cap;
  c->bpart_cap = sz.bpart_cap;
  if (workspace) {
    if (workspace_bytes < o.total) {
      delete c;
      return PPCG_ERR_OOM;
    }
    c->ws = workspace;
    c->ws_bytes = workspace_bytes;
  } else {
    if (cudaMalloc(&c->ws, o.total) != cudaSuccess) {
      cudaGetLastError();
      delete c;
      return PPCG_ERR_OOM;
    }
    c->own_ws = true;
    c->ws_bytes = o.total;
  }
  char* b = reinterpret_cast<char*>((reinterpret_cast<uintptr_t>(c->ws) + kAlign - 1) / kAlign * kAlign);
  auto D = [&](size_t off) { return reinterpret_cast<double*>(b + off); };
  auto I = [&](size_t off) { return reinterpret_cast<int*>(b + off); };
  c->V = D(o.V);
  c->dg = D(o.dg);
  c->tinv = D(o.tinv);
  for (int i = 0; i < 7; ++i) c->blk[i] = D(o.blk[i]);
  c->X = c->blk[0]; c->Xs = c->blk[1]; c->HX = c->blk[2]; c->W = c->blk[3];
  c->HW = c->blk[4]; c->P = c->blk[5]; c->HP = c->blk[6];
  c->G = D(o.G); c->M = D(o.M); c->C = D(o.C); c->Rinv = D(o.Rinv);
  c->lam = D(o.lam); c->lamlk = D(o.lamlk); c->norms = D(o.norms); c->normpart = D(o.normpart);
  c->gpart = D(o.gpart); c->bpart = D(o.bpart); c->coef = D(o.coef);
  c->cholws = D(o.cholws); c->jacws = D(o.jacws);
  c->iflag = I(o.iflag); c->icnt = I(o.icnt); c->jinfo = I(o.jinfo); c->idx = I(o.idx); c->bflags = I(o.bflags);
  c->bar = reinterpret_cast<unsigned*>(b + o.bar);
  c->tcflag = c->icnt + 2;
  c->mixed = (c->opt.precision == PPCG_MIXED_TF32 || c->opt.precision == PPCG_MIXED_BF16);
  c->bf16 = (c->opt.precision == PPCG_MIXED_BF16);
  c->ozaki = (c->opt.fp64_gemm == 1);
  c->ozexps = reinterpret_cast<int*>(b + o.ozexps);
  c->ozimg = sz.ozimg_bytes ? reinterpret_cast<uint8_t*>(b + o.ozimg) : nullptr;
  c->ozimg_bytes = sz.ozimg_bytes;
  c->lam_h.assign(c->kt, 0.0);
  c->nrm_h.assign(c->kt, 0.0);
  ppcg_status st = ppcg_set_potential(c, op->V);
  if (st != PPCG_OK) {
    ppcg_destroy(c);
    return st;
  }
  *out = c;
  return PPCG_OK;
}

ppcg_status ppcg_set_potential(ppcg_handle c, const double* V) {
  if (!c || !V) return PPCG_ERR_ARG;
  CK(cudaMemcpyAsync(c->V, V, sizeof(double) * c->ng, cudaMemcpyDefault, c->stream));
  CK(make_diag(c->V, c->grid.inv_h2, c->ng, c->dg, c->stream));
  c->tinv_valid = false;
  if (c->cplx)   // the real form's diagonal is diag(A) twice
    CK(cudaMemcpyAsync(c->dg + c->ng, c->dg, sizeof(double) * c->ng, cudaMemcpyDeviceToDevice, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return PPCG_OK;
}

ppcg_status ppcg_destroy(ppcg_handle c) {
  if (!c) return PPCG_OK;
  for (cudaEvent_t e : c->evpool) cudaEventDestroy(e);
  if (c->own_ws && c->ws) cudaFree(c->ws);
  delete c;
  return PPCG_OK;
}

ppcg_status ppcg_solve(ppcg_handle c, const double* X0, double tol, double* lambda, double* X, double* resnorm,
                       ppcg_stats* stats) {
  if (!c || !X0 || !lambda || !X || !(tol > 0.0)) return PPCG_ERR_ARG;
  ppcg_stats local{};
  ppcg_stats* S = stats ? stats : &local;
  std::memset(S, 0, sizeof(*S));
  c->t_solve0 = std::chrono::steady_clock::now();
  c->eig_count[0] = c->eig_count[1] = c->eig_count[2] = c->eig_count[3] = 0;
  std::memset(c->t_ms, 0, sizeof(c->t_ms));
  c->evused = 0;
  const long long launches0 = launch_count();
  const int kt = c->kt;
  const int64_t n = c->n, ld = c->ld;
  cudaStream_t s = c->stream;
  // pointers may be host or device (cudaMemcpyDefault resolves through unified addressing)
  phase_mark(c, PPCG_T_OTHER);
  if (c->cplx) {
    // complex X0 (ng x kt/2, interleaved) -> staging -> real form with J-paired columns
    CK(cudaMemcpyAsync(c->Xs, X0, sizeof(double) * 2 * (size_t)c->ng * (kt / 2), cudaMemcpyDefault, s));
    CK(cplx_to_realform(c->Xs, c->ng, c->ng, kt / 2, c->X, ld, s));
  } else {
    CK(cudaMemcpy2DAsync(c->X, ld * sizeof(double), X0, n * sizeof(double), n * sizeof(double), kt,
                         cudaMemcpyDefault, s));
  }
  CK(cudaMemsetAsync(c->icnt, 0, 4 * sizeof(int), s));
  SolveState st;
  st.k_lock = 0;
  st.k_act = kt;
  // step 1: X <- orth(X0)
  phase_mark(c, PPCG_T_CHOLQR);
  int fb = 0;
  PS(cholqr2(c, c->X, ld, c->Xs, ld, kt, &fb));
  if (fb) S->n_cholqr_fallback++;
  // Rayleigh-Ritz on orth(X0) before iteration 1 (provides sigma and the Ritz residual W)
  const int maxiter = c->opt.maxiter;
  PS(rr_step(c, st, maxiter > 0, S, tol));
  record(c, S, 0, 1, st.max_res, ritz_trace(c), kt);
  if (st.pos_act.empty()) {
    st.pos_act.resize(st.k_act);
    for (int j = 0; j < st.k_act; ++j) st.pos_act[j] = j;
  }
  bool last_rr = true;
  int it = 0;
  while (!st.done && it < maxiter) {
    ++it;
    const int ka = st.k_act, kl = st.k_lock;
    double* Xa = c->X + (int64_t)kl * ld;
    double* HXa = c->HX + (int64_t)kl * ld;
    // step 8 is fused into the residual of the previous step (W already holds T R)
    // steps 9-10: project W and P against [X_lock, X]
    phase_mark(c, PPCG_T_GEMM);
    if (st.has_p && 2 * ka <= kProjectFuse && 2 * ka <= kt) {
      // few active columns: the projections read all k_t columns of X for only 2 k_act columns of work, so W and P
      // are projected as one block [W, P] (staged in Xs, free until step 18): X is read twice instead of four times
      const size_t pitch = ld * sizeof(double), rows = n * sizeof(double);
      CK(cudaMemcpy2DAsync(c->Xs, pitch, c->W, pitch, rows, ka, cudaMemcpyDeviceToDevice, s));
      CK(cudaMemcpy2DAsync(c->Xs + (int64_t)ka * ld, pitch, c->P, pitch, rows, ka, cudaMemcpyDeviceToDevice, s));
      PS(project(c, c->X, ld, kt, c->Xs, ld, 2 * ka));
      CK(cudaMemcpy2DAsync(c->W, pitch, c->Xs, pitch, rows, ka, cudaMemcpyDeviceToDevice, s));
      CK(cudaMemcpy2DAsync(c->P, pitch, c->Xs + (int64_t)ka * ld, pitch, rows, ka, cudaMemcpyDeviceToDevice, s));
    } else {
      PS(project(c, c->X, ld, kt, c->W, ld, ka));
      if (st.has_p) PS(project(c, c->X, ld, kt, c->P, ld, ka));
    }
    phase_mark(c, PPCG_T_AX);
    PS(apply_H(c, c->W, ld, c->HW, ld, ka));
    if (st.has_p) PS(apply_H(c, c->P, ld, c->HP, ld, ka));
    // steps 11-16: sub-block Rayleigh-Ritz and update
    phase_mark(c, PPCG_T_BLOCKRR);
    BlockArgs ba{Xa, c->W, c->P, HXa, c->HW, c->HP, ld, n, ka, c->q, st.has_p ? 1 : 0};
    int nchunk = 0;
    CK(block_gram(ba, c->bpart, c->bpart_cap, &nchunk, s));
    CK(block_solve(ba, c->bpart, nchunk, c->coef, c->bflags, c->icnt, s));
    phase_mark(c, PPCG_T_GEMM);
    CK(block_update(Xa, c->W, c->P, ld, n, ka, c->q, st.has_p ? 1 : 0, c->coef, s));
    st.has_p = true;
    last_rr = false;
    bool do_rr = (it % c->rr_period) == 0;
    if (!do_rr) {
      // steps 18-20
      phase_mark(c, PPCG_T_CHOLQR);
      PS(orthonormalize(c, Xa, ld, c->Xs + (int64_t)kl * ld, ld, ka, S));
      phase_mark(c, PPCG_T_AX);
      PS(apply_H(c, Xa, ld, HXa, ld, ka));
      phase_mark(c, PPCG_T_GEMM);
      PS(gram(c, Xa, ld, HXa, ld, ka, ka, c->M, ka, true));            // M = X^T H X
      ResidualArgs ra = resid_args(c, st.sigma);
      PS(residual_m(c, Xa, HXa, ld, ka, c->M, ra, c->W));
      CK(reduce_colnorms(c->normpart, norm_row_tiles(n), ka, c->norms, s));
      CK(cudaMemcpyAsync(c->nrm_h.data(), c->norms, sizeof(double) * ka, cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      double wf2 = 0.0;
      for (int j = 0; j < ka; ++j) {
        if (!std::isfinite(c->nrm_h[j])) return PPCG_ERR_NUMERIC;
        if (st.pos_act[j] < c->k) wf2 += c->nrm_h[j];
      }
      record(c, S, it, 0, std::sqrt(wf2), 0.0, ka);
      if (std::sqrt(wf2) <= tol) {
        do_rr = true;            // forced Rayleigh-Ritz step: ||W||_F <= tol bounds every Ritz residual
        S->n_early_rr++;
      }
    }
    if (do_rr) {
      // steps 22-31
      PS(rr_step(c, st, it < maxiter, S, tol));
      record(c, S, it, 1, st.max_res, ritz_trace(c), ka);
      last_rr = true;
    }
  }
  if (!last_rr) {
    // step 32: final Rayleigh-Ritz (no compaction: X ends in ascending Ritz order)
    PS(rr_step(c, st, false, S, tol));
    record(c, S, it, 1, st.max_res, ritz_trace(c), st.k_act);
  }
  // outputs: first k Ritz pairs, phase convention, residuals recomputed on the returned vectors
  phase_mark(c, PPCG_T_OTHER);
  const int k = c->k;
  CK(cudaMemcpy2DAsync(c->Xs, ld * sizeof(double), c->X, ld * sizeof(double), n * sizeof(double), k,
                       cudaMemcpyDeviceToDevice, s));
  CK(normalize_phase(c->Xs, ld, n, k, nullptr, s));
  PS(apply_H(c, c->Xs, ld, c->HW, ld, k));
  ResidualArgs ra = resid_args(c, st.sigma);
  CK(residual_diag(c->Xs, c->HW, ld, n, k, c->lam, ra, c->HP, s));
  CK(reduce_colnorms(c->normpart, norm_row_tiles(n), k, c->norms, s));
  CK(cudaMemcpyAsync(c->nrm_h.data(), c->norms, sizeof(double) * k, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(c->lam_h.data(), c->lam, sizeof(double) * kt, cudaMemcpyDeviceToHost, s));
  if (c->cplx) {
    // complex pair j is real-form column 2j (its partner 2j+1 is the same vector times i)
    CK(realform_to_cplx(c->Xs, ld, c->ng, c->kc, c->W, c->ng, s));
    CK(cudaMemcpyAsync(X, c->W, sizeof(double) * 2 * (size_t)c->ng * c->kc, cudaMemcpyDefault, s));
  } else {
    CK(cudaMemcpy2DAsync(X, n * sizeof(double), c->Xs, ld * sizeof(double), n * sizeof(double), k,
                         cudaMemcpyDefault, s));
  }
  CK(cudaMemcpyAsync(c->counters_h, c->icnt, 4 * sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  phase_mark(c, PPCG_T_OTHER);
  phase_flush(c);
  double mx = 0.0;
  const int f = c->cplx ? 2 : 1;
  for (int i = 0; i < k / f; ++i) {
    const double li = c->lam_h[f * i];
    if (c->cplx && !(std::fabs(c->lam_h[f * i + 1] - li) <= 1e-6 * std::max(1.0, std::fabs(li))))
      return PPCG_ERR_NUMERIC;   // the real form's eigenvalues must come in equal pairs
    lambda[i] = li;
    const double r = std::sqrt(c->nrm_h[f * i]);
    if (resnorm) resnorm[i] = r;
    if (!std::isfinite(r)) return PPCG_ERR_NUMERIC;
    mx = std::max(mx, r);
  }
  S->iters = it;
  S->n_locked = st.k_lock;
  S->n_drop_p = c->counters_h[0];
  S->n_stall = c->counters_h[1];
  S->converged = st.done ? 1 : 0;
  S->max_res = mx;
  S->kernel_launches = launch_count() - launches0;
  S->n_eig_diagonal = c->eig_count[1];
  S->n_eig_refined = c->eig_count[2];
  S->n_eig_mixed = c->eig_count[3];
  for (int i = 0; i < 8; ++i) S->t_phase_ms[i] = c->t_ms[i];
  return st.done ? PPCG_OK : PPCG_ERR_NOT_CONVERGED;
}

// ---------------------------------------------------------------------------------------------- step API
ppcg_status ppcg_apply_operator(ppcg_handle c, const double* X, int64_t ldx, double* Y, int64_t ldy, int32_t m) {
  if (!c || !X || !Y || m < 0 || ldx < c->n || ldy < c->n) return PPCG_ERR_ARG;
  return apply_H(c, X, ldx, Y, ldy, m);
}

ppcg_status ppcg_gram(ppcg_handle c, const double* A, int64_t lda, const double* B, int64_t ldb, int32_t ma,
                      int32_t mb, double* C) {
  if (!c || !A || !B || !C || ma < 1 || mb < 1 || ma > c->kt || mb > c->kt || lda < c->n || ldb < c->n)
    return PPCG_ERR_ARG;
  if (c->mixed) return gram_tc(c, A, lda, B, ldb, ma, mb, C, ma);
  return gram(c, A, lda, B, ldb, ma, mb, C, ma);
}

ppcg_status ppcg_project(ppcg_handle c, const double* X, int64_t ldx, int32_t mx, double* Y, int64_t ldy,
                         int32_t my) {
  if (!c || !X || !Y || mx < 0 || my < 0 || mx > c->kt || my > c->kt || ldx < c->n || ldy < c->n)
    return PPCG_ERR_ARG;
  return project(c, X, ldx, mx, Y, ldy, my);
}

ppcg_status ppcg_cholqr2(ppcg_handle c, double* X, int64_t ldx, int32_t m, int32_t* fallback) {
  if (!c || !X || m < 1 || m > c->kt || ldx < c->n) return PPCG_ERR_ARG;
  int fb = 0;
  ppcg_status st = cholqr2(c, X, ldx, c->Xs, c->ld, m, &fb);
  if (fallback) *fallback = fb;
  return st;
}

ppcg_status ppcg_dense_eigh(ppcg_handle c, const double* M, int32_t m, double* lambda, double* C) {
  if (!c || !M || !lambda || !C || m < 1 || m > c->kt) return PPCG_ERR_ARG;
  CK(cudaMemsetAsync(c->tcflag, 0, sizeof(int), c->stream));
  PS(dense_eigh(c, M, m, lambda, C));
  c->last_sweeps = last_sweeps(c);
  const int f = read_flag(c);
  int ft = 0;
  CK(cudaMemcpyAsync(&ft, c->tcflag, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  if (f < 0) return PPCG_ERR_CUDA;
  if ((f | ft) & kFlagTimeout) return PPCG_ERR_TIMEOUT;
  return PPCG_OK;
}

ppcg_status ppcg_barrier_timeout_check(ppcg_handle c, int32_t spin_polls) {
  if (!c || spin_polls < 32) return PPCG_ERR_ARG;
  CK(cudaMemsetAsync(c->iflag, 0, sizeof(int), c->stream));
  CK(barrier_timeout_probe(spin_polls, c->iflag, c->bar, c->stream));
  const int f = read_flag(c);
  if (f < 0) return PPCG_ERR_CUDA;
  return (f & kFlagTimeout) ? PPCG_ERR_TIMEOUT : PPCG_OK;
}

ppcg_status ppcg_block_coefficients(ppcg_handle c, const double* X, const double* W, const double* P,
                                    const double* HX, const double* HW, const double* HP, int64_t ld,
                                    int32_t k_act, int32_t has_p, double* coef, int32_t* flags) {
  if (!c || !X || !W || !HX || !HW || !coef || k_act < 1 || k_act > c->kt || ld < c->n) return PPCG_ERR_ARG;
  if (has_p && (!P || !HP)) return PPCG_ERR_ARG;
  BlockArgs ba{X, W, has_p ? P : W, HX, HW, has_p ? HP : HW, ld, c->n, k_act, c->q, has_p ? 1 : 0};
  int nchunk = 0;
  CK(block_gram(ba, c->bpart, c->bpart_cap, &nchunk, c->stream));
  CK(block_solve(ba, c->bpart, nchunk, coef, flags ? flags : c->bflags, c->icnt, c->stream));
  return PPCG_OK;
}

ppcg_status ppcg_block_update(ppcg_handle c, double* X, const double* W, double* P, int64_t ld, int32_t k_act,
                              int32_t has_p, const double* coef) {
  if (!c || !X || !W || !P || !coef || k_act < 1 || k_act > c->kt || ld < c->n) return PPCG_ERR_ARG;
  CK(block_update(X, W, P, ld, c->n, k_act, c->q, has_p ? 1 : 0, coef, c->stream));
  return PPCG_OK;
}

ppcg_status ppcg_residual(ppcg_handle c, const double* X, const double* HX, int64_t ld, int32_t m, const double* M,
                          const double* lam, double sigma, double* W, double* colnorm2) {
  if (!c || !X || !HX || !W || !colnorm2 || m < 1 || m > c->kt || ld < c->n) return PPCG_ERR_ARG;
  if (!M && !lam) return PPCG_ERR_ARG;
  ResidualArgs ra = resid_args(c, sigma);
  if (M) PS(residual_m(c, X, HX, ld, m, M, ra, W));
  else CK(residual_diag(X, HX, ld, c->n, m, lam, ra, W, c->stream));
  CK(reduce_colnorms(c->normpart, norm_row_tiles(c->n), m, colnorm2, c->stream));
  return PPCG_OK;
}

ppcg_status ppcg_energy_gradient(ppcg_handle c, const double* X, int64_t ld, int32_t k, double scale,
                                 double* grad_V) {
  if (!c || !X || !grad_V || k < 1 || ld < c->ng || !std::isfinite(scale)) return PPCG_ERR_ARG;
  if (c->cplx) CK(density_c(X, ld, c->ng, k, scale, grad_V, c->stream));
  else CK(density(X, ld, c->n, k, scale, grad_V, c->stream));
  return PPCG_OK;
}

}  // extern "C"

// ------------------------------------------------------------------------------------------ batched solves
extern "C" ppcg_status ppcg_solve_batched(ppcg_batch_item* items, int32_t count, int32_t max_concurrent) {
  if (!items || count < 0) return PPCG_ERR_ARG;
  for (int i = 0; i < count; ++i)
    if (!items[i].h) return PPCG_ERR_ARG;
  if (count == 0) return PPCG_OK;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return PPCG_ERR_CUDA;
  int workers = max_concurrent > 0 ? max_concurrent : 16;
  if (workers > count) workers = count;
  std::atomic<int> next{0};
  auto work = [&]() {
    cudaSetDevice(dev);
    for (int i = next.fetch_add(1); i < count; i = next.fetch_add(1)) {
      ppcg_batch_item& it = items[i];
      const auto t0 = std::chrono::steady_clock::now();
      it.status = ppcg_solve(it.h, it.X0, it.tol, it.lambda, it.X, it.resnorm, it.stats);
      it.time_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    }
  };
  std::vector<std::thread> pool;
  pool.reserve(workers > 1 ? workers - 1 : 0);
  for (int w = 1; w < workers; ++w) pool.emplace_back(work);
  work();
  for (auto& t : pool) t.join();
  for (int i = 0; i < count; ++i)
    if (items[i].status != PPCG_OK) return (ppcg_status)items[i].status;
  return PPCG_OK;
}

extern "C" ppcg_status ppcg_autotune_sbsize(const ppcg_operator* op, int64_t n, int32_t k, int32_t rr_period,
                                            const ppcg_options* opt, const double* X0, double tol,
                                            const int32_t* candidates, int32_t ncand, void* cuda_stream,
                                            int32_t* best, double* time_ms) {
  if (!op || !X0 || !candidates || ncand < 1 || !best || !(tol > 0.0)) return PPCG_ERR_ARG;
  const int nbuf = opt ? opt->nbuf : 0;
  std::vector<double> lam((size_t)k), res((size_t)k);
  double* Xout = nullptr;
  if (cudaMalloc(&Xout, sizeof(double) * (size_t)n * k) != cudaSuccess) return PPCG_ERR_OOM;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  ppcg_status last = PPCG_ERR_ARG;
  double best_ms = -1.0;
  *best = 0;
  for (int i = 0; i < ncand; ++i) {
    const int q = candidates[i];
    if (time_ms) time_ms[i] = -1.0;
    if (q < 1 || q > kMaxSbsize || q > k + nbuf) continue;
    ppcg_handle h = nullptr;
    last = ppcg_create(op, n, k, q, rr_period, opt, cuda_stream, nullptr, 0, &h);
    if (last != PPCG_OK) continue;
    cudaEventRecord(e0, s);
    last = ppcg_solve(h, X0, tol, lam.data(), Xout, res.data(), nullptr);
    cudaEventRecord(e1, s);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    ppcg_destroy(h);
    if (last != PPCG_OK) continue;
    if (time_ms) time_ms[i] = ms;
    if (best_ms < 0.0 || ms < best_ms) {
      best_ms = ms;
      *best = q;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(Xout);
  return best_ms >= 0.0 ? PPCG_OK : last;
}
