// Dense k x k kernels of Algorithm 3 (the ScaLAPACK part of Section 6):
//   chol_inv     R^{-1} for the Cholesky factor of the Gram X^T X = R^T R (CholQR, Section 5.5, steps 18-19):
//                blocked right-looking Cholesky on 32 x 32 tiles with the inverse of L = R^T formed in the
//                same sweep; one cooperative persistent kernel, quarter-tile tasks spread over the CTAs.
//   jacobi_eigh  eigen-decomposition of the projected matrix of the Rayleigh-Ritz step (steps 23-24,
//                Section 5.6): parallel cyclic Jacobi with round-robin pairing. In every round each 2 x 2 block
//                of A is rotated from both sides independently (ping-pong buffers), each CTA recomputing the
//                rotations it needs from the previous round's matrix, so one grid barrier separates rounds.
// On GB300 FP64 is scarce (2 DFMA lanes per clock per SM); these kernels spread the O(k^3) work over all SMs
// instead of one process grid. Every device-side wait is bounded: a barrier that gives up sets kFlagTimeout
// and every CTA returns.
#include "ppcg_internal.h"

#include <cmath>
#include <math_constants.h>
#include <mutex>

namespace ppcg {

namespace {

constexpr int TB = 32;
constexpr long long kSpinLimit = 1LL << 22;   // polls of ~0.3-1 us: a wait longer than ~1-4 s is an error

// GPU-scope memory operations. (A volatile load is a relaxed load at system scope; on a CPU-coherent
// Grace-Blackwell node that scope is far more expensive than the GPU scope these barriers need.)
__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ int ld_relaxed_gpu(const int* p) {
  int v;
  asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void red_release_gpu(unsigned* p, unsigned v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" :: "l"(p), "r"(v) : "memory");
}

// Software grid barrier for cooperative launches (all CTAs co-resident). bar[0] counts arrivals over the whole
// launch and is never reset, so barrier number g is passed once it reaches g * nblocks: arriving is one
// fire-and-forget release add and waiting is polling with acquire loads (no return trip on arrival, no release
// store by a last arriver). Every CTA tracks g locally in `gen`. The wait is bounded: after kSpinLimit polls the
// CTA sets kFlagTimeout and every CTA returns false.
__device__ bool grid_sync(unsigned* bar, unsigned nblocks, int* flag, unsigned& gen,
                          long long spin_limit = kSpinLimit) {
  __shared__ int ok;
  gen += 1u;
  __syncthreads();
  if (threadIdx.x == 0) {
    // The CTA barrier above orders every thread's writes before this release add, and release is cumulative, so
    // they are visible at GPU scope to any CTA whose acquire load observes the count; the CTA barrier below orders
    // that acquire before every thread's later reads.
    const unsigned target = gen * nblocks;
    red_release_gpu(bar, 1u);
    int good = 1;
    long long spins = 0;
    while ((int)(ld_acquire_gpu(bar) - target) < 0) {
      if ((++spins & 31) == 0 && (spins > spin_limit || (ld_relaxed_gpu(flag) & kFlagTimeout))) {
        atomicOr(flag, kFlagTimeout);
        good = 0;
        break;
      }
    }
    if (ld_relaxed_gpu(flag) & kFlagTimeout) good = 0;
    ok = good;
  }
  __syncthreads();
  return ok != 0;
}

// ------------------------------------------------------------------------------------------- Cholesky
// Blocked right-looking Cholesky of the padded matrix A = [G + shift I, 0; 0, I] = L L^T on 32 x 32 tiles, with
// the inverse Y = L^{-1} formed in the same sweep by blocked forward substitution on an identity right-hand side
// B: at step kk, Y_kk,: = L_kk^{-1} B_kk,: and B_i,: -= L_ik Y_kk,: for i > kk. Each step is two phases separated
// by grid barriers:
//   P (panel)    L_ik = A_ik L_kk^{-T} (i > kk) into a panel buffer, and Y_kk,j = L_kk^{-1} B_kk,j (j <= kk);
//                every CTA with a task factors the diagonal tile A_kk itself, so no barrier separates the
//                factorization of A_kk from its use;
//   U (update)   A_ij -= L_ik L_jk^T (kk < j <= i) and B_ij -= L_ik Y_kk,j (i > kk, j <= kk).
// Tasks are quarter tiles (32 rows x 8 columns, one output per thread). The diagonal tile is factored as
// L1 D L1^T by Gaussian elimination that applies the same row operations to an identity (B1 = L1^{-1}), then
// L_kk^{-1} = D^{-1/2} B1; one block barrier per column, with the next pivot's reciprocal formed by the thread that
// finished that pivot.
__device__ void load_tile(const double* M, int ld, int ti, int tj, double (*s)[TB + 1]) {
  for (int e = threadIdx.x; e < TB * TB; e += blockDim.x) {
    const int r = e % TB, c = e / TB;
    s[r][c] = __ldcg(M + (int64_t)(ti * TB + r) + (int64_t)(tj * TB + c) * ld);
  }
}

__device__ __forceinline__ void tile_pivot(double (*a)[TB + 1], double* sinv, int c, double g0, int* flag) {
  double d = a[c][c];
  if (!(d > 0.0 && d >= kCholPivotTol * kCholPivotTol * g0)) {
    atomicOr(flag, kFlagCholBreakdown);
    if (!(d > 0.0)) { d = 1.0; a[c][c] = 1.0; }
  }
  sinv[c] = __drcp_rn(d);
}

// a: the symmetric diagonal tile (lower triangle used, overwritten); dinv receives L_kk^{-1} (lower triangular).
__device__ void factor_tile(double (*a)[TB + 1], double (*dinv)[TB + 1], double* sinv, const double* diag0,
                            int* flag) {
  const int t = threadIdx.x, lane = t & 31, w = t >> 5, nw = blockDim.x >> 5;
  for (int e = t; e < TB * TB; e += blockDim.x) dinv[e % TB][e / TB] = (e % TB == e / TB) ? 1.0 : 0.0;
  if (t == 0) tile_pivot(a, sinv, 0, __ldcg(diag0), flag);
  __syncthreads();
  for (int c = 0; c < TB; ++c) {
    const double ic = sinv[c];
    for (int r = c + 1 + w; r < TB; r += nw) {
      const double l = a[r][c] * ic;                 // multiplier of row c in row r
      const int j = lane;
      if (j <= r) {
        if (j > c) a[r][j] = fma(-l, a[j][c], a[r][j]);
        else       dinv[r][j] = fma(-l, dinv[c][j], dinv[r][j]);
      }
    }
    if (w == 0 && lane == c + 1) tile_pivot(a, sinv, c + 1, __ldcg(diag0 + c + 1), flag);
    __syncthreads();
  }
  if (t < TB) sinv[t] = rsqrt(a[t][t]);              // D^{-1/2}
  __syncthreads();
  for (int e = t; e < TB * TB; e += blockDim.x) {
    const int r = e % TB, j = e / TB;
    dinv[r][j] = (j <= r) ? dinv[r][j] * sinv[r] : 0.0;
  }
  __syncthreads();
}

__global__ void __launch_bounds__(256)
chol_inv_kernel(const double* __restrict__ G, int m, int mp, double shift, double* __restrict__ Rinv,
                double* Lw, double* Linv, double* Lp, double* diag0, int* flag, unsigned* bar) {
  const int T = mp / TB;
  const unsigned nb = gridDim.x;
  const int t = threadIdx.x;
  const int rr = t % TB, cq = t / TB;                // quarter-tile coordinates: row, column within the quarter
  unsigned gen = 0;
  __shared__ double s1[TB][TB + 1], s2[TB][TB + 1], s3[TB][TB + 1];
  __shared__ double sinv[TB];
  // A = [G + shift I, 0; 0, I] (lower tiles are used), B = 0 below the diagonal tiles
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + t; e < (int64_t)mp * mp; e += (int64_t)nb * blockDim.x) {
    const int i = (int)(e % mp), j = (int)(e / mp);
    double v;
    if (i < m && j < m) {
      v = G[(i < j ? i : j) + (int64_t)(i < j ? j : i) * m];
      if (i == j) v += shift;
    } else {
      v = (i == j) ? 1.0 : 0.0;
    }
    Lw[e] = v;
    Linv[e] = 0.0;
    if (i == j) diag0[i] = v;
  }
  if (!grid_sync(bar, nb, flag, gen)) return;
  for (int kk = 0; kk < T; ++kk) {
    // ---- P: factor A_kk (per CTA), panel L_ik = A_ik Dinv^T into Lp, Y_kk,j = Dinv B_kk,j
    const int np = 4 * T;
    if ((int)blockIdx.x < np) {
      load_tile(Lw, mp, kk, kk, s1);
      __syncthreads();
      factor_tile(s1, s2, sinv, diag0 + kk * TB, flag);      // s2 = Dinv
      for (int task = blockIdx.x; task < np; task += nb) {
        const int q = task & 3, u = task >> 2;
        const int c = q * 8 + cq;                            // column within the tile
        if (kk + 1 + u < T) {
          const int i = kk + 1 + u;
          load_tile(Lw, mp, i, kk, s3);
          __syncthreads();
          double v = 0.0;
          for (int l = 0; l <= c; ++l) v = fma(s3[rr][l], s2[c][l], v);
          Lp[(int64_t)i * TB + rr + (int64_t)c * mp] = v;
          __syncthreads();
        } else {
          const int j = u - (T - kk - 1);                    // 0..kk
          double* Yt = Linv + (int64_t)kk * TB + (int64_t)j * TB * mp;
          double v;
          if (j == kk) {
            v = s2[rr][c];
          } else {
            s3[rr][cq] = __ldcg(Yt + rr + (int64_t)c * mp);  // B_kk,j column c
            __syncthreads();
            v = 0.0;
            for (int l = 0; l <= rr; ++l) v = fma(s2[rr][l], s3[l][cq], v);
            __syncthreads();
          }
          Yt[rr + (int64_t)c * mp] = v;
        }
      }
    }
    if (!grid_sync(bar, nb, flag, gen)) return;
    if (kk == T - 1) break;
    // ---- U: A_ij -= L_ik L_jk^T (kk < j <= i), B_ij -= L_ik Y_kk,j (i > kk, j <= kk)
    const int R = T - kk - 1;
    const int na = 4 * (R * (R + 1) / 2), nbt = 4 * R * (kk + 1);
    for (int task = blockIdx.x; task < na + nbt; task += nb) {
      const int q = task & 3;
      const int c = q * 8 + cq;
      int i, j;
      bool is_a;
      if (task < na) {
        const int tt = task >> 2;
        int x = 0;
        while ((x + 1) * (x + 2) / 2 <= tt) ++x;
        i = kk + 1 + x;
        j = kk + 1 + (tt - x * (x + 1) / 2);
        is_a = true;
      } else {
        const int tt = (task - na) >> 2;
        i = kk + 1 + tt % R;
        j = tt / R;
        is_a = false;
      }
      // s1 = L_ik (panel), s3[:, 0:8] = the 8 needed columns of L_jk^T or Y_kk,j
      for (int e = t; e < TB * TB; e += blockDim.x) s1[e % TB][e / TB] = __ldcg(Lp + (int64_t)i * TB + e % TB + (int64_t)(e / TB) * mp);
      if (is_a) {
        for (int e = t; e < TB * 8; e += blockDim.x) {
          const int l = e % TB, cc = e / TB;                 // s3[l][cc] = L_jk[q*8+cc][l]
          s3[l][cc] = __ldcg(Lp + (int64_t)j * TB + q * 8 + cc + (int64_t)l * mp);
        }
      } else {
        for (int e = t; e < TB * 8; e += blockDim.x) {
          const int l = e % TB, cc = e / TB;                 // s3[l][cc] = Y_kk,j[l][q*8+cc]
          s3[l][cc] = __ldcg(Linv + (int64_t)kk * TB + l + (int64_t)(j * TB + q * 8 + cc) * mp);
        }
      }
      __syncthreads();
      double v = 0.0;
      for (int l = 0; l < TB; ++l) v = fma(s1[rr][l], s3[l][cq], v);
      double* dst = (is_a ? Lw : Linv) + (int64_t)i * TB + rr + (int64_t)(j * TB + c) * mp;
      *dst = __ldcg(dst) - v;
      __syncthreads();
    }
    if (!grid_sync(bar, nb, flag, gen)) return;
  }
  // R^{-1} = (L^{-1})^T, upper triangular, leading dimension m
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + t; e < (int64_t)m * m; e += (int64_t)nb * blockDim.x) {
    const int r = (int)(e % m), c = (int)(e / m);
    Rinv[e] = (r <= c) ? __ldcg(Linv + c + (int64_t)r * mp) : 0.0;
  }
}

// ------------------------------------------------------------------------------------------- Jacobi
// The matrix is kept in "slot order": in every round slot t is paired with slot mp-1-t (the circle method of
// round-robin scheduling with mirrored seats). After a round, slots 1..mp-1 shift by one (slot 0 stays), which is
// the next round's pairing; the round writes its output directly at the shifted slots, so every 2 x 2 block load
// and every store is coalesced. mp - 1 shifts form a full cycle, so the layout is the identity again at the end of
// every sweep. Dg[t] and Od[t] hold A[t][t] and A[t][mp-1-t] of the current layout (written by the previous round)
// so that rotation parameters are read from compact arrays. mp is m padded to a multiple of 32 with zero rows and
// columns, which never rotate (their pair entries are exactly zero) and never mix with the real ones.
//
// Work of one round is cut into tiles of 256 threads: A tiles of 16 row pairs x 16 column pairs (one 2 x 2 block
// per thread) and V tiles of 64 rows x 16 column pairs. A tile needs 32 rotations and a V tile 16; one warp
// computes them into shared memory while the other threads load their blocks, so each rotation is formed once per
// tile instead of once per block.
//
// The kernel runs in FP64 (the eigensolve of last resort, accurate to a few ulps of ||A||) and in FP32, where it
// only supplies the starting eigenvectors of the FP64 refinement below: FP32 arithmetic runs on the 64x wider FP32
// pipe, and the matrix and vectors take half the memory traffic.
constexpr int JR = 16;   // row pairs per A tile
constexpr int JC = 16;   // column pairs per A tile and per V tile
constexpr int JV = 64;   // rows per V tile

__device__ __forceinline__ int slot_shift(int t, int mp) { return t == 0 ? 0 : (t == mp - 1 ? 1 : t + 1); }

// FP64 rotation (c, s) that annihilates apq approximately: t = tan(phi) from a single-precision solve of
// t^2 + 2 theta t - 1 = 0, theta = (aqq - app) / (2 apq), then c = 1/sqrt(1 + t^2) refined by two FP64 Newton
// steps and s = t c, so that c^2 + s^2 = 1 to FP64 rounding and the rotation is an exact orthogonal similarity.
// theta is divided in single precision from operands scaled by inv = 1/||A||_F: |aqq - app| inv <= 2 and
// |2 apq| inv > 2e-14 whenever a rotation is made, well inside the single-precision range. (FP64 division and
// square root are long instruction sequences on GB300's 2-lane-per-clock FP64 pipe; the residual
// a'_pq ~ 1e-7 |apq| left by the single-precision angle is removed by later sweeps.)
__device__ __forceinline__ void rot_from(double app, double aqq, double apq, double thr, double inv, double& c,
                                         double& s) {
  c = 1.0; s = 0.0;
  if (!(fabs(apq) > thr)) return;
  const float num = (float)((aqq - app) * inv);
  const float den = (float)((apq + apq) * inv);
  const float th = num / den;
  const float at = fabsf(th);
  float tf = at > 1e18f ? 0.5f / at : 1.0f / (at + sqrtf(fmaf(at, at, 1.0f)));
  if (th < 0.0f) tf = -tf;
  const double t = (double)tf;
  const double q = fma(t, t, 1.0);                   // 1 + t^2
  double r = (double)rsqrtf((float)q);               // ~1e-7
  r = r * fma(-0.5 * q, r * r, 1.5);                 // ~1e-14
  r = r * fma(-0.5 * q, r * r, 1.5);                 // ~1 ulp
  c = r;
  s = t * r;
}

// FP32 rotation: the same angle, all in single precision
__device__ __forceinline__ void rot_from(float app, float aqq, float apq, float thr, float, float& c, float& s) {
  c = 1.0f; s = 0.0f;
  if (!(fabsf(apq) > thr)) return;
  const float th = (aqq - app) / (apq + apq);
  const float at = fabsf(th);
  float t = at > 1e18f ? 0.5f / at : 1.0f / (at + sqrtf(fmaf(at, at, 1.0f)));
  if (th < 0.0f) t = -t;
  c = rsqrtf(fmaf(t, t, 1.0f));
  s = t * c;
}

template <typename T>
__global__ void jacobi_init_kernel(const double* __restrict__ M, int m, int mp, T* A0, T* V0, T* Dg, T* Od) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)mp * mp;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % mp), j = (int)(e / mp);
    const T v = (T)((i < m && j < m) ? M[(i < j ? i : j) + (int64_t)(i < j ? j : i) * m] : 0.0);
    A0[e] = v;
    V0[e] = (T)((i == j) ? 1.0 : 0.0);
    if (i == j) Dg[i] = v;
    if (i + j == mp - 1 && i < j) Od[i] = v;
  }
}

template <typename T>
__global__ void frob_kernel(const T* __restrict__ A, int64_t cnt, double* out) {
  double s = 0.0;
  for (int64_t e = threadIdx.x; e < cnt; e += blockDim.x) s += (double)A[e] * (double)A[e];
  __shared__ double red[1024];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int off = blockDim.x / 2; off > 0; off >>= 1) {
    if ((int)threadIdx.x < off) red[threadIdx.x] += red[threadIdx.x + off];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = sqrt(red[0]);
}

template <typename T>
struct JacBuf {
  T *A[2], *V[2], *Dg[2], *Od[2];
};

// Sweeps until the matrix left by a sweep has no off-diagonal entry above tol ||A||_F (then the next sweep would
// rotate nothing, so it is not run), at most max_sweeps. The test is taken in the last round of each sweep, whose
// output is the whole matrix in identity layout. Only the FP64 kernel reports non-convergence: the FP32 result is
// a starting point whose accuracy the refinement measures itself.
template <typename T>
__global__ void __launch_bounds__(256)
jacobi_kernel(JacBuf<T> b, int m, int mp, const double* normA, double tol, int max_sweeps, int* counts, int* flag,
              unsigned* bar, int* info) {
  const double nrm = normA[0];
  const T thr = (T)(tol * nrm);
  const T inv = (T)(nrm > 0.0 ? 1.0 / nrm : 0.0);
  const int P = mp / 2;
  const int TA = P / JR;
  const int nTA = TA * TA;
  const int nVR = (mp + JV - 1) / JV;
  const int nT = nTA + nVR * (P / JC);
  const unsigned nb = gridDim.x;
  const int t = threadIdx.x;
  __shared__ T rc[JR + JC], rs[JR + JC];
  int cur = 0;
  int sweep = 0;
  bool converged = false;
  unsigned gen = 0;
  while (sweep < max_sweeps && !converged) {
    for (int r = 0; r < mp - 1; ++r) {
      const bool last = (r == mp - 2);
      const T* __restrict__ A = cur ? b.A[1] : b.A[0];
      T* __restrict__ An = cur ? b.A[0] : b.A[1];
      const T* __restrict__ V = cur ? b.V[1] : b.V[0];
      T* __restrict__ Vn = cur ? b.V[0] : b.V[1];
      const T* __restrict__ Dg = cur ? b.Dg[1] : b.Dg[0];
      const T* __restrict__ Od = cur ? b.Od[1] : b.Od[0];
      T* __restrict__ Dn = cur ? b.Dg[0] : b.Dg[1];
      T* __restrict__ On = cur ? b.Od[0] : b.Od[1];
      int big = 0;
      for (int tile = blockIdx.x; tile < nT; tile += nb) {
        if (tile < nTA) {
          const int R0 = (tile % TA) * JR, C0 = (tile / TA) * JC;
          const int ri = R0 + (t % JR), ci = C0 + (t / JR);   // row pair ri, column pair ci
          const int rb = mp - 1 - ri, cb = mp - 1 - ci;
          T x00, x01, x10, x11;             // rows (ri, rb) x cols (ci, cb)
          if (ri == ci) {
            x00 = __ldcg(Dg + ri); x11 = __ldcg(Dg + rb); x01 = __ldcg(Od + ri); x10 = x01;
          } else {
            x00 = __ldcg(A + ri + (int64_t)ci * mp); x10 = __ldcg(A + rb + (int64_t)ci * mp);
            x01 = __ldcg(A + ri + (int64_t)cb * mp); x11 = __ldcg(A + rb + (int64_t)cb * mp);
          }
          if (t < JR + JC) {
            const int p = t < JR ? R0 + t : C0 + (t - JR);
            T c, s;
            rot_from(__ldcg(Dg + p), __ldcg(Dg + mp - 1 - p), __ldcg(Od + p), thr, inv, c, s);
            rc[t] = c;
            rs[t] = s;
          }
          __syncthreads();
          const T cr = rc[t % JR], sr = rs[t % JR], cc = rc[JR + t / JR], sc = rs[JR + t / JR];
          const T y00 = cr * x00 - sr * x10, y01 = cr * x01 - sr * x11;
          const T y10 = sr * x00 + cr * x10, y11 = sr * x01 + cr * x11;
          T z00 = cc * y00 - sc * y01, z01 = sc * y00 + cc * y01;
          T z10 = cc * y10 - sc * y11, z11 = sc * y10 + cc * y11;
          if (ri == ci) z10 = z01;                   // keep the diagonal block exactly symmetric
          const int R0s = slot_shift(ri, mp), R1s = slot_shift(rb, mp);
          const int C0s = slot_shift(ci, mp), C1s = slot_shift(cb, mp);
          An[R0s + (int64_t)C0s * mp] = z00;
          An[R1s + (int64_t)C0s * mp] = z10;
          An[R0s + (int64_t)C1s * mp] = z01;
          An[R1s + (int64_t)C1s * mp] = z11;
          // next round's diagonal and pair entries
          if (R0s == C0s) Dn[R0s] = z00;
          if (R1s == C1s) Dn[R1s] = z11;
          if (R0s == C1s) Dn[R0s] = z01;
          if (R1s == C0s) Dn[R1s] = z10;
          if (R0s + C0s == mp - 1 && R0s < C0s) On[R0s] = z00;
          if (R1s + C0s == mp - 1 && R1s < C0s) On[R1s] = z10;
          if (R0s + C1s == mp - 1 && R0s < C1s) On[R0s] = z01;
          if (R1s + C1s == mp - 1 && R1s < C1s) On[R1s] = z11;
          if (last) {
            big |= (R0s != C0s && fabs(z00) > thr) | (R1s != C0s && fabs(z10) > thr) |
                   (R0s != C1s && fabs(z01) > thr) | (R1s != C1s && fabs(z11) > thr);
          }
          __syncthreads();                           // rc/rs are reused by the next tile
        } else {
          const int v = tile - nTA;
          const int R0 = (v % nVR) * JV, C0 = (v / nVR) * JC;
          const int ci = C0 + t / 16, cb = mp - 1 - ci;
          T vu[JV / 16], vv[JV / 16];
#pragma unroll
          for (int j = 0; j < JV / 16; ++j) {
            const int row = R0 + (t % 16) + 16 * j;
            vu[j] = row < mp ? __ldcg(V + row + (int64_t)ci * mp) : (T)0;
            vv[j] = row < mp ? __ldcg(V + row + (int64_t)cb * mp) : (T)0;
          }
          if (t < JC) {
            const int p = C0 + t;
            T c, s;
            rot_from(__ldcg(Dg + p), __ldcg(Dg + mp - 1 - p), __ldcg(Od + p), thr, inv, c, s);
            rc[t] = c;
            rs[t] = s;
          }
          __syncthreads();
          const T cc = rc[t / 16], sc = rs[t / 16];
          const int c0 = slot_shift(ci, mp), c1 = slot_shift(cb, mp);
#pragma unroll
          for (int j = 0; j < JV / 16; ++j) {
            const int row = R0 + (t % 16) + 16 * j;
            if (row < mp) {
              Vn[row + (int64_t)c0 * mp] = cc * vu[j] - sc * vv[j];
              Vn[row + (int64_t)c1 * mp] = sc * vu[j] + cc * vv[j];
            }
          }
          __syncthreads();
        }
      }
      if (last && __syncthreads_or(big) && t == 0) atomicOr(counts + sweep, 1);
      if (!grid_sync(bar, nb, flag, gen)) return;
      cur ^= 1;
    }
    converged = ld_relaxed_gpu(counts + sweep) == 0;
    ++sweep;
  }
  if (blockIdx.x == 0 && t == 0) {
    info[0] = sweep;                                 // sweeps run
    info[1] = cur;
    if (!converged && sizeof(T) == sizeof(double)) atomicOr(flag, kFlagJacobiNoConv);
  }
}

// lambda ascending; C[:, rank(i)] = V[0:m, i]. The layout is the identity at a sweep boundary.
__global__ void jacobi_sort_kernel(JacBuf<double> b, int m, int mp, const int* info, double* lambda, int* perm) {
  const double* A = b.A[info[1]];
  // rank by the strict total order (value, index) with NaN as +inf, so perm is always a permutation
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
    const double li = A[i + (int64_t)i * mp];
    const double ki = isnan(li) ? CUDART_INF : li;
    int rank = 0;
    for (int l = 0; l < m; ++l) {
      const double ll = A[l + (int64_t)l * mp];
      const double kl = isnan(ll) ? CUDART_INF : ll;
      rank += (kl < ki || (kl == ki && l < i)) ? 1 : 0;
    }
    lambda[rank] = li;
    perm[rank] = i;
  }
}

__global__ void jacobi_gather_kernel(JacBuf<double> b, int m, int mp, const int* info, const int* perm, double* C) {
  const double* V = b.V[info[1]];
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)m * m;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(e % m), c = (int)(e / m);
    C[e] = V[r + (int64_t)perm[c] * mp];
  }
}

// Z (m x m, FP64) = the FP32 Jacobi eigenvectors (unsorted; the refinement orders them itself)
__global__ void jacobi32_to_z_kernel(JacBuf<float> b, int m, int mp, const int* info, double* Z) {
  const float* V = b.V[info[1]];
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)m * m;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(e % m), c = (int)(e / m);
    Z[e] = (double)V[r + (int64_t)c * mp];
  }
}

// ------------------------------------------------------------------------------- nearly diagonal matrices
// Msym = M with its lower triangle taken from the upper one (the eigensolvers read the upper triangle)
__global__ void symmetrize_kernel(const double* __restrict__ M, int m, double* __restrict__ Msym) {
  const int64_t cnt = (int64_t)m * m;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < cnt; e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % m), j = (int)(e / m);
    Msym[e] = i <= j ? M[e] : M[j + (int64_t)i * m];
  }
}

// ||M||_F and max_{i != j} |M_ij| in two passes with a fixed summation order (repeated calls agree bit for bit):
// each CTA reduces a contiguous range into part[2 b], part[2 b + 1]; one CTA then combines the nb partials in order.
constexpr int kStatBlocks = 256;

__global__ void __launch_bounds__(256) eig_stats_part_kernel(const double* __restrict__ M, int m, double* part) {
  const int64_t cnt = (int64_t)m * m;
  const int64_t per = ceil_div(cnt, (int64_t)gridDim.x);
  const int64_t e0 = (int64_t)blockIdx.x * per, e1 = min(cnt, e0 + per);
  double s = 0.0, mx = 0.0;
  for (int64_t e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
    const double v = M[e];
    s += v * v;
    if (e % m != e / m) mx = fmax(mx, fabs(v));
  }
  __shared__ double rs[256], rm[256];
  rs[threadIdx.x] = s;
  rm[threadIdx.x] = mx;
  __syncthreads();
  for (int off = blockDim.x / 2; off > 0; off >>= 1) {
    if ((int)threadIdx.x < off) {
      rs[threadIdx.x] += rs[threadIdx.x + off];
      rm[threadIdx.x] = fmax(rm[threadIdx.x], rm[threadIdx.x + off]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = rs[0];
    part[2 * blockIdx.x + 1] = rm[0];
  }
}

__global__ void eig_stats_kernel(const double* __restrict__ part, int nb, double* out) {
  if (threadIdx.x != 0) return;
  double s = 0.0, mx = 0.0;
  for (int b = 0; b < nb; ++b) {
    s += part[2 * b];
    mx = fmax(mx, part[2 * b + 1]);
  }
  out[0] = sqrt(s);
  out[1] = mx;
}

// ---------------------------------------------------------------------------------- eigenvector refinement
// One step of the symmetric eigenvector refinement of Ogita and Aishima (2018), with clustered eigenvalues solved
// as small eigenproblems (the idea of their 2019 sequel on clustered eigenvalues). For approximate eigenvectors Z
// (columns), G = Z^T Z, R = I - G and S = Z^T M Z:
//   lam_i = S_ii / (1 - R_ii);
//   for a separated pair i != j: E_ij = (S_ij + lam_j R_ij) / (lam_j - lam_i)   (the first-order correction);
//   E_ii = R_ii / 2                                                               (first-order orthonormalisation);
//   Z <- Z (I + E): the error of Z roughly squares.
// S enters symmetrised, (S_ij + S_ji) / 2: then E_ij + E_ji = R_ij holds exactly, so the orthogonality of the new Z
// does not suffer from the rounding of S divided by small eigenvalue gaps.
// Pairs whose Ritz values are closer than max(kClusterGap x the largest coupling |S_ij + lam_j R_ij|,
// kClusterFloor ||M||_F) would divide by a difference that the coupling or the rounding of S can dwarf. Such values
// are grouped into clusters (runs of the sorted values with small gaps), and each cluster's block of the first-order
// orthonormalised S, B_ab = S_ab + (lam_a + lam_b) R_ab / 2 (B_aa = lam_a), is diagonalised exactly, B = Q D Q^T,
// by a cyclic Jacobi in shared memory. The cluster's columns of I + E are then rotated by Q (so the first-order
// corrections from outside the cluster follow the rotated vectors). A step is accepted once every separated |E_ij|
// is at most kRefineAccept and no cluster pair couples above the FP64 Jacobi threshold (the next error is then of
// order kRefineAccept^2 ||M||).
//
// stat: [0] ||M||_F, [2] largest separated |E_ij| (as bits), [3] largest in-cluster |S_ij| (bits), [4] largest
// coupling (bits), [5] clusters, [6] a cluster larger than kMaxCluster. Non-negative doubles order like their bit
// patterns, so the maxima merge with integer atomics in any order.
__device__ __forceinline__ void atomic_max_nonneg(double* p, double v) {
  if (!(v == v)) v = CUDART_INF;                     // a NaN rejects the step
  atomicMax(reinterpret_cast<unsigned long long*>(p), (unsigned long long)__double_as_longlong(v));
}

__device__ __forceinline__ double r_of(const double* G, int64_t e, int i, int j) {
  return G ? (i == j ? 1.0 : 0.0) - G[e] : 0.0;
}

// lam_i = S_ii / G_ii (G = null: Z = I); resets the step statistics. One CTA.
__global__ void refine_diag_kernel(const double* __restrict__ S, const double* __restrict__ G, int m, double* lam,
                                   double* stat) {
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    const double sii = S[i + (int64_t)i * m];
    lam[i] = G ? sii / G[i + (int64_t)i * m] : sii;
  }
  if (threadIdx.x == 0)
    for (int q = 2; q <= 6; ++q) stat[q] = 0.0;
}

// largest coupling |S_ij + lam_j R_ij|, i != j
__global__ void refine_coupling_kernel(const double* __restrict__ S, const double* __restrict__ G, int m,
                                       const double* __restrict__ lam, double* stat) {
  double mx = 0.0;
  const int64_t cnt = (int64_t)m * m;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < cnt; e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % m), j = (int)(e / m);
    if (i != j) mx = fmax(mx, fabs(0.5 * (S[e] + S[j + (int64_t)i * m]) + lam[j] * r_of(G, e, i, j)));
    else if (!(S[e] == S[e])) mx = CUDART_INF;
  }
  for (int off = 16; off > 0; off >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, off));
  if ((threadIdx.x & 31) == 0) atomic_max_nonneg(stat + 4, mx);
}

// Clusters: with order[r] the index of the r-th smallest lam and ls[r] its value (rank_sort_kernel: strict order
// (value, index), NaN as +inf), cut the sorted sequence where consecutive values differ by more than
// gap = max(kClusterGap x coupling, kClusterFloor ||M||_F), and number the runs of two or more.
// cid[i] = cluster of i or -1; cluster c = order[cls[c] .. cls[c] + cln[c]). One CTA of 1024 threads; the cut
// positions are a bitmask in shared memory (kt <= 65535 columns).
__global__ void __launch_bounds__(1024)
refine_cluster_kernel(const double* __restrict__ ls, const int* __restrict__ order, int m, double* stat, int* cid,
                      int* cls, int* cln) {
  __shared__ unsigned cut[2048];
  const double coupling = stat[4];
  const double gap = fmax(kClusterGap * coupling, kClusterFloor * stat[0]);
  for (int w = threadIdx.x; w < 2048; w += blockDim.x) cut[w] = 0u;
  for (int i = threadIdx.x; i < m; i += blockDim.x) cid[i] = -1;
  __syncthreads();
  for (int r = threadIdx.x; r < m; r += blockDim.x) {
    bool c = true;
    if (r > 0) {
      const double d = ls[r] - ls[r - 1];
      c = !(d <= gap);                               // NaN or inf: a cut
    }
    if (c) atomicOr(&cut[r >> 5], 1u << (r & 31));
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int ncl = 0, big = 0, start = 0;
    for (int r = 1; r <= m; ++r) {
      if (r == m || ((cut[r >> 5] >> (r & 31)) & 1u)) {
        const int len = r - start;
        if (len >= 2) {
          if (len > kMaxCluster) big = 1;
          cls[ncl] = start;
          cln[ncl] = len;
          for (int q = start; q < r; ++q) cid[order[q]] = ncl;
          ++ncl;
        }
        start = r;
      }
    }
    stat[5] = (double)ncl;
    stat[6] = big ? 1.0 : 0.0;
  }
}

// E for every pair outside a cluster block; within a block E = R / 2 until the cluster solve replaces it
__global__ void refine_coef_kernel(const double* __restrict__ S, const double* __restrict__ G, int m,
                                   const double* __restrict__ lam, const int* __restrict__ cid, double thr,
                                   double* stat, double* __restrict__ E) {
  double emax = 0.0, cmax = 0.0;
  const int64_t cnt = (int64_t)m * m;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < cnt; e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % m), j = (int)(e / m);
    const double r = r_of(G, e, i, j);
    const double sij = 0.5 * (S[e] + S[j + (int64_t)i * m]);
    double v;
    if (i == j) {
      v = 0.5 * r;
    } else if (cid[i] >= 0 && cid[i] == cid[j]) {
      v = 0.5 * r;
      cmax = fmax(cmax, fabs(sij) > thr ? fabs(sij) : 0.0);
    } else {
      v = (sij + lam[j] * r) / (lam[j] - lam[i]);
      emax = fmax(emax, fabs(v));
    }
    E[e] = v;
  }
  if (!(emax == emax)) emax = CUDART_INF;
  for (int off = 16; off > 0; off >>= 1) {
    emax = fmax(emax, __shfl_xor_sync(0xffffffffu, emax, off));
    cmax = fmax(cmax, __shfl_xor_sync(0xffffffffu, cmax, off));
  }
  if ((threadIdx.x & 31) == 0) {
    atomic_max_nonneg(stat + 2, emax);
    atomic_max_nonneg(stat + 3, cmax);
  }
}

// One CTA per cluster (blocks beyond the cluster count return): B = the first-order orthonormalised cluster block
// of S, diagonalised by cyclic Jacobi with round-robin pairs (FP64, shared memory); then the cluster's columns of
// I + E, over all m rows, are multiplied by Q.
__global__ void __launch_bounds__(256)
refine_cluster_eig_kernel(const double* __restrict__ S, const double* __restrict__ G, int m,
                          const double* __restrict__ lam, const int* __restrict__ order, const int* __restrict__ cls,
                          const int* __restrict__ cln, const double* __restrict__ stat, double* __restrict__ E) {
  const int c = blockIdx.x;
  if (c >= (int)stat[5] || stat[6] != 0.0) return;
  const int start = cls[c], sz = cln[c];
  const int sp = sz + (sz & 1);                      // padded to an even size (the pad index never rotates)
  __shared__ double B[kMaxCluster][kMaxCluster + 1], Q[kMaxCluster][kMaxCluster + 1];
  __shared__ double rcs[kMaxCluster / 2], rsn[kMaxCluster / 2];
  __shared__ int ra[kMaxCluster / 2], rb[kMaxCluster / 2];
  __shared__ int idx[kMaxCluster];
  __shared__ double offmax;
  const int t = threadIdx.x;
  for (int a = t; a < sz; a += blockDim.x) idx[a] = order[start + a];
  __syncthreads();
  for (int e = t; e < sp * sp; e += blockDim.x) {
    const int a = e % sp, b = e / sp;
    double v = 0.0;
    if (a < sz && b < sz) {
      const int i = idx[a], j = idx[b];
      if (a == b) {
        v = lam[i];
      } else {
        const int64_t eij = i + (int64_t)j * m, eji = j + (int64_t)i * m;
        v = 0.5 * (S[eij] + S[eji]) + 0.5 * (lam[i] + lam[j]) * r_of(G, eij, i, j);
      }
    }
    B[a][b] = v;
    Q[a][b] = (a == b) ? 1.0 : 0.0;
  }
  __syncthreads();
  const int np = sp / 2;
  for (int sweep = 0; sweep < 40; ++sweep) {
    if (t == 0) offmax = 0.0;
    __syncthreads();
    double om = 0.0;
    for (int e = t; e < sp * sp; e += blockDim.x) {
      const int a = e % sp, b = e / sp;
      if (a != b) om = fmax(om, fabs(B[a][b]));
    }
    for (int off = 16; off > 0; off >>= 1) om = fmax(om, __shfl_xor_sync(0xffffffffu, om, off));
    if ((t & 31) == 0) atomic_max_nonneg(&offmax, om);
    __syncthreads();
    double scale = 0.0;
    for (int a = 0; a < sz; ++a) scale = fmax(scale, fabs(B[a][a]));
    if (!(offmax > 1e-17 * scale) || !(offmax == offmax)) break;
    for (int r = 0; r < sp - 1; ++r) {
      if (t < np) {
        // circle method: element 0 fixed, the others rotate by r
        const int pa = t == 0 ? 0 : ((t - 1 + r) % (sp - 1)) + 1;
        const int pb = ((sp - 1 - t - 1 + r) % (sp - 1)) + 1;
        const int a = pa < pb ? pa : pb, b = pa < pb ? pb : pa;
        double cs = 1.0, sn = 0.0;
        const double apq = B[a][b];
        if (b < sz && apq != 0.0) {
          const double th = (B[b][b] - B[a][a]) / (2.0 * apq);
          double tt = 1.0 / (fabs(th) + sqrt(th * th + 1.0));
          if (th < 0.0) tt = -tt;
          cs = 1.0 / sqrt(tt * tt + 1.0);
          sn = tt * cs;
        }
        ra[t] = a; rb[t] = b; rcs[t] = cs; rsn[t] = sn;
      }
      __syncthreads();
      for (int e = t; e < np * sp; e += blockDim.x) {          // rows: B <- J^T B
        const int q = e % np, j = e / np;
        const int a = ra[q], b = rb[q];
        const double x = B[a][j], y = B[b][j];
        B[a][j] = rcs[q] * x - rsn[q] * y;
        B[b][j] = rsn[q] * x + rcs[q] * y;
      }
      __syncthreads();
      for (int e = t; e < np * sp; e += blockDim.x) {          // columns: B <- B J, Q <- Q J
        const int q = e % np, i = e / np;
        const int a = ra[q], b = rb[q];
        const double x = B[i][a], y = B[i][b];
        B[i][a] = rcs[q] * x - rsn[q] * y;
        B[i][b] = rsn[q] * x + rcs[q] * y;
        const double u = Q[i][a], w = Q[i][b];
        Q[i][a] = rcs[q] * u - rsn[q] * w;
        Q[i][b] = rsn[q] * u + rcs[q] * w;
      }
      __syncthreads();
    }
  }
  // F = I + E restricted to the cluster's columns, F <- F Q, row by row (each thread owns whole rows)
  for (int i = t; i < m; i += blockDim.x) {
    double f[kMaxCluster];
#pragma unroll 4
    for (int a = 0; a < sz; ++a) f[a] = E[i + (int64_t)idx[a] * m] + (i == idx[a] ? 1.0 : 0.0);
    for (int b = 0; b < sz; ++b) {
      double acc = 0.0;
      for (int a = 0; a < sz; ++a) acc = fma(f[a], Q[a][b], acc);
      E[i + (int64_t)idx[b] * m] = acc - (i == idx[b] ? 1.0 : 0.0);
    }
  }
}

// Z = I + E (first step, from Z = I)
__global__ void identity_plus_kernel(const double* __restrict__ E, int m, double* __restrict__ Z) {
  const int64_t cnt = (int64_t)m * m;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < cnt; e += (int64_t)gridDim.x * blockDim.x)
    Z[e] = E[e] + ((e % m == e / m) ? 1.0 : 0.0);
}

__global__ void add_kernel(const double* __restrict__ T, int64_t cnt, double* __restrict__ Z) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < cnt; e += (int64_t)gridDim.x * blockDim.x)
    Z[e] += T[e];
}

// Rayleigh quotients lam_i = z_i^T (M z_i) / z_i^T z_i of the accepted vectors (T = M Z); one warp per column
__global__ void rayleigh_quotient_kernel(const double* __restrict__ Z, const double* __restrict__ T, int m,
                                         double* __restrict__ lam) {
  const int col = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  const int lane = threadIdx.x & 31;
  if (col >= m) return;
  double num = 0.0, den = 0.0;
  for (int r = lane; r < m; r += 32) {
    const double z = Z[r + (int64_t)col * m];
    num += z * T[r + (int64_t)col * m];
    den += z * z;
  }
  for (int off = 16; off > 0; off >>= 1) {
    num += __shfl_xor_sync(0xffffffffu, num, off);
    den += __shfl_xor_sync(0xffffffffu, den, off);
  }
  if (lane == 0) lam[col] = num / den;
}

// lambda ascending by the strict total order (value, index), NaN as +inf; perm[rank] = index
__global__ void rank_sort_kernel(const double* __restrict__ v, int64_t stride, int m, double* lambda, int* perm) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
    const double li = v[(int64_t)i * stride];
    const double ki = isnan(li) ? CUDART_INF : li;
    int rank = 0;
    for (int l = 0; l < m; ++l) {
      const double ll = v[(int64_t)l * stride];
      const double kl = isnan(ll) ? CUDART_INF : ll;
      rank += (kl < ki || (kl == ki && l < i)) ? 1 : 0;
    }
    lambda[rank] = li;
    perm[rank] = i;
  }
}

// C[:, r] = Z[:, perm[r]] (Z = null: the identity)
__global__ void gather_perm_kernel(const double* __restrict__ Z, int m, const int* __restrict__ perm, double* C) {
  const int64_t cnt = (int64_t)m * m;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < cnt; e += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(e % m), c = (int)(e / m);
    const int pc = perm[c];
    C[e] = Z ? Z[r + (int64_t)pc * m] : (r == pc ? 1.0 : 0.0);
  }
}

inline unsigned grid_for(int64_t cnt) {
  const int64_t b = ceil_div(cnt, 256);
  return (unsigned)(b < 1 ? 1 : (b < 4096 ? b : 4096));
}

struct CoopLimit {
  int chol = 0, jac = 0, jac32 = 0;
};

const CoopLimit& coop_limits() {
  static const CoopLimit lim = [] {          // initialised once, thread-safe (concurrent batched solves)
    CoopLimit l;
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int per = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, chol_inv_kernel, 256, 0);
    l.chol = (per > 0 ? per : 1) * sms;
    per = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, jacobi_kernel<double>, 256, 0);
    l.jac = (per > 0 ? per : 1) * sms;
    per = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, jacobi_kernel<float>, 256, 0);
    l.jac32 = (per > 0 ? per : 1) * sms;
    return l;
  }();
  return lim;
}

// Cooperative launches from several streams (concurrent solves) are chained: each waits on the event recorded
// after the previous one, so two grid-barrier kernels are never resident together and waiting on each other's
// SMs. The chain only points back to earlier launches, so it cannot form a cycle.
constexpr int kMaxCoopDevices = 64;
std::mutex g_coop_mu;
cudaEvent_t g_coop_ev[kMaxCoopDevices] = {};
bool g_coop_any[kMaxCoopDevices] = {};

cudaError_t coop_launch(const void* fn, unsigned grid, void** args, cudaStream_t s) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxCoopDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_coop_mu);
  if (!g_coop_ev[dev]) {
    e = cudaEventCreateWithFlags(&g_coop_ev[dev], cudaEventDisableTiming);
    if (e != cudaSuccess) return e;
  }
  if (g_coop_any[dev]) {
    e = cudaStreamWaitEvent(s, g_coop_ev[dev], 0);
    if (e != cudaSuccess) return e;
  }
  e = cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(256), args, 0, s);
  if (e != cudaSuccess) return e;
  e = cudaEventRecord(g_coop_ev[dev], s);
  if (e != cudaSuccess) return e;
  g_coop_any[dev] = true;
  return cudaSuccess;
}

inline int pad_tile(int m) { return (int)ceil_div(m, TB) * TB; }
inline int pad_jac(int m) { return (int)ceil_div(m < 2 ? 2 : m, 32) * 32; }

// Eigensolver workspace (jacobi_ws_elems doubles). The refinement uses Z, E, T, S, lam, stat and the integer
// arrays; the FP64 Jacobi reuses Z..S as its matrix and vector ping-pong buffers and lam as its diagonal/pair
// arrays; the FP32 Jacobi keeps its buffers in T, S and lam, which the refinement only fills after reading Z.
struct EigWs {
  int mp;
  double *Z, *E, *T, *S, *lam, *stat;
  int *counts, *perm, *order, *cid, *cls, *cln;
};

EigWs eig_ws(double* ws, int m) {
  EigWs w;
  w.mp = pad_jac(m);
  const size_t sq = (size_t)w.mp * w.mp;
  w.Z = ws;
  w.E = ws + sq;
  w.T = ws + 2 * sq;
  w.S = ws + 3 * sq;
  w.lam = ws + 4 * sq;
  w.stat = w.lam + 4 * (size_t)w.mp;
  w.counts = reinterpret_cast<int*>(w.stat + 16);
  w.perm = w.counts + kJacobiMaxSweeps + 8;
  w.order = w.perm + w.mp;
  w.cid = w.order + w.mp;
  w.cls = w.cid + w.mp;
  w.cln = w.cls + w.mp;
  return w;
}

template <typename T>
JacBuf<T> jac_buffers(const EigWs& w) {
  JacBuf<T> jb;
  const size_t sq = (size_t)w.mp * w.mp;
  if (sizeof(T) == sizeof(double)) {
    T* p = reinterpret_cast<T*>(w.Z);
    for (int i = 0; i < 2; ++i) { jb.A[i] = p; p += sq; }
    for (int i = 0; i < 2; ++i) { jb.V[i] = p; p += sq; }
  } else {
    T* p = reinterpret_cast<T*>(w.T);                // 4 mp^2 floats in the 2 mp^2 doubles of T and S
    for (int i = 0; i < 2; ++i) { jb.A[i] = p; p += sq; }
    for (int i = 0; i < 2; ++i) { jb.V[i] = p; p += sq; }
  }
  T* d = reinterpret_cast<T*>(w.lam);
  for (int i = 0; i < 2; ++i) { jb.Dg[i] = d; d += w.mp; }
  for (int i = 0; i < 2; ++i) { jb.Od[i] = d; d += w.mp; }
  return jb;
}

// Runs the Jacobi kernel of precision T on M (m x m, upper triangle read) into the buffers of w; info receives the
// sweep count and the buffer holding the result.
template <typename T>
cudaError_t run_jacobi(const double* M, int m, const EigWs& w, const JacBuf<T>& jb, double tol, int max_sweeps,
                       int* flag, unsigned* bar, int* info, cudaStream_t s) {
  const int mp = w.mp;
  double* nrm = w.stat + 8;
  cudaError_t e = cudaMemsetAsync(bar, 0, barrier_words() * sizeof(unsigned), s);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(w.counts, 0, sizeof(int) * kJacobiMaxSweeps, s);
  if (e != cudaSuccess) return e;
  const int64_t cnt = (int64_t)mp * mp;
  jacobi_init_kernel<T><<<grid_for(cnt), 256, 0, s>>>(M, m, mp, jb.A[0], jb.V[0], jb.Dg[0], jb.Od[0]);
  count_launch();
  frob_kernel<T><<<1, 1024, 0, s>>>(jb.A[0], cnt, nrm);
  count_launch();
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int P = mp / 2;
  const int64_t want = (int64_t)(P / JR) * (P / JR) + ceil_div(mp, JV) * (P / JC);
  const int lim = sizeof(T) == sizeof(double) ? coop_limits().jac : coop_limits().jac32;
  const int grid = (int)(want < lim ? (want < 1 ? 1 : want) : lim);
  const double* nrm_c = nrm;
  JacBuf<T> b = jb;
  void* args[] = {(void*)&b, (void*)&m, (void*)&mp, (void*)&nrm_c, (void*)&tol, (void*)&max_sweeps,
                  (void*)&w.counts, (void*)&flag, (void*)&bar, (void*)&info};
  count_launch();
  return coop_launch((const void*)jacobi_kernel<T>, (unsigned)grid, args, s);
}

// Every CTA but the last waits at one grid barrier that the last CTA never reaches, so the wait cannot complete:
// the bounded spin gives up after spin_limit polls, sets kFlagTimeout and every waiting CTA returns.
__global__ void __launch_bounds__(256) barrier_probe_kernel(unsigned* bar, int* flag, long long spin_limit) {
  unsigned gen = 0;
  if (blockIdx.x == gridDim.x - 1) return;
  grid_sync(bar, gridDim.x, flag, gen, spin_limit);
}

}  // namespace

cudaError_t barrier_timeout_probe(long long spin_limit, int* flag, unsigned* bar, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(bar, 0, barrier_words() * sizeof(unsigned), s);
  if (e != cudaSuccess) return e;
  int grid = coop_limits().chol;
  if (grid > 64) grid = 64;
  if (grid < 2) grid = 2;
  void* args[] = {(void*)&bar, (void*)&flag, (void*)&spin_limit};
  count_launch();
  return coop_launch((const void*)barrier_probe_kernel, (unsigned)grid, args, s);
}

size_t barrier_words() { return 2; }

size_t chol_ws_elems(int m) {
  const size_t mp = (size_t)pad_tile(m);
  return 2 * mp * mp + mp * TB + mp;
}

cudaError_t chol_inv(const double* G, int m, double shift, double* Rinv, double* ws, int* flag, unsigned* bar,
                     cudaStream_t s) {
  if (m <= 0) return cudaSuccess;
  const int mp = pad_tile(m);
  const int T = mp / TB;
  double* Lw = ws;
  double* Linv = Lw + (size_t)mp * mp;
  double* Lp = Linv + (size_t)mp * mp;
  double* diag0 = Lp + (size_t)mp * TB;
  cudaError_t e = cudaMemsetAsync(bar, 0, barrier_words() * sizeof(unsigned), s);
  if (e != cudaSuccess) return e;
  int tasks = 2 * (T - 1) * (T + 2);                  // update tasks of the first step (the most)
  if (tasks < 4 * T) tasks = 4 * T;
  const int lim = coop_limits().chol;
  const int grid = tasks < lim ? tasks : lim;
  void* args[] = {(void*)&G, (void*)&m, (void*)&mp, (void*)&shift, (void*)&Rinv, (void*)&Lw,
                  (void*)&Linv, (void*)&Lp, (void*)&diag0, (void*)&flag, (void*)&bar};
  count_launch();
  return coop_launch((const void*)chol_inv_kernel, (unsigned)grid, args, s);
}

size_t jacobi_ws_elems(int m) {
  const size_t mp = (size_t)pad_jac(m);
  return 4 * mp * mp + 4 * mp + 16 + ceil_div((int64_t)kJacobiMaxSweeps + 8 + 5 * (int64_t)mp, 2) + 8;
}

cudaError_t jacobi_eigh(const double* M, int m, double* lambda, double* C, double* ws, int* flag, unsigned* bar,
                        int* sweeps_out_dev, cudaStream_t s) {
  if (m <= 0) return cudaSuccess;
  const EigWs w = eig_ws(ws, m);
  const JacBuf<double> jb = jac_buffers<double>(w);
  int* info = sweeps_out_dev;
  cudaError_t e = run_jacobi<double>(M, m, w, jb, kJacobiTol, kJacobiMaxSweeps, flag, bar, info, s);
  if (e != cudaSuccess) return e;
  jacobi_sort_kernel<<<(unsigned)ceil_div(m, 256), 256, 0, s>>>(jb, m, w.mp, info, lambda, w.perm);
  count_launch();
  jacobi_gather_kernel<<<grid_for((int64_t)m * m), 256, 0, s>>>(jb, m, w.mp, info, w.perm, C);
  count_launch();
  return cudaGetLastError();
}

// Eigen-decomposition of the Rayleigh-Ritz matrix M, cheapest route first. The matrix of a Rayleigh-Ritz step late
// in a solve is nearly diagonal in the basis of the previous Ritz vectors, and then the parallel Jacobi method still
// pays its full rounds of grid barriers. (1) If no off-diagonal entry exceeds kJacobiTol ||M||_F (the Jacobi stop
// test), the eigenpairs are the sorted diagonal and unit vectors. (2) If none exceeds kRefineTau ||M||_F, the
// eigenvectors are refined from the identity (see the refinement kernels above). (3) Otherwise, or if (2) does not
// settle, a single-precision Jacobi, whose rotations run on the wide FP32 pipe, gives eigenvectors accurate to about
// 1e-6, and the refinement takes them to FP64 accuracy in two or three steps of m x m products. (4) If that does not
// settle within kRefineSteps steps, or a cluster exceeds kMaxCluster values, FP64 Jacobi on M. Accepted refinements
// take the Rayleigh quotients of the final vectors as eigenvalues.
// msym: m x m scratch (not aliasing M or C) for the symmetrised M.
cudaError_t dense_eigh_auto(const double* Min, int m, double* lambda, double* C, double* ws, double* msym,
                            const KxK& g, int* flag, unsigned* bar, int* sweeps_out_dev, int* path_out,
                            cudaStream_t s) {
  *path_out = 0;
  if (m <= 0) return cudaSuccess;
  const EigWs w = eig_ws(ws, m);
  double* G = C;                              // Z^T Z lives in the output until the final gather
  const double* M = msym;
  symmetrize_kernel<<<grid_for((int64_t)m * m), 256, 0, s>>>(Min, m, msym);
  count_launch();
  cudaError_t e;
  eig_stats_part_kernel<<<kStatBlocks, 256, 0, s>>>(M, m, w.E);
  eig_stats_kernel<<<1, 32, 0, s>>>(w.E, kStatBlocks, w.stat);
  count_launch(2);
  double h[8] = {};
  if ((e = cudaMemcpyAsync(h, w.stat, 2 * sizeof(double), cudaMemcpyDeviceToHost, s)) != cudaSuccess) return e;
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
  const double nM = h[0], off = h[1], thr = kJacobiTol * nM;
  if (!std::isfinite(nM)) return jacobi_eigh(Min, m, lambda, C, ws, flag, bar, sweeps_out_dev, s);
  if (off <= thr) {
    rank_sort_kernel<<<(unsigned)ceil_div(m, 256), 256, 0, s>>>(M, (int64_t)m + 1, m, lambda, w.perm);
    count_launch();
    gather_perm_kernel<<<grid_for((int64_t)m * m), 256, 0, s>>>(nullptr, m, w.perm, C);
    count_launch();
    *path_out = 1;
    return cudaGetLastError();
  }
  const int64_t cnt = (int64_t)m * m;
  const unsigned gcl = (unsigned)ceil_div(m, 2);
  // kRefineSteps refinement steps from Z = I (from_identity) or from the Z the FP32 Jacobi left in w.Z; returns
  // 1 when a step was accepted (outputs written), 0 when not, -1 on a CUDA error (in e)
  auto refine = [&](bool from_identity) -> int {
    for (int t = 0; t < kRefineSteps; ++t) {
      const double* St = M;
      const double* Gt = nullptr;
      if (t > 0 || !from_identity) {
        if ((e = kxk_gemm(g, true, w.Z, m, w.Z, m, m, m, m, G, m, s)) != cudaSuccess) return -1;      // Z^T Z
        if ((e = kxk_gemm(g, true, M, m, w.Z, m, m, m, m, w.T, m, s)) != cudaSuccess) return -1;      // M Z
        if ((e = kxk_gemm(g, true, w.Z, m, w.T, m, m, m, m, w.S, m, s)) != cudaSuccess) return -1;    // Z^T M Z
        St = w.S;
        Gt = G;
      }
      refine_diag_kernel<<<1, 1024, 0, s>>>(St, Gt, m, w.lam, w.stat);
      refine_coupling_kernel<<<grid_for(cnt), 256, 0, s>>>(St, Gt, m, w.lam, w.stat);
      rank_sort_kernel<<<(unsigned)ceil_div(m, 256), 256, 0, s>>>(w.lam, 1, m, w.lam + w.mp, w.order);
      refine_cluster_kernel<<<1, 1024, 0, s>>>(w.lam + w.mp, w.order, m, w.stat, w.cid, w.cls, w.cln);
      refine_coef_kernel<<<grid_for(cnt), 256, 0, s>>>(St, Gt, m, w.lam, w.cid, thr, w.stat, w.E);
      refine_cluster_eig_kernel<<<gcl, 256, 0, s>>>(St, Gt, m, w.lam, w.order, w.cls, w.cln, w.stat, w.E);
      count_launch(6);
      if (t == 0 && from_identity) {
        identity_plus_kernel<<<grid_for(cnt), 256, 0, s>>>(w.E, m, w.Z);
        count_launch();
      } else {
        if ((e = kxk_gemm(g, false, w.Z, m, w.E, m, m, m, m, w.T, m, s)) != cudaSuccess) return -1;   // Z E
        add_kernel<<<grid_for(cnt), 256, 0, s>>>(w.T, cnt, w.Z);
        count_launch();
      }
      if ((e = cudaMemcpyAsync(h + 2, w.stat + 2, 5 * sizeof(double), cudaMemcpyDeviceToHost, s)) != cudaSuccess)
        return -1;
      if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return -1;
      if (h[6] != 0.0) return 0;                              // a cluster too large for shared memory
      if (h[2] <= kRefineAccept && h[3] <= thr) {
        if ((e = kxk_gemm(g, true, M, m, w.Z, m, m, m, m, w.T, m, s)) != cudaSuccess) return -1;    // M Z
        rayleigh_quotient_kernel<<<(unsigned)ceil_div(m, 8), 256, 0, s>>>(w.Z, w.T, m, w.lam);
        count_launch();
        rank_sort_kernel<<<(unsigned)ceil_div(m, 256), 256, 0, s>>>(w.lam, 1, m, lambda, w.perm);
        count_launch();
        gather_perm_kernel<<<grid_for(cnt), 256, 0, s>>>(w.Z, m, w.perm, C);
        count_launch();
        if ((e = cudaGetLastError()) != cudaSuccess) return -1;
        return 1;
      }
      if (!(h[2] <= 1.0)) return 0;                           // diverging: corrections of order one
    }
    return 0;
  };
  if (off <= kRefineTau * nM) {
    const int r = refine(true);
    if (r < 0) return e;
    if (r > 0) {
      *path_out = 2;
      return cudaSuccess;
    }
  }
  {
    // single-precision Jacobi for the starting vectors
    const JacBuf<float> jb = jac_buffers<float>(w);
    e = run_jacobi<float>(M, m, w, jb, kJacobiTol32, kJacobiMaxSweeps32, flag, bar, sweeps_out_dev, s);
    if (e != cudaSuccess) return e;
    jacobi32_to_z_kernel<<<grid_for((int64_t)m * m), 256, 0, s>>>(jb, m, w.mp, sweeps_out_dev, w.Z);
    count_launch();
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const int r = refine(false);
    if (r < 0) return e;
    if (r > 0) {
      *path_out = 3;
      return cudaSuccess;
    }
  }
  return jacobi_eigh(Min, m, lambda, C, ws, flag, bar, sweeps_out_dev, s);
}

}  // namespace ppcg
