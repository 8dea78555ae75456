// Dense k x k kernels of Algorithm 3 (the ScaLAPACK part of Section 6):
//   chol_inv     R^{-1} for the Cholesky factor of the Gram X^T X = R^T R (CholQR, Section 5.4, steps 18-19):
//                blocked right-looking Cholesky on 32 x 32 tiles, then the inverse of L = R^T by tile
//                diagonals; one cooperative persistent kernel, tile tasks spread over the CTAs.
//   jacobi_eigh  eigen-decomposition of the projected matrix of the Rayleigh-Ritz step (steps 23-24,
//                Section 5.5): parallel cyclic Jacobi with round-robin pairing. In every round each 2 x 2 block
//                of A is rotated from both sides independently (ping-pong buffers), each CTA recomputing the
//                rotations it needs from the previous round's matrix, so one grid barrier separates rounds.
// On GB300 FP64 is scarce (2 DFMA lanes per clock per SM); these kernels spread the O(k^3) work over all SMs
// instead of one process grid. Every device-side wait is bounded: a barrier that gives up sets kFlagTimeout
// and every CTA returns.
#include "ppcg_internal.h"

#include <cmath>
#include <math_constants.h>

namespace ppcg {

namespace {

constexpr int TB = 32;
constexpr long long kSpinLimit = 1LL << 25;   // polls of ~50-100 ns: a wait longer than ~2-3 s is an error

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
__device__ __forceinline__ unsigned atom_add_acq_rel_gpu(unsigned* p, unsigned v) {
  unsigned old;
  asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
  return old;
}
__device__ __forceinline__ void st_release_gpu(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" :: "l"(p), "r"(v) : "memory");
}

// Software grid barrier for cooperative launches (all CTAs co-resident). bar[0] counts arrivals, bar[1] is the
// generation, which every CTA also tracks locally in `gen` (one increment per barrier), so arriving needs a single
// atomic round trip. The wait is bounded: after kSpinLimit polls the CTA sets kFlagTimeout and every CTA returns
// false.
__device__ bool grid_sync(unsigned* bar, unsigned nblocks, int* flag, unsigned& gen) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned g = gen;
    __threadfence();                                   // publish this CTA's writes at GPU scope
    const unsigned arrived = atom_add_acq_rel_gpu(bar, 1u);
    int good = 1;
    if (arrived == nblocks - 1) {
      bar[0] = 0u;                                     // ordered before the release below
      st_release_gpu(bar + 1, g + 1u);
    } else {
      long long spins = 0;
      while (ld_acquire_gpu(bar + 1) == g) {
        if (++spins > kSpinLimit || (ld_relaxed_gpu(flag) & kFlagTimeout)) {
          atomicOr(flag, kFlagTimeout);
          good = 0;
          break;
        }
      }
    }
    __threadfence();
    if (ld_relaxed_gpu(flag) & kFlagTimeout) good = 0;
    ok = good;
  }
  gen += 1u;
  __syncthreads();
  return ok != 0;
}

// ------------------------------------------------------------------------------------------- Cholesky
__device__ void load_tile(const double* M, int ld, int ti, int tj, double (*s)[TB + 1]) {
  for (int e = threadIdx.x; e < TB * TB; e += blockDim.x) {
    const int r = e % TB, c = e / TB;
    s[r][c] = __ldcg(M + (int64_t)(ti * TB + r) + (int64_t)(tj * TB + c) * ld);
  }
}

__device__ void store_tile(double* M, int ld, int ti, int tj, double (*s)[TB + 1]) {
  for (int e = threadIdx.x; e < TB * TB; e += blockDim.x) {
    const int r = e % TB, c = e / TB;
    M[(int64_t)(ti * TB + r) + (int64_t)(tj * TB + c) * ld] = s[r][c];
  }
}

__global__ void __launch_bounds__(256)
chol_inv_kernel(const double* __restrict__ G, int m, int mp, double shift, double* __restrict__ Rinv,
                double* Lw, double* Linv, double* Dinv, double* diag0, int* flag, unsigned* bar) {
  const int T = mp / TB;
  const unsigned nb = gridDim.x;
  const int t = threadIdx.x;
  unsigned gen = 0;
  __shared__ double s1[TB][TB + 1], s2[TB][TB + 1], s3[TB][TB + 1];
  // fill the padded matrix [G + shift I, 0; 0, I]; only the lower triangle is used
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
    if (blockIdx.x == 0) {
      load_tile(Lw, mp, kk, kk, s1);
      __syncthreads();
      for (int c = 0; c < TB; ++c) {
        if (t == 0) {
          const double a = s1[c][c];
          const double g0 = __ldcg(diag0 + kk * TB + c);
          double piv = a > 0.0 ? sqrt(a) : 0.0;
          if (!(piv >= kCholPivotTol * sqrt(g0))) {
            atomicOr(flag, kFlagCholBreakdown);
            if (!(piv > 0.0)) piv = 1.0;
          }
          s1[c][c] = piv;
        }
        __syncthreads();
        if (t > c && t < TB) s1[t][c] /= s1[c][c];
        __syncthreads();
        for (int e = t; e < TB * TB; e += blockDim.x) {
          const int r = e % TB, j = e / TB;
          if (j > c && r >= j) s1[r][j] -= s1[r][c] * s1[j][c];
        }
        __syncthreads();
      }
      // inverse of the lower-triangular tile (column per thread)
      if (t < TB) {
        const int c = t;
        for (int i = 0; i < TB; ++i) s2[i][c] = 0.0;
        s2[c][c] = 1.0 / s1[c][c];
        for (int i = c + 1; i < TB; ++i) {
          double v = 0.0;
          for (int l = c; l < i; ++l) v += s1[i][l] * s2[l][c];
          s2[i][c] = -v / s1[i][i];
        }
      }
      __syncthreads();
      store_tile(Lw, mp, kk, kk, s1);
      store_tile(Dinv + (int64_t)kk * TB * TB, TB, 0, 0, s2);
    }
    if (!grid_sync(bar, nb, flag, gen)) return;
    // panel: L_ik = A_ik Dinv_kk^T
    for (int i = kk + 1 + blockIdx.x; i < T; i += nb) {
      load_tile(Lw, mp, i, kk, s1);
      load_tile(Dinv + (int64_t)kk * TB * TB, TB, 0, 0, s2);
      __syncthreads();
      for (int e = t; e < TB * TB; e += blockDim.x) {
        const int r = e % TB, c = e / TB;
        double v = 0.0;
        for (int l = 0; l <= c; ++l) v += s1[r][l] * s2[c][l];
        s3[r][c] = v;
      }
      __syncthreads();
      store_tile(Lw, mp, i, kk, s3);
      __syncthreads();
    }
    if (!grid_sync(bar, nb, flag, gen)) return;
    // trailing update: A_ij -= L_ik L_jk^T, kk < j <= i
    const int R = T - kk - 1;
    const int ntasks = R * (R + 1) / 2;
    for (int task = blockIdx.x; task < ntasks; task += nb) {
      int a = 0;
      while ((a + 1) * (a + 2) / 2 <= task) ++a;
      const int b = task - a * (a + 1) / 2;
      const int i = kk + 1 + a, j = kk + 1 + b;
      load_tile(Lw, mp, i, kk, s1);
      load_tile(Lw, mp, j, kk, s2);
      load_tile(Lw, mp, i, j, s3);
      __syncthreads();
      for (int e = t; e < TB * TB; e += blockDim.x) {
        const int r = e % TB, c = e / TB;
        double v = s3[r][c];
        for (int l = 0; l < TB; ++l) v -= s1[r][l] * s2[c][l];
        s3[r][c] = v;
      }
      __syncthreads();
      store_tile(Lw, mp, i, j, s3);
      __syncthreads();
    }
    if (!grid_sync(bar, nb, flag, gen)) return;
  }
  // L^{-1}: diagonal tiles are Dinv; tile (i, j), j < i: -Dinv_i * sum_{l=j}^{i-1} L_il Linv_lj
  for (int i = blockIdx.x; i < T; i += nb) {
    load_tile(Dinv + (int64_t)i * TB * TB, TB, 0, 0, s1);
    __syncthreads();
    store_tile(Linv, mp, i, i, s1);
    __syncthreads();
  }
  if (!grid_sync(bar, nb, flag, gen)) return;
  for (int d = 1; d < T; ++d) {
    for (int i = d + blockIdx.x; i < T; i += nb) {
      const int j = i - d;
      double acc[4] = {0.0, 0.0, 0.0, 0.0};
      for (int l = j; l < i; ++l) {
        load_tile(Lw, mp, i, l, s1);
        load_tile(Linv, mp, l, j, s2);
        __syncthreads();
        for (int u = 0; u < 4; ++u) {
          const int e = t + u * blockDim.x;
          const int r = e % TB, c = e / TB;
          double v = 0.0;
          for (int x = 0; x < TB; ++x) v += s1[r][x] * s2[x][c];
          acc[u] += v;
        }
        __syncthreads();
      }
      for (int u = 0; u < 4; ++u) {
        const int e = t + u * blockDim.x;
        s2[e % TB][e / TB] = acc[u];
      }
      load_tile(Dinv + (int64_t)i * TB * TB, TB, 0, 0, s1);
      __syncthreads();
      for (int e = t; e < TB * TB; e += blockDim.x) {
        const int r = e % TB, c = e / TB;
        double v = 0.0;
        for (int x = 0; x <= r; ++x) v += s1[r][x] * s2[x][c];
        s3[r][c] = -v;
      }
      __syncthreads();
      store_tile(Linv, mp, i, j, s3);
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
// so that rotation parameters are read from compact arrays.
__device__ __forceinline__ int slot_shift(int t, int mp) { return t == 0 ? 0 : (t == mp - 1 ? 1 : t + 1); }

// Rotation (c, s) that annihilates apq approximately: t = tan(phi) from a single-precision solve of
// t^2 + 2 theta t - 1 = 0 (theta = (aqq - app) / (2 apq)), then c = 1/sqrt(1 + t^2) refined by two FP64 Newton
// steps and s = t c, so that c^2 + s^2 = 1 to FP64 rounding and the rotation is an exact orthogonal similarity.
// (FP64 division and square root are long instruction sequences on GB300's 2-lane-per-clock FP64 pipe; the
// residual a'_pq ~ 1e-7 |apq| left by the single-precision angle is removed by later sweeps.)
__device__ __forceinline__ bool rot_from(double app, double aqq, double apq, double thr, double& c, double& s) {
  c = 1.0; s = 0.0;
  if (!(fabs(apq) > thr)) return false;
  const float th = (float)((aqq - app) / (2.0 * apq));   // FP64 quotient: no single-precision underflow
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
  return true;
}

__global__ void jacobi_init_kernel(const double* __restrict__ M, int m, int mp, double* A0, double* V0, double* Dg,
                                   double* Od) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)mp * mp;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % mp), j = (int)(e / mp);
    const double v = (i < m && j < m) ? M[(i < j ? i : j) + (int64_t)(i < j ? j : i) * m] : 0.0;
    A0[e] = v;
    V0[e] = (i == j) ? 1.0 : 0.0;
    if (i == j) Dg[i] = v;
    if (i + j == mp - 1 && i < j) Od[i] = v;
  }
}

__global__ void frob_kernel(const double* __restrict__ A, int64_t cnt, double* out) {
  double s = 0.0;
  for (int64_t e = threadIdx.x; e < cnt; e += blockDim.x) s += A[e] * A[e];
  __shared__ double red[1024];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int off = blockDim.x / 2; off > 0; off >>= 1) {
    if ((int)threadIdx.x < off) red[threadIdx.x] += red[threadIdx.x + off];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = sqrt(red[0]);
}

struct JacBuf {
  double *A[2], *V[2], *Dg[2], *Od[2];
};

__global__ void __launch_bounds__(256)
jacobi_kernel(JacBuf b, int m, int mp, const double* normA, int* counts, int* flag, unsigned* bar, int* info) {
  const double thr = kJacobiTol * normA[0];
  const int P = mp / 2;
  const int64_t nA = (int64_t)P * P;
  const int64_t total = nA + (int64_t)mp * P;
  const unsigned nb = gridDim.x;
  const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t gstride = (int64_t)nb * blockDim.x;
  int cur = 0;
  int sweep = 0;
  unsigned gen = 0;
  for (; sweep < kJacobiMaxSweeps; ++sweep) {
    for (int r = 0; r < mp - 1; ++r) {
      const double* __restrict__ A = b.A[cur];
      double* __restrict__ An = b.A[cur ^ 1];
      const double* __restrict__ V = b.V[cur];
      double* __restrict__ Vn = b.V[cur ^ 1];
      const double* __restrict__ Dg = b.Dg[cur];
      const double* __restrict__ Od = b.Od[cur];
      double* __restrict__ Dn = b.Dg[cur ^ 1];
      double* __restrict__ On = b.Od[cur ^ 1];
      for (int64_t task = gtid; task < total; task += gstride) {
        if (task < nA) {
          const int ri = (int)(task % P), ci = (int)(task / P);   // row pair ri, column pair ci
          const int rb = mp - 1 - ri, cb = mp - 1 - ci;
          double cr, sr, cc, sc;
          const bool drot = rot_from(__ldcg(Dg + ri), __ldcg(Dg + rb), __ldcg(Od + ri), thr, cr, sr);
          rot_from(__ldcg(Dg + ci), __ldcg(Dg + cb), __ldcg(Od + ci), thr, cc, sc);
          double x00, x01, x10, x11;        // rows (ri, rb) x cols (ci, cb)
          if (ri == ci) {
            x00 = __ldcg(Dg + ri); x11 = __ldcg(Dg + rb); x01 = __ldcg(Od + ri); x10 = x01;
            if (drot) atomicAdd(counts + sweep, 1);
          } else {
            x00 = __ldcg(A + ri + (int64_t)ci * mp); x10 = __ldcg(A + rb + (int64_t)ci * mp);
            x01 = __ldcg(A + ri + (int64_t)cb * mp); x11 = __ldcg(A + rb + (int64_t)cb * mp);
          }
          const double y00 = cr * x00 - sr * x10, y01 = cr * x01 - sr * x11;
          const double y10 = sr * x00 + cr * x10, y11 = sr * x01 + cr * x11;
          double z00 = cc * y00 - sc * y01, z01 = sc * y00 + cc * y01;
          double z10 = cc * y10 - sc * y11, z11 = sc * y10 + cc * y11;
          if (ri == ci) z10 = z01;                   // keep the diagonal block exactly symmetric
          const int R0 = slot_shift(ri, mp), R1 = slot_shift(rb, mp);
          const int C0 = slot_shift(ci, mp), C1 = slot_shift(cb, mp);
          An[R0 + (int64_t)C0 * mp] = z00;
          An[R1 + (int64_t)C0 * mp] = z10;
          An[R0 + (int64_t)C1 * mp] = z01;
          An[R1 + (int64_t)C1 * mp] = z11;
          // next round's diagonal and pair entries
          if (R0 == C0) Dn[R0] = z00;
          if (R1 == C1) Dn[R1] = z11;
          if (R0 == C1) Dn[R0] = z01;
          if (R1 == C0) Dn[R1] = z10;
          if (R0 + C0 == mp - 1 && R0 < C0) On[R0] = z00;
          if (R1 + C0 == mp - 1 && R1 < C0) On[R1] = z10;
          if (R0 + C1 == mp - 1 && R0 < C1) On[R0] = z01;
          if (R1 + C1 == mp - 1 && R1 < C1) On[R1] = z11;
        } else {
          const int64_t vt = task - nA;
          const int row = (int)(vt % mp);
          const int ci = (int)(vt / mp);
          const int cb = mp - 1 - ci;
          double cc, sc;
          rot_from(__ldcg(Dg + ci), __ldcg(Dg + cb), __ldcg(Od + ci), thr, cc, sc);
          const double vu = __ldcg(V + row + (int64_t)ci * mp), vv = __ldcg(V + row + (int64_t)cb * mp);
          Vn[row + (int64_t)slot_shift(ci, mp) * mp] = cc * vu - sc * vv;
          Vn[row + (int64_t)slot_shift(cb, mp) * mp] = sc * vu + cc * vv;
        }
      }
      if (!grid_sync(bar, nb, flag, gen)) return;
      cur ^= 1;
    }
    if (ld_relaxed_gpu(counts + sweep) == 0) break;
  }
  if (gtid == 0) {
    info[0] = sweep;
    info[1] = cur;
    if (sweep >= kJacobiMaxSweeps) atomicOr(flag, kFlagJacobiNoConv);
  }
}

// lambda ascending; C[:, rank(i)] = V[0:m, i]. The layout is the identity at a sweep boundary.
__global__ void jacobi_sort_kernel(JacBuf b, int m, int mp, const int* info, double* lambda, int* perm) {
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

__global__ void jacobi_gather_kernel(JacBuf b, int m, int mp, const int* info, const int* perm, double* C) {
  const double* V = b.V[info[1]];
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)m * m;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(e % m), c = (int)(e / m);
    C[e] = V[r + (int64_t)perm[c] * mp];
  }
}

struct CoopLimit {
  int chol = 0, jac = 0;
};

CoopLimit& coop_limits() {
  static CoopLimit lim;
  if (lim.chol == 0) {
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int per = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, chol_inv_kernel, 256, 0);
    lim.chol = (per > 0 ? per : 1) * sms;
    per = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, jacobi_kernel, 256, 0);
    lim.jac = (per > 0 ? per : 1) * sms;
  }
  return lim;
}

inline int pad_tile(int m) { return (int)ceil_div(m, TB) * TB; }
inline int pad_even(int m) { return (m + 1) & ~1; }

}  // namespace

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
  double* Dinv = Linv + (size_t)mp * mp;
  double* diag0 = Dinv + (size_t)mp * TB;
  cudaError_t e = cudaMemsetAsync(bar, 0, barrier_words() * sizeof(unsigned), s);
  if (e != cudaSuccess) return e;
  int tasks = T * (T - 1) / 2;
  if (tasks < T) tasks = T;
  if (tasks < 1) tasks = 1;
  const int lim = coop_limits().chol;
  const int grid = tasks < lim ? tasks : lim;
  void* args[] = {(void*)&G, (void*)&m, (void*)&mp, (void*)&shift, (void*)&Rinv, (void*)&Lw,
                  (void*)&Linv, (void*)&Dinv, (void*)&diag0, (void*)&flag, (void*)&bar};
  count_launch();
  return cudaLaunchCooperativeKernel((const void*)chol_inv_kernel, dim3(grid), dim3(256), args, 0, s);
}

size_t jacobi_ws_elems(int m) {
  const size_t mp = (size_t)pad_even(m < 2 ? 2 : m);
  return 4 * mp * mp + 4 * mp + 8 + (size_t)kJacobiMaxSweeps + mp + 8;
}

cudaError_t jacobi_eigh(const double* M, int m, double* lambda, double* C, double* ws, int* flag, unsigned* bar,
                        int* sweeps_out_dev, cudaStream_t s) {
  if (m <= 0) return cudaSuccess;
  const int mp = pad_even(m < 2 ? 2 : m);
  JacBuf jb;
  double* p = ws;
  for (int i = 0; i < 2; ++i) { jb.A[i] = p; p += (size_t)mp * mp; }
  for (int i = 0; i < 2; ++i) { jb.V[i] = p; p += (size_t)mp * mp; }
  for (int i = 0; i < 2; ++i) { jb.Dg[i] = p; p += mp; }
  for (int i = 0; i < 2; ++i) { jb.Od[i] = p; p += mp; }
  double* nrm = p;
  int* counts = reinterpret_cast<int*>(nrm + 8);
  int* perm = counts + kJacobiMaxSweeps + 8;
  int* info = sweeps_out_dev;
  cudaError_t e = cudaMemsetAsync(bar, 0, barrier_words() * sizeof(unsigned), s);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(counts, 0, sizeof(int) * kJacobiMaxSweeps, s);
  if (e != cudaSuccess) return e;
  const int64_t cnt = (int64_t)mp * mp;
  jacobi_init_kernel<<<(unsigned)(ceil_div(cnt, 256) < 4096 ? ceil_div(cnt, 256) : 4096), 256, 0, s>>>(
      M, m, mp, jb.A[0], jb.V[0], jb.Dg[0], jb.Od[0]);
  count_launch();
  frob_kernel<<<1, 1024, 0, s>>>(jb.A[0], cnt, nrm);
  count_launch();
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int P = mp / 2;
  const int64_t total = (int64_t)P * P + (int64_t)mp * P;
  const int64_t want = ceil_div(total, 256);
  const int lim = coop_limits().jac;
  const int grid = (int)(want < lim ? (want < 1 ? 1 : want) : lim);
  const double* nrm_c = nrm;
  void* args[] = {(void*)&jb, (void*)&m, (void*)&mp, (void*)&nrm_c, (void*)&counts, (void*)&flag, (void*)&bar,
                  (void*)&info};
  count_launch();
  e = cudaLaunchCooperativeKernel((const void*)jacobi_kernel, dim3(grid), dim3(256), args, 0, s);
  if (e != cudaSuccess) return e;
  jacobi_sort_kernel<<<(unsigned)ceil_div(m, 256), 256, 0, s>>>(jb, m, mp, info, lambda, perm);
  count_launch();
  jacobi_gather_kernel<<<(unsigned)(ceil_div((int64_t)m * m, 256) < 4096 ? ceil_div((int64_t)m * m, 256) : 4096), 256,
                         0, s>>>(jb, m, mp, info, perm, C);
  count_launch();
  return cudaGetLastError();
}

}  // namespace ppcg
