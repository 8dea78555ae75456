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
constexpr long long kSpinLimit = 1LL << 24;   // polls of ~100 ns: a wait longer than ~2 s is an error

__device__ bool grid_sync(unsigned* bar, unsigned nblocks, int* flag) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* vgen = bar + 1;
    const unsigned g = *vgen;
    __threadfence();
    const unsigned arrived = atomicAdd(bar, 1u);
    if (arrived == nblocks - 1) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      long long spins = 0;
      while (*vgen == g) {
        if (++spins > kSpinLimit || (*(volatile int*)flag & kFlagTimeout)) {
          atomicOr(flag, kFlagTimeout);
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
    ok = (*(volatile int*)flag & kFlagTimeout) ? 0 : 1;
  }
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
  if (!grid_sync(bar, nb, flag)) return;
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
    if (!grid_sync(bar, nb, flag)) return;
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
    if (!grid_sync(bar, nb, flag)) return;
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
    if (!grid_sync(bar, nb, flag)) return;
  }
  // L^{-1}: diagonal tiles are Dinv; tile (i, j), j < i: -Dinv_i * sum_{l=j}^{i-1} L_il Linv_lj
  for (int i = blockIdx.x; i < T; i += nb) {
    load_tile(Dinv + (int64_t)i * TB * TB, TB, 0, 0, s1);
    __syncthreads();
    store_tile(Linv, mp, i, i, s1);
    __syncthreads();
  }
  if (!grid_sync(bar, nb, flag)) return;
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
    if (!grid_sync(bar, nb, flag)) return;
  }
  // R^{-1} = (L^{-1})^T, upper triangular, leading dimension m
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + t; e < (int64_t)m * m; e += (int64_t)nb * blockDim.x) {
    const int r = (int)(e % m), c = (int)(e / m);
    Rinv[e] = (r <= c) ? __ldcg(Linv + c + (int64_t)r * mp) : 0.0;
  }
}

// ------------------------------------------------------------------------------------------- Jacobi
__device__ __forceinline__ void rr_pair(int mp, int r, int i, int& p, int& q) {
  const int M1 = mp - 1;
  int a, b;
  if (i == 0) {
    a = 0;
    b = 1 + r % M1;
  } else {
    a = 1 + (r + i) % M1;
    b = 1 + (r - i + M1) % M1;
  }
  p = a < b ? a : b;
  q = a < b ? b : a;
}

__device__ __forceinline__ bool rot_params(const double* A, int mp, int m, int p, int q, double thr, double& c,
                                           double& s, double& t) {
  c = 1.0; s = 0.0; t = 0.0;
  if (q >= m) return false;
  const double apq = __ldcg(A + p + (int64_t)q * mp);
  if (!(fabs(apq) > thr)) return false;
  const double app = __ldcg(A + p + (int64_t)p * mp);
  const double aqq = __ldcg(A + q + (int64_t)q * mp);
  const double theta = (aqq - app) / (2.0 * apq);
  const double at = fabs(theta);
  double tt = at > 1e150 ? 0.5 / at : 1.0 / (at + sqrt(at * at + 1.0));
  if (theta < 0.0) tt = -tt;
  t = tt;
  c = 1.0 / sqrt(tt * tt + 1.0);
  s = tt * c;
  return true;
}

__global__ void jacobi_init_kernel(const double* __restrict__ M, int m, int mp, double* A0, double* V) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)mp * mp;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % mp), j = (int)(e / mp);
    A0[e] = (i < m && j < m) ? M[(i < j ? i : j) + (int64_t)(i < j ? j : i) * m] : 0.0;
    V[e] = (i == j) ? 1.0 : 0.0;
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

__global__ void __launch_bounds__(256)
jacobi_kernel(double* A0, double* A1, double* V, int m, int mp, const double* normA, int* counts, int* flag,
              unsigned* bar, int* info) {
  const double thr = kJacobiTol * normA[0];
  const int P = mp / 2;
  const int nA = P * (P + 1) / 2;
  const int64_t total = (int64_t)nA + (int64_t)mp * P;
  const unsigned nb = gridDim.x;
  const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t gstride = (int64_t)nb * blockDim.x;
  int cur = 0;
  int sweep = 0;
  for (; sweep < kJacobiMaxSweeps; ++sweep) {
    for (int r = 0; r < mp - 1; ++r) {
      const double* src = cur ? A1 : A0;
      double* dst = cur ? A0 : A1;
      for (int64_t task = gtid; task < total; task += gstride) {
        if (task < nA) {
          int pb = (int)((sqrt(8.0 * (double)task + 1.0) - 1.0) * 0.5);
          while (pb * (pb + 1) / 2 > task) --pb;
          while ((pb + 1) * (pb + 2) / 2 <= task) ++pb;
          const int pa = (int)task - pb * (pb + 1) / 2;
          int p, q, u, v;
          rr_pair(mp, r, pa, p, q);
          rr_pair(mp, r, pb, u, v);
          double ca, sa, ta;
          const bool da = rot_params(src, mp, m, p, q, thr, ca, sa, ta);
          if (pa == pb) {
            const double app = __ldcg(src + p + (int64_t)p * mp);
            const double aqq = __ldcg(src + q + (int64_t)q * mp);
            const double apq = __ldcg(src + p + (int64_t)q * mp);
            if (da) {
              atomicAdd(counts + sweep, 1);
              dst[p + (int64_t)p * mp] = app - ta * apq;
              dst[q + (int64_t)q * mp] = aqq + ta * apq;
              dst[p + (int64_t)q * mp] = 0.0;
              dst[q + (int64_t)p * mp] = 0.0;
            } else {
              dst[p + (int64_t)p * mp] = app;
              dst[q + (int64_t)q * mp] = aqq;
              dst[p + (int64_t)q * mp] = apq;
              dst[q + (int64_t)p * mp] = apq;
            }
          } else {
            double cb, sb, tb;
            rot_params(src, mp, m, u, v, thr, cb, sb, tb);
            const double xpu = __ldcg(src + p + (int64_t)u * mp), xpv = __ldcg(src + p + (int64_t)v * mp);
            const double xqu = __ldcg(src + q + (int64_t)u * mp), xqv = __ldcg(src + q + (int64_t)v * mp);
            const double ypu = ca * xpu - sa * xqu, ypv = ca * xpv - sa * xqv;
            const double yqu = sa * xpu + ca * xqu, yqv = sa * xpv + ca * xqv;
            const double zpu = cb * ypu - sb * ypv, zpv = sb * ypu + cb * ypv;
            const double zqu = cb * yqu - sb * yqv, zqv = sb * yqu + cb * yqv;
            dst[p + (int64_t)u * mp] = zpu; dst[p + (int64_t)v * mp] = zpv;
            dst[q + (int64_t)u * mp] = zqu; dst[q + (int64_t)v * mp] = zqv;
            dst[u + (int64_t)p * mp] = zpu; dst[v + (int64_t)p * mp] = zpv;
            dst[u + (int64_t)q * mp] = zqu; dst[v + (int64_t)q * mp] = zqv;
          }
        } else {
          const int64_t vt = task - nA;
          const int pb = (int)(vt / mp);
          const int row = (int)(vt % mp);
          int u, v;
          rr_pair(mp, r, pb, u, v);
          double cb, sb, tb;
          if (rot_params(src, mp, m, u, v, thr, cb, sb, tb)) {
            const double zu = __ldcg(V + row + (int64_t)u * mp), zv = __ldcg(V + row + (int64_t)v * mp);
            V[row + (int64_t)u * mp] = cb * zu - sb * zv;
            V[row + (int64_t)v * mp] = sb * zu + cb * zv;
          }
        }
      }
      if (!grid_sync(bar, nb, flag)) return;
      cur ^= 1;
    }
    if (*(volatile int*)(counts + sweep) == 0) break;
  }
  if (gtid == 0) {
    info[0] = sweep;
    info[1] = cur;
    if (sweep >= kJacobiMaxSweeps) atomicOr(flag, kFlagJacobiNoConv);
  }
}

// lambda ascending; C[:, rank(i)] = V[0:m, i]
__global__ void jacobi_sort_kernel(const double* A0, const double* A1, const double* V, int m, int mp,
                                   const int* info, double* lambda, int* perm) {
  const double* A = info[1] ? A1 : A0;
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

__global__ void jacobi_gather_kernel(const double* V, int m, int mp, const int* perm, double* C) {
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
  const size_t mp = (size_t)pad_even(m);
  return 3 * mp * mp + 8 + (size_t)kJacobiMaxSweeps + 2 * mp + 8;
}

cudaError_t jacobi_eigh(const double* M, int m, double* lambda, double* C, double* ws, int* flag, unsigned* bar,
                        int* sweeps_out_dev, cudaStream_t s) {
  if (m <= 0) return cudaSuccess;
  const int mp = pad_even(m < 2 ? 2 : m);
  double* A0 = ws;
  double* A1 = A0 + (size_t)mp * mp;
  double* V = A1 + (size_t)mp * mp;
  double* nrm = V + (size_t)mp * mp;
  int* counts = reinterpret_cast<int*>(nrm + 8);
  int* perm = counts + kJacobiMaxSweeps + 8;
  int* info = sweeps_out_dev;
  cudaError_t e = cudaMemsetAsync(bar, 0, barrier_words() * sizeof(unsigned), s);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(counts, 0, sizeof(int) * kJacobiMaxSweeps, s);
  if (e != cudaSuccess) return e;
  const int64_t cnt = (int64_t)mp * mp;
  jacobi_init_kernel<<<(unsigned)(ceil_div(cnt, 256) < 4096 ? ceil_div(cnt, 256) : 4096), 256, 0, s>>>(M, m, mp, A0,
                                                                                                      V);
  count_launch();
  frob_kernel<<<1, 1024, 0, s>>>(A0, cnt, nrm);
  count_launch();
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int P = mp / 2;
  const int64_t total = (int64_t)P * (P + 1) / 2 + (int64_t)mp * P;
  int64_t want = ceil_div(total, 256);
  const int lim = coop_limits().jac;
  const int grid = (int)(want < lim ? want : lim);
  const double* nrm_c = nrm;
  void* args[] = {(void*)&A0, (void*)&A1, (void*)&V, (void*)&m, (void*)&mp, (void*)&nrm_c,
                  (void*)&counts, (void*)&flag, (void*)&bar, (void*)&info};
  count_launch();
  e = cudaLaunchCooperativeKernel((const void*)jacobi_kernel, dim3(grid), dim3(256), args, 0, s);
  if (e != cudaSuccess) return e;
  jacobi_sort_kernel<<<(unsigned)ceil_div(m, 256), 256, 0, s>>>(A0, A1, V, m, mp, info, lambda, perm);
  count_launch();
  jacobi_gather_kernel<<<(unsigned)(ceil_div((int64_t)m * m, 256) < 4096 ? ceil_div((int64_t)m * m, 256) : 4096), 256,
                         0, s>>>(V, m, mp, perm, C);
  count_launch();
  return cudaGetLastError();
}

}  // namespace ppcg
