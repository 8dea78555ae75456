// Sub-block Rayleigh-Ritz of PPCG (Section 3 eq. upd_col, Section 5.1 eq. upd_block; Algorithm 3 steps 11-15).
//
// For each of the s = ceil(k_act / q) sub-blocks S_j = [X_j, W_j, P_j] (q_j = q columns each, the last one the
// remainder) the method needs the q_j smallest eigenpairs of the 3q_j x 3q_j pencil
// (S_j^T A S_j) c = theta (S_j^T S_j) c, c^T S_j^T S_j c = 1 (eq. projev); 2q_j x 2q_j when P = [] (first
// iteration). The paper solves these s problems one after the other; here:
//   block_gram   one pass over the 6 q-column panels X_j, W_j, P_j, AX_j, AW_j, AP_j computes both Grams of
//                every sub-block (upper triangles), split over row chunks into partials;
//   block_solve  one warp per sub-block sums the partials and solves its pencil entirely in shared memory:
//                unit column scaling, Cholesky of S^T S, the standard form L^{-1} G_A L^{-T}, cyclic Jacobi,
//                back-substitution; Theorem 1 (C_X non-singular) and the Cholesky pivots decide the back-track
//                of Section 3 (redo without P; Theorem 2 guarantees it succeeds for HPD T and r_j != 0);
//   block_update P_j <- W_j C_W + P_j C_P ; X_j <- X_j C_X + P_j in one streaming pass.
#include "ppcg_internal.h"

#include <math_constants.h>

namespace ppcg {

namespace {

constexpr int kMaxM = 3 * kMaxSbsize;  // 48
constexpr int kGramRows = 32;          // rows per shared-memory sub-tile in block_gram

__host__ __device__ constexpr int entries(int m) { return m * (m + 1); }   // both upper triangles

__device__ __forceinline__ const double* panel_col(const BlockArgs& a, bool h, int col, int c0, int qj) {
  const int which = col / qj, off = col % qj;
  const double* base;
  if (!h) base = which == 0 ? a.X : (which == 1 ? a.W : a.P);
  else base = which == 0 ? a.HX : (which == 1 ? a.HW : a.HP);
  return base + (int64_t)(c0 + off) * a.ld;
}

// grid (s, nchunk). part[(chunk * s + j) * Emax + e]: e < m(m+1)/2 -> G_A upper (a <= b, packed by column),
// else G_B upper.
__global__ void __launch_bounds__(256)
block_gram_kernel(BlockArgs a, int s, int64_t rows_per_chunk, double* __restrict__ part, int Emax) {
  const int j = blockIdx.x, chunk = blockIdx.y;
  const int c0 = j * a.q;
  const int qj = min(a.q, a.k_act - c0);
  const int m = (a.has_p ? 3 : 2) * qj;
  const int Eh = m * (m + 1) / 2, E = 2 * Eh;
  const int64_t r_begin = (int64_t)chunk * rows_per_chunk;
  const int64_t r_end = min(a.n, r_begin + rows_per_chunk);
  __shared__ double S[kGramRows][kMaxM + 1];
  __shared__ double HS[kGramRows][kMaxM + 1];
  __shared__ const double* colS[kMaxM];
  __shared__ const double* colH[kMaxM];
  __shared__ double red[256];
  const int t = threadIdx.x;
  if (t < m) {
    colS[t] = panel_col(a, false, t, c0, qj);
    colH[t] = panel_col(a, true, t, c0, qj);
  }
  // thread -> (entry e, row group g)
  const int ngroups = E <= 256 ? 256 / E : 1;
  const int g = E <= 256 ? t / E : 0;
  constexpr int kMaxPer = (entries(kMaxM) + 255) / 256;   // 10
  double acc[kMaxPer];
  int ea[kMaxPer], eb[kMaxPer];
  bool eg[kMaxPer];
  int ne = 0;
  if (g < ngroups) {
    for (int e = (E <= 256 ? t % E : t); e < E && ne < kMaxPer; e += (E <= 256 ? E : 256)) {
      const bool isB = e >= Eh;
      int r = isB ? e - Eh : e;
      int b = 0;
      while ((b + 1) * (b + 2) / 2 <= r) ++b;
      ea[ne] = r - b * (b + 1) / 2;
      eb[ne] = b;
      eg[ne] = isB;
      acc[ne] = 0.0;
      ++ne;
      if (E <= 256) break;
    }
  }
  __syncthreads();
  for (int64_t r0 = r_begin; r0 < r_end; r0 += kGramRows) {
    for (int u = t; u < kGramRows * m; u += 256) {
      const int col = u / kGramRows, rr = u % kGramRows;
      const int64_t row = r0 + rr;
      const bool ok = row < r_end;
      S[rr][col] = ok ? colS[col][row] : 0.0;
      HS[rr][col] = ok ? colH[col][row] : 0.0;
    }
    __syncthreads();
    for (int i = 0; i < ne; ++i) {
      const int aa = ea[i], bb = eb[i];
      double sacc = acc[i];
      if (eg[i]) {
        for (int rr = g; rr < kGramRows; rr += ngroups) sacc = fma(S[rr][aa], S[rr][bb], sacc);
      } else {
        for (int rr = g; rr < kGramRows; rr += ngroups) sacc = fma(S[rr][aa], HS[rr][bb], sacc);
      }
      acc[i] = sacc;
    }
    __syncthreads();
  }
  double* out = part + ((int64_t)chunk * s + j) * Emax;
  if (E <= 256) {
    red[t] = (g < ngroups && ne > 0) ? acc[0] : 0.0;
    __syncthreads();
    if (t < E) {
      double sum = 0.0;
      for (int gg = 0; gg < ngroups; ++gg) sum += red[gg * E + t];
      out[t] = sum;
    }
  } else {
    int i = 0;
    for (int e = t; e < E && i < ne; e += 256, ++i) out[e] = acc[i];
  }
}

// ------------------------------------------------------------------------------------------------ warp solver
// Round-robin (circle method) pairing of mp (even) indices: round r, pair i.
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

__device__ __forceinline__ double sort_key(double x) { return isnan(x) ? CUDART_INF : x; }

// Jacobi rotation for a 2 x 2 symmetric [app apq; apq aqq]: returns t (tan), c, s; rotated = |apq| > thr
__device__ __forceinline__ bool jac_rot(double app, double aqq, double apq, double thr, double& t, double& c,
                                        double& s) {
  if (!(fabs(apq) > thr)) {
    t = 0.0; c = 1.0; s = 0.0;
    return false;
  }
  const double theta = (aqq - app) / (2.0 * apq);
  const double at = fabs(theta);
  double tt;
  if (at > 1e150) tt = 0.5 / theta;
  else tt = 1.0 / (at + sqrt(at * at + 1.0));
  if (theta < 0.0) tt = -tt;
  t = tt;
  c = 1.0 / sqrt(tt * tt + 1.0);
  s = tt * c;
  return true;
}

// Cyclic Jacobi on the symmetric mp x mp matrix K (row-major, stride ld) in shared memory, accumulating the
// eigenvectors into Z (initialised here). Indices >= m are padding (zero rows/cols, never rotated).
__device__ void warp_jacobi(double* K, double* Z, int m, int mp, int ld, double* rot, int lane) {
  for (int idx = lane; idx < mp * mp; idx += 32) {
    const int i = idx / mp, j = idx % mp;
    Z[i * ld + j] = (i == j) ? 1.0 : 0.0;
    if (i >= m || j >= m) K[i * ld + j] = 0.0;
  }
  double nrm = 0.0;
  for (int idx = lane; idx < m * m; idx += 32) {
    const double v = K[(idx / m) * ld + idx % m];
    nrm += v * v;
  }
  for (int off = 16; off > 0; off >>= 1) nrm += __shfl_xor_sync(0xffffffffu, nrm, off);
  const double thr = kJacobiTolSmall * sqrt(nrm);
  __syncwarp();
  const int P = mp / 2;
  for (int sweep = 0; sweep < kJacobiMaxSweeps; ++sweep) {
    int any = 0;
    for (int r = 0; r < mp - 1; ++r) {
      for (int i = lane; i < P; i += 32) {
        int p, q;
        rr_pair(mp, r, i, p, q);
        double t, c, s;
        bool did = false;
        if (q < m) did = jac_rot(K[p * ld + p], K[q * ld + q], K[p * ld + q], thr, t, c, s);
        else { t = 0.0; c = 1.0; s = 0.0; }
        rot[3 * i] = c;
        rot[3 * i + 1] = s;
        rot[3 * i + 2] = t;
        any |= did ? 1 : 0;
      }
      __syncwarp();
      // 2 x 2 blocks (pa <= pb)
      for (int task = lane; task < P * (P + 1) / 2; task += 32) {
        int pb = 0;
        while ((pb + 1) * (pb + 2) / 2 <= task) ++pb;
        const int pa = task - pb * (pb + 1) / 2;
        int p, q, u, v;
        rr_pair(mp, r, pa, p, q);
        rr_pair(mp, r, pb, u, v);
        const double ca = rot[3 * pa], sa = rot[3 * pa + 1], ta = rot[3 * pa + 2];
        if (pa == pb) {
          if (sa != 0.0) {
            const double apq = K[p * ld + q];
            K[p * ld + p] -= ta * apq;
            K[q * ld + q] += ta * apq;
            K[p * ld + q] = 0.0;
            K[q * ld + p] = 0.0;
          }
        } else {
          const double cb = rot[3 * pb], sb = rot[3 * pb + 1];
          const double xpu = K[p * ld + u], xpv = K[p * ld + v], xqu = K[q * ld + u], xqv = K[q * ld + v];
          const double ypu = ca * xpu - sa * xqu, ypv = ca * xpv - sa * xqv;
          const double yqu = sa * xpu + ca * xqu, yqv = sa * xpv + ca * xqv;
          const double zpu = cb * ypu - sb * ypv, zpv = sb * ypu + cb * ypv;
          const double zqu = cb * yqu - sb * yqv, zqv = sb * yqu + cb * yqv;
          K[p * ld + u] = zpu; K[p * ld + v] = zpv; K[q * ld + u] = zqu; K[q * ld + v] = zqv;
          K[u * ld + p] = zpu; K[v * ld + p] = zpv; K[u * ld + q] = zqu; K[v * ld + q] = zqv;
        }
      }
      // eigenvectors Z <- Z J
      for (int task = lane; task < mp * P; task += 32) {
        const int row = task / P, pb = task % P;
        int u, v;
        rr_pair(mp, r, pb, u, v);
        const double cb = rot[3 * pb], sb = rot[3 * pb + 1];
        if (sb != 0.0) {
          const double zu = Z[row * ld + u], zv = Z[row * ld + v];
          Z[row * ld + u] = cb * zu - sb * zv;
          Z[row * ld + v] = sb * zu + cb * zv;
        }
      }
      __syncwarp();
    }
    if (!__any_sync(0xffffffffu, any)) break;
  }
}

struct WarpSmem {
  double *Ga, *Gb, *K, *L, *Z, *D, *rot, *C, *U;
  int* sel;
};

// Solve the m x m pencil (leading m x m of Ga, Gb) for the qj smallest pairs; C (m x qj, row-major stride qj).
// Returns true on success (pivots and Theorem 1 check passed).
__device__ bool warp_try_solve(const WarpSmem& w, int m, int qj, int ld, int lane) {
  // unit column scaling
  int bad = 0;
  for (int i = lane; i < m; i += 32) {
    const double d = w.Gb[i * ld + i];
    if (!(d > 0.0) || !isfinite(d)) bad = 1;
    w.D[i] = bad ? 1.0 : 1.0 / sqrt(d);
  }
  if (__any_sync(0xffffffffu, bad)) return false;
  __syncwarp();
  for (int idx = lane; idx < m * m; idx += 32) {
    const int i = idx / m, j = idx % m;
    const double dd = w.D[i] * w.D[j];
    w.K[i * ld + j] = w.Ga[i * ld + j] * dd;
    w.L[i * ld + j] = w.Gb[i * ld + j] * dd;
  }
  __syncwarp();
  // Cholesky of the unit-diagonal Gram (left-looking, lower L)
  for (int c = 0; c < m; ++c) {
    if (lane == 0) {
      double v = w.L[c * ld + c];
      for (int l = 0; l < c; ++l) v -= w.L[c * ld + l] * w.L[c * ld + l];
      w.L[c * ld + c] = (v > 0.0) ? sqrt(v) : -1.0;
    }
    __syncwarp();
    const double piv = w.L[c * ld + c];
    if (!(piv >= kPivotTol)) return false;
    for (int r = c + 1 + lane; r < m; r += 32) {
      double v = w.L[r * ld + c];
      for (int l = 0; l < c; ++l) v -= w.L[r * ld + l] * w.L[c * ld + l];
      w.L[r * ld + c] = v / piv;
    }
    __syncwarp();
  }
  // Y = L^{-1} K (column per lane, in place in K)
  for (int col = lane; col < m; col += 32) {
    for (int i = 0; i < m; ++i) {
      double v = w.K[i * ld + col];
      for (int l = 0; l < i; ++l) v -= w.L[i * ld + l] * w.K[l * ld + col];
      w.K[i * ld + col] = v / w.L[i * ld + i];
    }
  }
  __syncwarp();
  // Z = Y^T, then K = L^{-1} Z (column per lane), then symmetrise into K
  for (int idx = lane; idx < m * m; idx += 32) {
    const int i = idx / m, j = idx % m;
    w.Z[i * ld + j] = w.K[j * ld + i];
  }
  __syncwarp();
  for (int col = lane; col < m; col += 32) {
    for (int i = 0; i < m; ++i) {
      double v = w.Z[i * ld + col];
      for (int l = 0; l < i; ++l) v -= w.L[i * ld + l] * w.Z[l * ld + col];
      w.Z[i * ld + col] = v / w.L[i * ld + i];
    }
  }
  __syncwarp();
  for (int idx = lane; idx < m * m; idx += 32) {
    const int i = idx / m, j = idx % m;
    w.K[i * ld + j] = 0.5 * (w.Z[i * ld + j] + w.Z[j * ld + i]);
  }
  __syncwarp();
  const int mp = (m + 1) & ~1;
  warp_jacobi(w.K, w.Z, m, mp, ld, w.rot, lane);
  __syncwarp();
  // select the qj smallest eigenvalues (ascending; ties by index)
  // rank by the strict total order (value, index) with NaN as +inf, so the ranks are a permutation
  for (int i = lane; i < m; i += 32) {
    const double ti = sort_key(w.K[i * ld + i]);
    int rank = 0;
    for (int l = 0; l < m; ++l) {
      const double tl = sort_key(w.K[l * ld + l]);
      rank += (tl < ti || (tl == ti && l < i)) ? 1 : 0;
    }
    if (rank < qj) w.sel[rank] = i;
  }
  __syncwarp();
  // C = D L^{-T} Z[:, sel] (back substitution, column per lane)
  for (int tcol = lane; tcol < qj; tcol += 32) {
    const int zc = w.sel[tcol];
    for (int i = m - 1; i >= 0; --i) {
      double v = w.Z[i * ld + zc];
      for (int l = i + 1; l < m; ++l) v -= w.L[l * ld + i] * w.C[l * qj + tcol];
      w.C[i * qj + tcol] = v / w.L[i * ld + i];
    }
    for (int i = 0; i < m; ++i) w.C[i * qj + tcol] *= w.D[i];
  }
  __syncwarp();
  // Theorem 1: X_bar_j has full rank iff C_X is non-singular; smallest singular value by one-sided Jacobi
  double smin;
  if (qj == 1) {
    smin = fabs(w.C[0]);
  } else {
    for (int idx = lane; idx < qj * qj; idx += 32) w.U[idx] = w.C[idx];   // U = C_X (row-major, stride qj)
    __syncwarp();
    const int qp = (qj + 1) & ~1;
    for (int sweep = 0; sweep < kJacobiMaxSweeps; ++sweep) {
      int any = 0;
      for (int r = 0; r < qp - 1; ++r) {
        for (int i = lane; i < qp / 2; i += 32) {
          int p, q;
          rr_pair(qp, r, i, p, q);
          if (q >= qj) continue;
          double al = 0.0, be = 0.0, ga = 0.0;
          for (int k = 0; k < qj; ++k) {
            const double up = w.U[k * qj + p], uq = w.U[k * qj + q];
            al += up * up; be += uq * uq; ga += up * uq;
          }
          if (fabs(ga) > 1e-15 * sqrt(al * be) && ga != 0.0) {
            any = 1;
            const double zeta = (be - al) / (2.0 * ga);
            double tt = 1.0 / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
            if (zeta < 0.0) tt = -tt;
            const double c = 1.0 / sqrt(1.0 + tt * tt), s = c * tt;
            for (int k = 0; k < qj; ++k) {
              const double up = w.U[k * qj + p], uq = w.U[k * qj + q];
              w.U[k * qj + p] = c * up - s * uq;
              w.U[k * qj + q] = s * up + c * uq;
            }
          }
        }
        __syncwarp();
      }
      if (!__any_sync(0xffffffffu, any)) break;
    }
    double mn = 1e300;
    for (int col = lane; col < qj; col += 32) {
      double nn = 0.0;
      for (int k = 0; k < qj; ++k) nn += w.U[k * qj + col] * w.U[k * qj + col];
      mn = fmin(mn, sqrt(nn));
    }
    for (int off = 16; off > 0; off >>= 1) mn = fmin(mn, __shfl_xor_sync(0xffffffffu, mn, off));
    smin = mn;
  }
  return smin >= kAlphaTol;
}

// One warp per sub-block. coef slot j: 3q x q column-major, rows [C_X (qj); C_W (qj); C_P (qj)], ld 3q.
__global__ void block_solve_kernel(BlockArgs a, int s, const double* __restrict__ part, int nchunk, int Emax,
                                   double* __restrict__ coef, int* __restrict__ flags, int* __restrict__ counters,
                                   int ld, int warps_per_block) {
  extern __shared__ double smem[];
  const int warp = threadIdx.x / 32, lane = threadIdx.x & 31;
  const int j = blockIdx.x * warps_per_block + warp;
  if (j >= s) return;
  const int per = 5 * ld * ld + ld + 3 * (ld / 2) + ld * kMaxSbsize + kMaxSbsize * kMaxSbsize + ld;
  double* base = smem + (size_t)warp * per;
  WarpSmem w;
  w.Ga = base;
  w.Gb = w.Ga + ld * ld;
  w.K = w.Gb + ld * ld;
  w.L = w.K + ld * ld;
  w.Z = w.L + ld * ld;
  w.D = w.Z + ld * ld;
  w.rot = w.D + ld;
  w.C = w.rot + 3 * (ld / 2);
  w.U = w.C + ld * kMaxSbsize;
  w.sel = reinterpret_cast<int*>(w.U + kMaxSbsize * kMaxSbsize);

  const int c0 = j * a.q;
  const int qj = min(a.q, a.k_act - c0);
  const int mfull = (a.has_p ? 3 : 2) * qj;
  const int Eh = mfull * (mfull + 1) / 2;
  // sum partials (fixed chunk order) and unpack both Grams, mirrored
  for (int e = lane; e < 2 * Eh; e += 32) {
    double v = 0.0;
    for (int c = 0; c < nchunk; ++c) v += part[((int64_t)c * s + j) * Emax + e];
    const bool isB = e >= Eh;
    const int r = isB ? e - Eh : e;
    int b = 0;
    while ((b + 1) * (b + 2) / 2 <= r) ++b;
    const int aa = r - b * (b + 1) / 2;
    double* G = isB ? w.Gb : w.Ga;
    G[aa * ld + b] = v;
    G[b * ld + aa] = v;
  }
  __syncwarp();
  int flag = 0;
  int m = mfull;
  bool ok = warp_try_solve(w, m, qj, ld, lane);
  if (!ok && a.has_p) {
    flag = 1;                        // back-track without P (Section 3, Theorems 1-2)
    m = 2 * qj;
    __syncwarp();
    ok = warp_try_solve(w, m, qj, ld, lane);
  }
  if (!ok) flag = 2;
  __syncwarp();
  double* out = coef + (int64_t)j * 3 * a.q * a.q;
  const int ldc = 3 * a.q;
  for (int idx = lane; idx < 3 * qj * qj; idx += 32) {
    const int row = idx % (3 * qj), col = idx / (3 * qj);
    double v;
    if (ok) v = row < m ? w.C[row * qj + col] : 0.0;
    else v = (row == col) ? 1.0 : 0.0;           // keep X_j
    out[row + (int64_t)col * ldc] = v;
  }
  if (lane == 0) {
    if (flags) flags[j] = flag;
    if (flag == 1) atomicAdd(counters + 0, 1);
    if (flag == 2) atomicAdd(counters + 1, 1);
  }
}

// P_j <- W_j C_W + P_j C_P ; X_j <- X_j C_X + P_j  (one thread per row, one block-row of grid per sub-block)
template <int Q>
__global__ void __launch_bounds__(256)
block_update_kernel(double* __restrict__ X, const double* __restrict__ W, double* __restrict__ P, int64_t ld,
                    int64_t n, int k_act, int q, int has_p, const double* __restrict__ coef) {
  const int j = blockIdx.y;
  const int c0 = j * q;
  const int qj = min(q, k_act - c0);
  const int ldc = 3 * q;
  __shared__ double Cs[3 * Q * Q];
  for (int idx = threadIdx.x; idx < 3 * qj * qj; idx += blockDim.x) {
    const int row = idx % (3 * qj), col = idx / (3 * qj);
    Cs[row + col * 3 * Q] = coef[(int64_t)j * 3 * q * q + row + (int64_t)col * ldc];
  }
  __syncthreads();
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
    double x[Q], w[Q], p[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      const bool ok = i < qj;
      const int64_t o = (int64_t)(c0 + i) * ld + r;
      x[i] = ok ? X[o] : 0.0;
      w[i] = ok ? W[o] : 0.0;
      p[i] = (ok && has_p) ? P[o] : 0.0;
    }
#pragma unroll
    for (int t = 0; t < Q; ++t) {
      if (t >= qj) break;
      const double* cc = Cs + t * 3 * Q;
      double pn = 0.0, xn = 0.0;
#pragma unroll
      for (int i = 0; i < Q; ++i) {
        if (i < qj) {
          pn = fma(w[i], cc[qj + i], pn);
          pn = fma(p[i], cc[2 * qj + i], pn);
          xn = fma(x[i], cc[i], xn);
        }
      }
      const int64_t o = (int64_t)(c0 + t) * ld + r;
      P[o] = pn;
      X[o] = xn + pn;
    }
  }
}

int block_solve_ld(int q) { return ((3 * q + 1) & ~1); }

}  // namespace

size_t block_gram_part_elems(int64_t n, int k_act, int q) {
  const int64_t s = ceil_div(k_act, q);
  const int64_t Emax = entries(3 * q);
  const int64_t nchunk_max = 64;
  (void)n;
  return (size_t)(s * Emax * nchunk_max);
}

cudaError_t block_gram(const BlockArgs& a, double* part, size_t part_capacity, int* nchunk_out, cudaStream_t s) {
  if (a.q < 1 || a.q > kMaxSbsize) return cudaErrorInvalidValue;
  const int sb = (int)ceil_div(a.k_act, a.q);
  const int Emax = entries(3 * a.q);
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int64_t nchunk = ceil_div(4LL * sms, sb);
  const int64_t maxc = ceil_div(a.n, 512);
  if (nchunk > maxc) nchunk = maxc;
  if (nchunk > 64) nchunk = 64;
  if (nchunk < 1) nchunk = 1;
  while (nchunk > 1 && (size_t)(nchunk * sb * Emax) > part_capacity) --nchunk;
  if ((size_t)(nchunk * sb * Emax) > part_capacity) return cudaErrorInvalidValue;
  int64_t rows = ceil_div(a.n, nchunk);
  rows = ceil_div(rows, kGramRows) * kGramRows;
  nchunk = ceil_div(a.n, rows);
  dim3 grid(sb, (unsigned)nchunk);
  block_gram_kernel<<<grid, 256, 0, s>>>(a, sb, rows, part, Emax);
  count_launch();
  *nchunk_out = (int)nchunk;
  return cudaGetLastError();
}

cudaError_t block_solve(const BlockArgs& a, const double* part, int nchunk, double* coef, int* flags,
                        int* counters, cudaStream_t s) {
  const int sb = (int)ceil_div(a.k_act, a.q);
  const int ld = block_solve_ld(a.q);
  const size_t per = (size_t)(5 * ld * ld + ld + 3 * (ld / 2) + ld * kMaxSbsize + kMaxSbsize * kMaxSbsize + ld) *
                     sizeof(double);
  int wpb = (int)(64 * 1024 / per);
  if (wpb > 8) wpb = 8;
  if (wpb < 1) wpb = 1;
  const size_t smem = per * wpb;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(block_solve_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  block_solve_kernel<<<(unsigned)ceil_div(sb, wpb), 32 * wpb, smem, s>>>(a, sb, part, nchunk, entries(3 * a.q), coef,
                                                                        flags, counters, ld, wpb);
  count_launch();
  return cudaGetLastError();
}

cudaError_t block_update(double* X, const double* W, double* P, int64_t ld, int64_t n, int k_act, int q, int has_p,
                         const double* coef, cudaStream_t s) {
  const int sb = (int)ceil_div(k_act, q);
  int64_t bx = ceil_div(n, 256);
  if (bx > 2048) bx = 2048;
  dim3 grid((unsigned)bx, sb);
  if (q <= 1) block_update_kernel<1><<<grid, 256, 0, s>>>(X, W, P, ld, n, k_act, q, has_p, coef);
  else if (q <= 2) block_update_kernel<2><<<grid, 256, 0, s>>>(X, W, P, ld, n, k_act, q, has_p, coef);
  else if (q <= 4) block_update_kernel<4><<<grid, 256, 0, s>>>(X, W, P, ld, n, k_act, q, has_p, coef);
  else if (q <= 8) block_update_kernel<8><<<grid, 256, 0, s>>>(X, W, P, ld, n, k_act, q, has_p, coef);
  else if (q <= 16) block_update_kernel<16><<<grid, 256, 0, s>>>(X, W, P, ld, n, k_act, q, has_p, coef);
  else return cudaErrorInvalidValue;
  count_launch();
  return cudaGetLastError();
}

}  // namespace ppcg
