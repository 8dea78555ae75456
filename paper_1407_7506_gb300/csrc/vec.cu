// Column-wise kernels of Algorithm 3: the Ritz residual with the preconditioner fused (steps 25 and 8), column
// norms, column gathers for locking/compaction (steps 27-29), the output phase convention, and small helpers.
// All are HBM-bound streaming kernels (one read and at most one write per element).
#include "ppcg_internal.h"

namespace ppcg {

namespace {

constexpr int kRows = 64;   // rows per tile; must match gemm_nn's row tile (norm_part layout)

constexpr int kColsPerThread = 8;   // columns per thread: one reciprocal of the diagonal serves all of them

// RESID: R = HX - lam_c X, else R = W (already AX - XM). Then W = T R with T = 1 / max(dg - sigma, delta), and the
// per-tile column sums of R^2 go to norm_part. A block covers 64 rows x 32 columns; each thread forms the reciprocal
// of its row once (FP64 division is a long instruction sequence on GB300's narrow FP64 pipe) and applies it to 8
// columns.
template <bool RESID>
__global__ void __launch_bounds__(256)
precond_kernel(const double* __restrict__ X, const double* __restrict__ HX, double* W, int64_t ld, int64_t n, int m,
               const double* __restrict__ lam, const double* __restrict__ dg, double sigma, double delta,
               const double* __restrict__ tinvp, double* __restrict__ norm_part) {
  const int r_loc = threadIdx.x % kRows;
  const int c_loc = threadIdx.x / kRows;          // 4 column lanes; columns c0 + c_loc + 4 j
  const int64_t r = (int64_t)blockIdx.x * kRows + r_loc;
  const int c0 = blockIdx.y * 4 * kColsPerThread;
  const double tinv = r < n ? (tinvp ? tinvp[r] : 1.0 / fmax(dg[r] - sigma, delta)) : 0.0;
  double sq[kColsPerThread];
#pragma unroll
  for (int j = 0; j < kColsPerThread; ++j) {
    const int c = c0 + c_loc + 4 * j;
    sq[j] = 0.0;
    if (r < n && c < m) {
      const int64_t o = (int64_t)c * ld + r;
      const double rr = RESID ? HX[o] - lam[c] * X[o] : W[o];
      sq[j] = rr * rr;
      W[o] = rr * tinv;
    }
  }
  // reduce each column over the 64 rows of the tile: warps 2 c_loc and 2 c_loc + 1
  __shared__ double red[8][kColsPerThread];
  const int warp = threadIdx.x / 32;
#pragma unroll
  for (int j = 0; j < kColsPerThread; ++j) {
    double v = sq[j];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    if ((threadIdx.x & 31) == 0) red[warp][j] = v;
  }
  __syncthreads();
  if (threadIdx.x < 4 * kColsPerThread) {
    const int cl = threadIdx.x % 4, j = threadIdx.x / 4;
    const int c = c0 + cl + 4 * j;
    if (c < m) norm_part[(int64_t)blockIdx.x * m + c] = red[2 * cl][j] + red[2 * cl + 1][j];
  }
}

__global__ void reduce_colnorms_kernel(const double* __restrict__ part, int64_t tiles, int m, double* out) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= m) return;
  double s = 0.0;
  for (int64_t t = 0; t < tiles; ++t) s += part[t * m + c];
  out[c] = s;
}

__global__ void gather_cols_kernel(const double* __restrict__ in, int64_t ldi, double* __restrict__ out, int64_t ldo,
                                   int64_t n, const int* __restrict__ idx) {
  const int j = blockIdx.y;
  const int src = idx[j];
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x)
    out[(int64_t)j * ldo + r] = (src >= 0) ? in[(int64_t)src * ldi + r] : 0.0;
}

// One block per column: norm^2 and the (first) index of the largest |x|; then scale by sign(x_p)/norm.
__global__ void __launch_bounds__(1024) phase_kernel(double* X, int64_t ld, int64_t n) {
  double* x = X + (int64_t)blockIdx.x * ld;
  double sq = 0.0, best = -1.0;
  int64_t bi = 0;
  for (int64_t r = threadIdx.x; r < n; r += blockDim.x) {
    const double v = x[r];
    sq += v * v;
    const double a = fabs(v);
    if (a > best) { best = a; bi = r; }   // rows visited ascending: keeps the first maximum
  }
  __shared__ double s_sq[32], s_best[32];
  __shared__ long long s_bi[32];
  for (int off = 16; off > 0; off >>= 1) {
    sq += __shfl_down_sync(0xffffffffu, sq, off);
    const double ob = __shfl_down_sync(0xffffffffu, best, off);
    const long long oi = __shfl_down_sync(0xffffffffu, (long long)bi, off);
    if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
  }
  const int warp = threadIdx.x / 32, lane = threadIdx.x & 31;
  if (lane == 0) { s_sq[warp] = sq; s_best[warp] = best; s_bi[warp] = bi; }
  __syncthreads();
  __shared__ double scale;
  if (threadIdx.x == 0) {
    const int nw = (blockDim.x + 31) / 32;
    double t = 0.0, b = -1.0;
    long long i = 0;
    for (int w = 0; w < nw; ++w) {
      t += s_sq[w];
      if (s_best[w] > b || (s_best[w] == b && s_bi[w] < i)) { b = s_best[w]; i = s_bi[w]; }
    }
    const double sgn = (x[i] < 0.0) ? -1.0 : 1.0;
    scale = sgn / sqrt(t);
  }
  __syncthreads();
  const double sc = scale;
  for (int64_t r = threadIdx.x; r < n; r += blockDim.x) x[r] *= sc;
}

// rho[p] = scale * sum_{c < k} X[p, c]^2 : the Hellmann-Feynman gradient of the sum of the k Ritz values with
// respect to the potential (one thread per grid point; every column read is coalesced across the warp)
__global__ void __launch_bounds__(256)
density_kernel(const double* __restrict__ X, int64_t ld, int64_t n, int k, double scale, double* __restrict__ rho) {
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
    int c = 0;
    for (; c + 4 <= k; c += 4) {
      const double a = __ldg(X + p + (int64_t)c * ld), b = __ldg(X + p + (int64_t)(c + 1) * ld);
      const double d = __ldg(X + p + (int64_t)(c + 2) * ld), e = __ldg(X + p + (int64_t)(c + 3) * ld);
      s0 = fma(a, a, s0); s1 = fma(b, b, s1); s2 = fma(d, d, s2); s3 = fma(e, e, s3);
    }
    for (; c < k; ++c) {
      const double a = __ldg(X + p + (int64_t)c * ld);
      s0 = fma(a, a, s0);
    }
    rho[p] = scale * ((s0 + s1) + (s2 + s3));
  }
}

// ---- complex Hermitian (Bloch) problems, solved in the real form R = [[Re H, -Im H], [Im H, Re H]] of order 2n:
// a complex vector z = u + i v is the real column [u; v]; J [u; v] = [-v; u] represents i z.

// Complex start block Z (n x kt, interleaved re/im, leading dimension ldz complex entries) -> real form X
// (2n x 2kt): column 2j = [Re z_j; Im z_j], column 2j+1 = J of it, so every pair spans a J-invariant plane.
__global__ void cplx_to_realform_kernel(const double* __restrict__ Z, int64_t ldz, int64_t n, double* __restrict__ X,
                                        int64_t ldx) {
  const int j = blockIdx.y;
  const double* z = Z + 2 * (int64_t)j * ldz;
  double* a = X + (int64_t)(2 * j) * ldx;
  double* b = a + ldx;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
    const double re = z[2 * p], im = z[2 * p + 1];
    a[p] = re;
    a[p + n] = im;
    b[p] = -im;
    b[p + n] = re;
  }
}

// Output column j of a complex handle: z = Y[0:n, 2j] + i Y[n:2n, 2j], scaled to unit norm with its entry of
// largest modulus (lowest index on ties) real positive; one block per column.
__global__ void __launch_bounds__(1024)
realform_to_cplx_kernel(const double* __restrict__ Y, int64_t ldy, int64_t n, double* __restrict__ Z, int64_t ldz) {
  const double* u = Y + (int64_t)(2 * blockIdx.x) * ldy;
  const double* v = u + n;
  double* z = Z + 2 * (int64_t)blockIdx.x * ldz;
  double sq = 0.0, best = -1.0;
  int64_t bi = 0;
  for (int64_t r = threadIdx.x; r < n; r += blockDim.x) {
    const double a2 = u[r] * u[r] + v[r] * v[r];
    sq += a2;
    if (a2 > best) { best = a2; bi = r; }
  }
  __shared__ double s_sq[32], s_best[32];
  __shared__ long long s_bi[32];
  for (int off = 16; off > 0; off >>= 1) {
    sq += __shfl_down_sync(0xffffffffu, sq, off);
    const double ob = __shfl_down_sync(0xffffffffu, best, off);
    const long long oi = __shfl_down_sync(0xffffffffu, (long long)bi, off);
    if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
  }
  const int warp = threadIdx.x / 32, lane = threadIdx.x & 31;
  if (lane == 0) { s_sq[warp] = sq; s_best[warp] = best; s_bi[warp] = bi; }
  __syncthreads();
  __shared__ double sc_re, sc_im;
  if (threadIdx.x == 0) {
    const int nw = (blockDim.x + 31) / 32;
    double t = 0.0, b = -1.0;
    long long i = 0;
    for (int w = 0; w < nw; ++w) {
      t += s_sq[w];
      if (s_best[w] > b || (s_best[w] == b && s_bi[w] < i)) { b = s_best[w]; i = s_bi[w]; }
    }
    const double mod = sqrt(u[i] * u[i] + v[i] * v[i]);
    const double inv = (mod > 0.0 ? 1.0 / mod : 0.0) / sqrt(t);   // conj(z_p) / |z_p| / ||z||
    sc_re = u[i] * inv;
    sc_im = -v[i] * inv;
  }
  __syncthreads();
  const double cr = sc_re, ci = sc_im;
  for (int64_t r = threadIdx.x; r < n; r += blockDim.x) {
    const double a = u[r], b = v[r];
    z[2 * r] = a * cr - b * ci;
    z[2 * r + 1] = a * ci + b * cr;
  }
}

// rho[p] = scale * sum_{c < k} |Z[p, c]|^2 for a complex block (interleaved, leading dimension ldz complex)
__global__ void __launch_bounds__(256)
density_c_kernel(const double* __restrict__ Z, int64_t ldz, int64_t n, int k, double scale, double* __restrict__ rho) {
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
    double s0 = 0.0, s1 = 0.0;
    for (int c = 0; c < k; ++c) {
      const double2 z = __ldg(reinterpret_cast<const double2*>(Z + 2 * (p + (int64_t)c * ldz)));
      s0 = fma(z.x, z.x, s0);
      s1 = fma(z.y, z.y, s1);
    }
    rho[p] = scale * (s0 + s1);
  }
}

__global__ void make_diag_kernel(const double* __restrict__ V, double six_inv_h2, int64_t n, double* dg) {
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x)
    dg[r] = six_inv_h2 + V[r];
}

__global__ void check_finite_kernel(const double* __restrict__ v, int m, int* bad) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x)
    if (!isfinite(v[i])) atomicAdd(bad, 1);
}

// Y = G - I in place (m x m, leading dimension m) and out[0] = ||Y||_F^2 (one CTA, fixed summation order).
__global__ void __launch_bounds__(1024) eye_residual_kernel(double* G, int m, double* out) {
  double acc = 0.0;
  for (int64_t e = threadIdx.x; e < (int64_t)m * m; e += blockDim.x) {
    const int i = (int)(e % m), j = (int)(e / m);
    const double y = G[e] - (i == j ? 1.0 : 0.0);
    G[e] = y;
    acc = fma(y, y, acc);
  }
  __shared__ double red[1024];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int off = blockDim.x / 2; off > 0; off >>= 1) {
    if ((int)threadIdx.x < off) red[threadIdx.x] += red[threadIdx.x + off];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = red[0];
}

// Z = a Y + b I (m x m)
__global__ void scaled_plus_identity_kernel(const double* __restrict__ Y, int m, double a, double b, double* Z) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)m * m;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % m), j = (int)(e / m);
    Z[e] = a * Y[e] + (i == j ? b : 0.0);
  }
}

__global__ void add_diag_kernel(double* Z, int m, double b) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) Z[i + (int64_t)i * m] += b;
}

}  // namespace

int64_t norm_row_tiles(int64_t n) { return ceil_div(n, kRows); }

// Rayleigh-Ritz Grams with kl leading locked columns (m x m, leading dimension m, columns kl.. computed): the
// locked block becomes I (G) and diag(lam_lock) (M), and the lower-left blocks mirror the computed upper-right ones.
__global__ void locked_gram_fill_kernel(double* G, double* M, int m, int kl, const double* __restrict__ lam_lock) {
  const int64_t cnt = (int64_t)kl * m;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < cnt; e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % m), j = (int)(e / m);      // column j < kl
    const int64_t o = i + (int64_t)j * m;
    if (i < kl) {
      G[o] = (i == j) ? 1.0 : 0.0;
      M[o] = (i == j) ? lam_lock[i] : 0.0;
    } else {
      G[o] = G[j + (int64_t)i * m];
      M[o] = M[j + (int64_t)i * m];
    }
  }
}

cudaError_t locked_gram_fill(double* G, double* M, int m, int kl, const double* lam_lock, cudaStream_t s) {
  if (kl <= 0) return cudaSuccess;
  const int64_t cnt = (int64_t)kl * m;
  const int64_t b = ceil_div(cnt, 256);
  locked_gram_fill_kernel<<<(unsigned)(b < 4096 ? b : 4096), 256, 0, s>>>(G, M, m, kl, lam_lock);
  count_launch();
  return cudaGetLastError();
}

// Gs = G_aa - T (ka x ka, leading dimension ka; G_aa read from the k_t x k_t Gram at offset kl); a Schur pivot
// Gs_ii below pivot_tol^2 G_aa,ii (the active column nearly inside the span of the locked ones) flags a breakdown
__global__ void locked_schur_kernel(const double* __restrict__ G, int kt, int kl, const double* __restrict__ T,
                                    double pivot_tol, double* __restrict__ Gs, int* flag) {
  const int ka = kt - kl;
  const int64_t cnt = (int64_t)ka * ka;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < cnt; e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % ka), j = (int)(e / ka);
    const double g = G[(kl + i) + (int64_t)(kl + j) * kt];
    const double v = g - T[e];
    Gs[e] = v;
    if (i == j && !(v >= pivot_tol * pivot_tol * g)) atomicOr(flag, kFlagCholBreakdown);
  }
}

// R^{-1} of G = [[I, G_la], [G_la^T, G_aa]] from U = G_la Ra^{-1} and Ra^{-1} (Ra^T Ra = G_aa - G_la^T G_la):
// R^{-1} = [[I, -U], [0, Ra^{-1}]] (k_t x k_t, leading dimension k_t)
__global__ void locked_rinv_fill_kernel(double* __restrict__ Rinv, int kt, int kl, const double* __restrict__ U,
                                        const double* __restrict__ Rainv) {
  const int ka = kt - kl;
  const int64_t cnt = (int64_t)kt * kt;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < cnt; e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % kt), j = (int)(e / kt);
    double v;
    if (j < kl) v = (i == j) ? 1.0 : 0.0;
    else if (i < kl) v = -U[i + (int64_t)(j - kl) * kl];
    else v = Rainv[(i - kl) + (int64_t)(j - kl) * ka];
    Rinv[e] = v;
  }
}

cudaError_t locked_schur(const double* G, int kt, int kl, const double* T, double pivot_tol, double* Gs, int* flag,
                         cudaStream_t s) {
  const int64_t cnt = (int64_t)(kt - kl) * (kt - kl);
  const int64_t b = ceil_div(cnt, 256);
  locked_schur_kernel<<<(unsigned)(b < 4096 ? (b < 1 ? 1 : b) : 4096), 256, 0, s>>>(G, kt, kl, T, pivot_tol, Gs,
                                                                                   flag);
  count_launch();
  return cudaGetLastError();
}

cudaError_t locked_rinv_fill(double* Rinv, int kt, int kl, const double* U, const double* Rainv, cudaStream_t s) {
  const int64_t cnt = (int64_t)kt * kt;
  const int64_t b = ceil_div(cnt, 256);
  locked_rinv_fill_kernel<<<(unsigned)(b < 4096 ? b : 4096), 256, 0, s>>>(Rinv, kt, kl, U, Rainv);
  count_launch();
  return cudaGetLastError();
}

cudaError_t eye_residual(double* G, int m, double* fro2, cudaStream_t s) {
  if (m <= 0) return cudaSuccess;
  eye_residual_kernel<<<1, 1024, 0, s>>>(G, m, fro2);
  count_launch();
  return cudaGetLastError();
}

cudaError_t scaled_plus_identity(const double* Y, int m, double a, double b, double* Z, cudaStream_t s) {
  if (m <= 0) return cudaSuccess;
  const int64_t blocks = ceil_div((int64_t)m * m, 256);
  scaled_plus_identity_kernel<<<(unsigned)(blocks < 1024 ? blocks : 1024), 256, 0, s>>>(Y, m, a, b, Z);
  count_launch();
  return cudaGetLastError();
}

cudaError_t add_diag(double* Z, int m, double b, cudaStream_t s) {
  if (m <= 0) return cudaSuccess;
  add_diag_kernel<<<(unsigned)ceil_div(m, 256), 256, 0, s>>>(Z, m, b);
  count_launch();
  return cudaGetLastError();
}

cudaError_t residual_diag(const double* X, const double* HX, int64_t ld, int64_t n, int m, const double* lam,
                          const ResidualArgs& ra, double* W, cudaStream_t s) {
  if (m <= 0) return cudaSuccess;
  dim3 grid((unsigned)norm_row_tiles(n), (unsigned)ceil_div(m, 4 * kColsPerThread));
  precond_kernel<true><<<grid, 256, 0, s>>>(X, HX, W, ld, n, m, lam, ra.dg, ra.sigma, ra.delta, ra.tinv,
                                            ra.norm_part);
  count_launch();
  return cudaGetLastError();
}

cudaError_t precond_norms(double* W, int64_t ld, int64_t n, int m, const ResidualArgs& ra, cudaStream_t s) {
  if (m <= 0) return cudaSuccess;
  dim3 grid((unsigned)norm_row_tiles(n), (unsigned)ceil_div(m, 4 * kColsPerThread));
  precond_kernel<false><<<grid, 256, 0, s>>>(nullptr, nullptr, W, ld, n, m, nullptr, ra.dg, ra.sigma, ra.delta,
                                             ra.tinv, ra.norm_part);
  count_launch();
  return cudaGetLastError();
}

__global__ void precond_diag_kernel(const double* __restrict__ dg, double sigma, double delta, int64_t n,
                                    double* __restrict__ tinv) {
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x)
    tinv[r] = 1.0 / fmax(dg[r] - sigma, delta);
}

cudaError_t precond_diag(const double* dg, double sigma, double delta, int64_t n, double* tinv, cudaStream_t s) {
  const int64_t b = ceil_div(n, 256);
  precond_diag_kernel<<<(unsigned)(b < 4096 ? b : 4096), 256, 0, s>>>(dg, sigma, delta, n, tinv);
  count_launch();
  return cudaGetLastError();
}

cudaError_t reduce_colnorms(const double* norm_part, int64_t tiles, int m, double* out, cudaStream_t s) {
  if (m <= 0) return cudaSuccess;
  reduce_colnorms_kernel<<<(unsigned)ceil_div(m, 128), 128, 0, s>>>(norm_part, tiles, m, out);
  count_launch();
  return cudaGetLastError();
}

cudaError_t gather_cols(const double* in, int64_t ldi, double* out, int64_t ldo, int64_t n, const int* idx, int m,
                        cudaStream_t s) {
  if (m <= 0) return cudaSuccess;
  const int64_t bx = ceil_div(n, 256);
  dim3 grid((unsigned)(bx < 1024 ? bx : 1024), m);
  gather_cols_kernel<<<grid, 256, 0, s>>>(in, ldi, out, ldo, n, idx);
  count_launch();
  return cudaGetLastError();
}

// rows[j] = the row of the nonzero entry of column j of an m x m matrix whose columns are unit vectors (one block
// per column; exactly one thread writes)
__global__ void unit_column_rows_kernel(const double* __restrict__ C, int m, int* __restrict__ rows) {
  const int j = blockIdx.x;
  for (int i = threadIdx.x; i < m; i += blockDim.x)
    if (C[i + (int64_t)j * m] != 0.0) rows[j] = i;
}

cudaError_t unit_column_rows(const double* C, int m, int* rows, cudaStream_t s) {
  if (m <= 0) return cudaSuccess;
  unit_column_rows_kernel<<<m, 256, 0, s>>>(C, m, rows);
  count_launch();
  return cudaGetLastError();
}

cudaError_t normalize_phase(double* X, int64_t ld, int64_t n, int m, double* /*scratch*/, cudaStream_t s) {
  if (m <= 0) return cudaSuccess;
  phase_kernel<<<m, 1024, 0, s>>>(X, ld, n);
  count_launch();
  return cudaGetLastError();
}

cudaError_t density(const double* X, int64_t ld, int64_t n, int k, double scale, double* rho, cudaStream_t s) {
  int64_t blocks = ceil_div(n, 256);
  if (blocks > 8192) blocks = 8192;
  density_kernel<<<(unsigned)blocks, 256, 0, s>>>(X, ld, n, k, scale, rho);
  count_launch();
  return cudaGetLastError();
}

cudaError_t cplx_to_realform(const double* Z, int64_t ldz, int64_t n, int kt, double* X, int64_t ldx,
                             cudaStream_t s) {
  if (kt <= 0) return cudaSuccess;
  const int64_t bx = ceil_div(n, 256);
  cplx_to_realform_kernel<<<dim3((unsigned)(bx < 1024 ? bx : 1024), (unsigned)kt), 256, 0, s>>>(Z, ldz, n, X, ldx);
  count_launch();
  return cudaGetLastError();
}

cudaError_t realform_to_cplx(const double* Y, int64_t ldy, int64_t n, int k, double* Z, int64_t ldz,
                             cudaStream_t s) {
  if (k <= 0) return cudaSuccess;
  realform_to_cplx_kernel<<<(unsigned)k, 1024, 0, s>>>(Y, ldy, n, Z, ldz);
  count_launch();
  return cudaGetLastError();
}

cudaError_t density_c(const double* Z, int64_t ldz, int64_t n, int k, double scale, double* rho, cudaStream_t s) {
  int64_t blocks = ceil_div(n, 256);
  if (blocks > 8192) blocks = 8192;
  density_c_kernel<<<(unsigned)blocks, 256, 0, s>>>(Z, ldz, n, k, scale, rho);
  count_launch();
  return cudaGetLastError();
}

cudaError_t make_diag(const double* V, double inv_h2, int64_t n, double* dg, cudaStream_t s) {
  make_diag_kernel<<<(unsigned)(ceil_div(n, 256) < 4096 ? ceil_div(n, 256) : 4096), 256, 0, s>>>(V, 6.0 * inv_h2, n,
                                                                                                  dg);
  count_launch();
  return cudaGetLastError();
}

cudaError_t check_finite(const double* v, int m, int* bad, cudaStream_t s) {
  if (m <= 0) return cudaSuccess;
  check_finite_kernel<<<(unsigned)ceil_div(m, 256), 256, 0, s>>>(v, m, bad);
  count_launch();
  return cudaGetLastError();
}

}  // namespace ppcg
