// Tall-skinny FP64 GEMMs of Algorithm 3 (the "GEMM" phase of Section 6).
//
//   gram     C = A^T B, A: n x ma, B: n x mb (n >> ma, mb). Split over n into chunks ("DGEMM on the local row
//            block followed by a global sum", Section 6): each CTA reduces a 64 x 64 tile of C over one chunk
//            into a partial, and a second kernel sums the partials in a fixed order (deterministic).
//            Used by steps 9-10 (X^T W, X^T P), 18 (X^T X), 20 (X^T AX) and 23 (S^T AS).
//   gemm_nn  Y (+)= A G with A: n x m, G: m x p small; epilogues for steps 9-10 (Y - X G, in place),
//            19 / 24 (X R^{-1}, S C) and 20 + 8 fused (W = T (AX - X M) with column norms of the residual).
//   small_gemm  C = op(A) B for the k x k products (steps 23-24, polar step 18), split over K.
//
// On GB300 FP64 runs at 2 DFMA lanes per clock per SM (measured 1.195 TFLOP/s for the whole GPU), so these
// GEMMs, with arithmetic intensity k/8 flop/byte, are FP64-pipe bound by a wide margin; the tiling only has to
// keep the FP64 pipe fed: 64 x 64 output tiles, 16-deep K slices staged in shared memory, 4 x 4 register
// micro-tiles per thread (16 DFMA per 2 vector shared loads).
#include "ppcg_internal.h"
#include "ppcg_steps.h"

#include <mutex>

namespace ppcg {

namespace {

constexpr int kT = 64;       // output tile
constexpr int kBK = 16;      // K slice
constexpr int kPad = 2;      // shared-memory row padding (keeps 16-byte alignment)
constexpr int kThreads = 256;

__device__ __forceinline__ void fma_tile(const double (*As)[kT + kPad], const double (*Bs)[kT + kPad], int ra,
                                         int cb, double acc[4][4]) {
#pragma unroll
  for (int kk = 0; kk < kBK; ++kk) {
    const double2 a01 = *reinterpret_cast<const double2*>(&As[kk][ra]);
    const double2 a23 = *reinterpret_cast<const double2*>(&As[kk][ra + 2]);
    const double2 b01 = *reinterpret_cast<const double2*>(&Bs[kk][cb]);
    const double2 b23 = *reinterpret_cast<const double2*>(&Bs[kk][cb + 2]);
    const double a[4] = {a01.x, a01.y, a23.x, a23.y};
    const double b[4] = {b01.x, b01.y, b23.x, b23.y};
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
  }
}

// part[split][i + j*ma] = sum over the split's rows of A[r, i] * B[r, j]
__global__ void __launch_bounds__(kThreads)
gram_tn_kernel(const double* __restrict__ A, int64_t lda, const double* __restrict__ B, int64_t ldb, int64_t n,
               int ma, int mb, int tiles_b, int64_t rows_per_split, double* __restrict__ part, int symmetric) {
  const int ti = blockIdx.x / tiles_b;
  const int tj = blockIdx.x % tiles_b;
  if (symmetric && ti > tj) return;
  const int i0 = ti * kT, j0 = tj * kT;
  const int64_t r_begin = (int64_t)blockIdx.y * rows_per_split;
  const int64_t r_end = min(n, r_begin + rows_per_split);
  __shared__ __align__(16) double As[kBK][kT + kPad];
  __shared__ __align__(16) double Bs[kBK][kT + kPad];
  const int t = threadIdx.x;
  const int tr = t % 16, tc = t / 16;        // micro-tile: C rows tr*4.., C cols tc*4..
  double acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
  const int lk = t % kBK;                     // loader: row within the slice
  const int lc = t / kBK;                     // loader: column (0..15) + 16 u
  for (int64_t r0 = r_begin; r0 < r_end; r0 += kBK) {
    const int64_t row = r0 + lk;
    const bool rok = row < r_end;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int cc = lc + 16 * u;
      As[lk][cc] = (rok && i0 + cc < ma) ? __ldg(A + row + (int64_t)(i0 + cc) * lda) : 0.0;
      Bs[lk][cc] = (rok && j0 + cc < mb) ? __ldg(B + row + (int64_t)(j0 + cc) * ldb) : 0.0;
    }
    __syncthreads();
    fma_tile(As, Bs, tr * 4, tc * 4, acc);
    __syncthreads();
  }
  double* out = part + (int64_t)blockIdx.y * ma * mb;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int gi = i0 + tr * 4 + i;
    if (gi >= ma) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int gj = j0 + tc * 4 + j;
      if (gj < mb) out[gi + (int64_t)gj * ma] = acc[i][j];
    }
  }
}

__global__ void gram_reduce_kernel(const double* __restrict__ part, int nsplit, int ma, int mb, double* __restrict__ C,
                                   int ldc, int symmetric) {
  const int64_t total = (int64_t)ma * mb;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    int i = (int)(e % ma), j = (int)(e / ma);
    int si = i, sj = j;
    if (symmetric && i > j) { si = j; sj = i; }   // only upper tiles were computed; mirror for exact symmetry
    const int64_t o = si + (int64_t)sj * ma;
    double s = 0.0;
    for (int p = 0; p < nsplit; ++p) s += part[(int64_t)p * total + o];
    C[i + (int64_t)j * ldc] = s;
  }
}

// Y tile rows r0.., cols c0..; thread micro-tile rows tr*4.., cols tc*4.. (tr fastest: coalesced stores)
__global__ void __launch_bounds__(kThreads)
gemm_nn_kernel(const double* __restrict__ A, int64_t lda, const double* __restrict__ G, int ldg, int64_t n, int m,
               int p, double* Y, int64_t ldy, const double* Yin, int64_t ldyin, int epi, int g_upper,
               ResidualArgs ra) {
  const int64_t r0 = (int64_t)blockIdx.x * kT;
  const int c0 = blockIdx.y * kT;
  __shared__ __align__(16) double As[kBK][kT + kPad];
  __shared__ __align__(16) double Gs[kBK][kT + kPad];
  const int t = threadIdx.x;
  const int tr = t % 16, tc = t / 16;
  double acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
  const int kend = g_upper ? min(m, c0 + kT) : m;
  const int la_r = t % kT, la_k = t / kT;     // A loader: 64 rows x 4 k, 4 passes
  const int lg_k = t % kBK, lg_c = t / kBK;   // G loader: 16 k x 16 cols, 4 passes
  for (int k0 = 0; k0 < kend; k0 += kBK) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int kk = la_k + 4 * u;
      const int64_t row = r0 + la_r;
      As[kk][la_r] = (row < n && k0 + kk < kend) ? __ldg(A + row + (int64_t)(k0 + kk) * lda) : 0.0;
      const int cc = lg_c + 16 * u;
      Gs[lg_k][cc] = (k0 + lg_k < kend && c0 + cc < p) ? __ldg(G + (k0 + lg_k) + (int64_t)(c0 + cc) * ldg) : 0.0;
    }
    __syncthreads();
    fma_tile(As, Gs, tr * 4, tc * 4, acc);
    __syncthreads();
  }
  // epilogue
  double colsq[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int64_t r = r0 + tr * 4 + i;
    if (r >= n) continue;
    double tinv = 0.0;
    if (epi == (int)Epi::Residual) tinv = ra.tinv ? ra.tinv[r] : 1.0 / fmax(ra.dg[r] - ra.sigma, ra.delta);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int c = c0 + tc * 4 + j;
      if (c >= p) continue;
      const int64_t o = r + (int64_t)c * ldy;
      if (epi == (int)Epi::Store) {
        Y[o] = acc[i][j];
      } else if (epi == (int)Epi::Sub) {
        Y[o] = Y[o] - acc[i][j];
      } else {
        const double rr = Yin[r + (int64_t)c * ldyin] - acc[i][j];
        colsq[j] += rr * rr;
        Y[o] = rr * tinv;
      }
    }
  }
  if (epi == (int)Epi::Residual) {
    __shared__ double red[16][kT];
#pragma unroll
    for (int j = 0; j < 4; ++j) red[tr][tc * 4 + j] = colsq[j];
    __syncthreads();
    if (t < kT) {
      double s = 0.0;
      for (int u = 0; u < 16; ++u) s += red[u][t];
      const int c = c0 + t;
      if (c < p) ra.norm_part[(int64_t)blockIdx.x * p + c] = s;
    }
  }
}

// part[split][i + j*m] = sum over the split's K range of op(A)[i, l] * B[l, j], op(A) = A^T (TRANS) or A.
// The k x k products of Algorithm 3 (steps 23-24 and the polar variant of step 18) have K = k only, too short
// for a 64 x 64 tile per CTA to fill the GPU; splitting K into 32-deep chunks gives 8x more CTAs at k = 256.
template <bool TRANS>
__global__ void __launch_bounds__(kThreads)
small_gemm_kernel(const double* __restrict__ A, int64_t lda, const double* __restrict__ B, int64_t ldb, int m,
                  int p, int kdim, int tiles_p, int k_per_split, double* __restrict__ part) {
  const int ti = blockIdx.x / tiles_p, tj = blockIdx.x % tiles_p;
  const int i0 = ti * kT, j0 = tj * kT;
  const int k_begin = blockIdx.y * k_per_split;
  const int k_end = min(kdim, k_begin + k_per_split);
  __shared__ __align__(16) double As[kBK][kT + kPad];
  __shared__ __align__(16) double Bs[kBK][kT + kPad];
  const int t = threadIdx.x;
  const int tr = t % 16, tc = t / 16;
  double acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
  for (int k0 = k_begin; k0 < k_end; k0 += kBK) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      if (TRANS) {                                   // A^T: K index runs down A's columns (coalesced in K)
        const int lk = t % kBK, cc = t / kBK + 16 * u;
        const int kk = k0 + lk;
        As[lk][cc] = (kk < k_end && i0 + cc < m) ? __ldg(A + kk + (int64_t)(i0 + cc) * lda) : 0.0;
      } else {                                       // A: rows i are contiguous
        const int cc = t % kT, lk = t / kT + 4 * u;
        const int kk = k0 + lk;
        As[lk][cc] = (kk < k_end && i0 + cc < m) ? __ldg(A + (i0 + cc) + (int64_t)kk * lda) : 0.0;
      }
      const int lk = t % kBK, cc = t / kBK + 16 * u;
      const int kk = k0 + lk;
      Bs[lk][cc] = (kk < k_end && j0 + cc < p) ? __ldg(B + kk + (int64_t)(j0 + cc) * ldb) : 0.0;
    }
    __syncthreads();
    fma_tile(As, Bs, tr * 4, tc * 4, acc);
    __syncthreads();
  }
  double* out = part + (int64_t)blockIdx.y * m * p;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int gi = i0 + tr * 4 + i;
    if (gi >= m) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int gj = j0 + tc * 4 + j;
      if (gj < p) out[gi + (int64_t)gj * m] = acc[i][j];
    }
  }
}

int grid_sm_count() {
  static const int sms = [] {               // initialised once, thread-safe (concurrent batched solves)
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    return v > 0 ? v : 1;
  }();
  return sms;
}

}  // namespace

int gram_splits(int64_t n, int ma, int mb, size_t part_capacity) {
  const int64_t tiles = ceil_div(ma, kT) * ceil_div(mb, kT);
  const int64_t want = ceil_div(4LL * grid_sm_count(), tiles);
  int64_t maxs = ceil_div(n, 256);                 // at least 256 rows per chunk
  const int64_t cap = (int64_t)(part_capacity / ((size_t)ma * mb));
  int64_t sp = want;
  if (sp > maxs) sp = maxs;
  if (sp > cap) sp = cap;
  if (sp > 65535) sp = 65535;
  if (sp < 1) sp = 1;
  return (int)sp;
}

cudaError_t gram(const double* A, int64_t lda, const double* B, int64_t ldb, int64_t n, int ma, int mb, double* C,
                 int ldc, bool symmetric, double* part, size_t part_capacity, cudaStream_t s) {
  if (ma <= 0 || mb <= 0) return cudaSuccess;
  if ((size_t)ma * mb > part_capacity) return cudaErrorInvalidValue;
  const int nsplit = gram_splits(n, ma, mb, part_capacity);
  int64_t rows = ceil_div(n, nsplit);
  rows = ceil_div(rows, kBK) * kBK;
  const int nsp = (int)ceil_div(n, rows);
  const int tiles_a = (int)ceil_div(ma, kT), tiles_b = (int)ceil_div(mb, kT);
  dim3 grid(tiles_a * tiles_b, nsp);
  gram_tn_kernel<<<grid, kThreads, 0, s>>>(A, lda, B, ldb, n, ma, mb, tiles_b, rows, part, symmetric ? 1 : 0);
  count_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int64_t total = (int64_t)ma * mb;
  const int64_t blocks = ceil_div(total, 256);
  gram_reduce_kernel<<<(unsigned)(blocks < 8192 ? blocks : 8192), 256, 0, s>>>(part, nsp, ma, mb, C, ldc,
                                                                                symmetric ? 1 : 0);
  count_launch();
  return cudaGetLastError();
}

cudaError_t gram_reduce_partials(const double* part, int nsplit, int ma, int mb, double* C, int ldc, bool symmetric,
                                 cudaStream_t s) {
  const int64_t total = (int64_t)ma * mb;
  const int64_t blocks = ceil_div(total, 256);
  gram_reduce_kernel<<<(unsigned)(blocks < 8192 ? blocks : 8192), 256, 0, s>>>(part, nsplit, ma, mb, C, ldc,
                                                                                symmetric ? 1 : 0);
  count_launch();
  return cudaGetLastError();
}

cudaError_t small_gemm(bool trans_a, const double* A, int64_t lda, const double* B, int64_t ldb, int m, int p,
                       int kdim, double* C, int ldc, double* part, size_t part_capacity, cudaStream_t s) {
  if (m <= 0 || p <= 0) return cudaSuccess;
  if (kdim <= 0 || (size_t)m * p > part_capacity) return cudaErrorInvalidValue;
  int nsplit = (int)ceil_div(kdim, 32);
  const int64_t cap = (int64_t)(part_capacity / ((size_t)m * p));
  if (nsplit > cap) nsplit = (int)cap;
  int kps = (int)ceil_div(kdim, nsplit);
  kps = (int)ceil_div(kps, kBK) * kBK;
  nsplit = (int)ceil_div(kdim, kps);
  const int tiles_m = (int)ceil_div(m, kT), tiles_p = (int)ceil_div(p, kT);
  dim3 grid(tiles_m * tiles_p, nsplit);
  if (trans_a)
    small_gemm_kernel<true><<<grid, kThreads, 0, s>>>(A, lda, B, ldb, m, p, kdim, tiles_p, kps, part);
  else
    small_gemm_kernel<false><<<grid, kThreads, 0, s>>>(A, lda, B, ldb, m, p, kdim, tiles_p, kps, part);
  count_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return gram_reduce_partials(part, nsplit, m, p, C, ldc, false, s);
}

cudaError_t kxk_gemm(const KxK& g, bool trans_a, const double* A, int64_t lda, const double* B, int64_t ldb, int m,
                     int p, int kdim, double* C, int ldc, cudaStream_t s) {
  if (m <= 0 || p <= 0) return cudaSuccess;
  // the emulation needs a 128 x 64 output tile grid and a reduction long enough to amortise its exponent and
  // slicing passes; smaller products stay on the FP64 pipe
  const bool tc = g.ozaki && m >= 128 && p >= 128 && kdim >= 128;
  if (!tc) return small_gemm(trans_a, A, lda, B, ldb, m, p, kdim, C, ldc, g.part, g.part_cap, s);
  if (trans_a) {
    const bool sym = (A == B && lda == ldb && m == p);
    return oz_gram(A, lda, B, ldb, kdim, m, p, C, ldc, sym, g.part, g.part_cap, g.exps, g.img, g.img_bytes, g.flag,
                   s);
  }
  return oz_update(A, lda, B, (int)ldb, m, kdim, p, C, ldc, Epi::Store, g.exps, g.img, g.img_bytes, g.flag, s);
}

cudaError_t gemm_nn(const double* A, int64_t lda, const double* G, int ldg, int64_t n, int m, int p, double* Y,
                    int64_t ldy, const double* Yin, int64_t ldyin, Epi epi, bool g_upper, const ResidualArgs* ra,
                    cudaStream_t s) {
  if (p <= 0 || n <= 0) return cudaSuccess;
  ResidualArgs args{};
  if (ra) args = *ra;
  dim3 grid((unsigned)ceil_div(n, kT), (unsigned)ceil_div(p, kT));
  gemm_nn_kernel<<<grid, kThreads, 0, s>>>(A, lda, G, ldg, n, m, p, Y, ldy, Yin, ldyin, (int)epi, g_upper ? 1 : 0,
                                           args);
  count_launch();
  return cudaGetLastError();
}

}  // namespace ppcg

// ------------------------------------------------------------------------------------------ allocation-free Gram
// ppcg_gram_noalloc serves callers that cannot allocate device memory at all: code that runs under a fixed,
// pre-reserved memory budget or inside an application's own memory pool that forbids cudaMalloc (whose implicit
// synchronisation such callers also cannot afford), and callers that have no ppcg handle (creating one allocates a
// workspace). Its split-K partial sums live in the file-scope array below instead of a caller-provided or
// library-allocated workspace. Every GPU that loads this library holds the array until the process exits.
namespace {
constexpr size_t kNoAllocScratchDoubles = size_t(1) << 20;   // 8 MiB: ma * mb must not exceed 1,048,576
constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
double* g_noalloc_addr[kMaxDevices] = {};
}  // namespace

static __device__ __align__(256) double g_gram_scratch[kNoAllocScratchDoubles];

extern "C" ppcg_status ppcg_gram_noalloc(const double* A, int64_t lda, const double* B, int64_t ldb, int64_t n,
                                         int32_t ma, int32_t mb, double* C, void* cuda_stream) {
  if (!A || !B || !C || n < 1 || ma < 1 || mb < 1 || lda < n || ldb < n) return PPCG_ERR_ARG;
  if ((size_t)ma * (size_t)mb > kNoAllocScratchDoubles) return PPCG_ERR_ARG;   // beyond the static scratch
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return PPCG_ERR_CUDA;
  double* scratch = nullptr;
  {
    // Set-up, once per device, with that device current: the array's name is only a host-side stand-in, so
    // the device address must come from the runtime.
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_gram_scratch) != cudaSuccess || !p) return PPCG_ERR_CUDA;
      g_noalloc_addr[dev] = static_cast<double*>(p);
    }
    scratch = g_noalloc_addr[dev];
  }
  const bool sym = (A == B && lda == ldb && ma == mb);
  if (ppcg::gram(A, lda, B, ldb, n, ma, mb, C, ma, sym, scratch, kNoAllocScratchDoubles,
                 static_cast<cudaStream_t>(cuda_stream)) != cudaSuccess)
    return PPCG_ERR_CUDA;
  return PPCG_OK;
}

