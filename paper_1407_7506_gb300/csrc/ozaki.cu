// FP64-accurate tall-skinny GEMMs on the BF16 tensor cores by error-free splitting (the Ozaki scheme: Ozaki,
// Ogita, Oishi, Rump, "Error-free transformations of matrix multiplication by using fast routines of matrix
// multiplication and its applications", Numer. Algorithms 2012), written for tcgen05.
//
// Every FP64 element x of a column (Gram) or row (update) whose magnitudes are below 2^E is rounded to the
// integer T = round(x 2^(54 - E)) and written as 8 balanced base-128 digits d_j in [-63, 64]:
//   x = sum_{j<8} d_j 2^(E - 5 - 7 j)  (to 2^-55 relative to the column maximum).
// A digit is exact in BF16 and a digit product is at most 2^12, so the 36 digit-pair products with
// j + l = g (g = 0..7) can share one FP32 TMEM accumulator: over a chunk of 512 summed terms each group stays an
// integer of magnitude at most 8 * 512 * 2^12 = 2^24, every partial sum is an integer that FP32 represents exactly,
// and the tensor-core accumulation is exact. After every chunk the 8 group accumulators are
// folded, with weights 2^(-7 g), into a double-float (FP32 pair) register accumulator; one FP64 scale by
// 2^(E_a + E_b - 10) per element produces the result. The error is that of the 55-bit digits plus the ~2^-48
// relative rounding of the double-float sum, below the rounding of an FP64 GEMM of these lengths.
//
// Two forms. The register-staged kernels (narrow products, where a slice would not be re-used) take tiles of
// M = 128 rows (TMEM lanes) x N = 64 columns, whose 8 group accumulators fill the 512 TMEM columns of an SM; their
// operand tiles are staged by the threads (coalesced FP64 loads, integer digit extraction, BF16 stores into the
// K-major canonical layout, 8 digit planes per operand, 2 stages) and one thread issues the 72 MMAs of a stage.
// The image-fed product (wide operands, below) slices each operand once into digit images and runs 128 x 128
// tiles in two passes of four group accumulators, fed by bulk copies.
#include "ppcg_internal.h"
#include "tc_util.cuh"

#include <cuda_bf16.h>

#include <algorithm>

namespace ppcg {

cudaError_t gram_reduce_partials(const double* part, int nsplit, int ma, int mb, double* C, int ldc, bool symmetric,
                                 cudaStream_t s);

namespace {

using namespace tc;

constexpr int kM = 128;
constexpr int kN = 64;
constexpr int kDig = 8;                   // digits per element
constexpr int kGroups = 8;                // g = j + l <= 7
constexpr int kBK = 32;                   // K per stage (2 MMAs of K = 16)
constexpr int kChunk = 512;               // exact-accumulation chunk (8 * 512 * 2^12 = 2^24: FP32-exact integers)
constexpr int kThreads = 256;
constexpr uint32_t kLBO = 128;            // bytes between core matrices along K (8 bf16)
constexpr uint32_t kSBO = (kBK / 8) * 128;  // bytes between 8-row groups
constexpr uint32_t kAPlane = (kM / 8) * kSBO;   // 8 KB
constexpr uint32_t kBPlane = (kN / 8) * kSBO;   // 4 KB
constexpr uint32_t kStageBytes = kDig * (kAPlane + kBPlane);   // 96 KB
constexpr int kNoExp = -2000;             // exponent of an all-zero line

__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ uint32_t tile_off(int row, int k) {
  return (uint32_t)(row >> 3) * kSBO + (uint32_t)(row & 7) * 16u + (uint32_t)(k >> 3) * kLBO + (uint32_t)(k & 7) * 2u;
}

// Balanced base-128 digits of T = round(x 2^(54 - E)) (|T| <= 2^54), through one biased integer: adding
// kBias = 63 (1 + 128 + ... + 128^7) makes T' = T + kBias lie in (0, 2^56), and the eight plain 7-bit fields u_f of
// T' give the balanced digits u_f - 63 in [-63, 64] (the representation is unique, so these are the digits of T).
// Digit j (j = 0 most significant) is field 7 - j. A field becomes an exact float by the 2^23 bit-pattern trick.
constexpr long long kBias = 35745105703854015LL;   // 63 * (2^56 - 1) / 127

__device__ __forceinline__ unsigned long long biased_digits(double x, int E) {
  const long long bits = __double_as_longlong(x);
  const int ex = (int)((bits >> 52) & 0x7FF);
  long long T = 0;
  if (ex != 0 && E > kNoExp) {
    const long long m = (bits & 0xFFFFFFFFFFFFFLL) | (1LL << 52);
    const int sh = ex - 1021 - E;                 // x = m 2^(ex - 1075); T = m 2^(ex - 1075 + 54 - E)
    if (sh >= 0) T = m << (sh < 2 ? sh : 2);      // |x| < 2^E gives sh <= 1
    else if (sh > -63) T = (m + (1LL << (-sh - 1))) >> (-sh);
    if (bits < 0) T = -T;
  }
  return (unsigned long long)(T + kBias);
}

__device__ __forceinline__ float digit_of(unsigned long long t, int j) {
  const uint32_t u = (uint32_t)(t >> (7 * (kDig - 1 - j))) & 127u;
  return __uint_as_float(0x4B000000u | u) - 8388671.0f;          // (2^23 + u) - (2^23 + 63), exact
}

// digit j of two elements as a packed BF16 pair (exact: |digit| <= 64)
__device__ __forceinline__ uint32_t digit_pair(unsigned long long t0, unsigned long long t1, int j) {
  __nv_bfloat162 v = __floats2bfloat162_rn(digit_of(t0, j), digit_of(t1, j));
  return *reinterpret_cast<uint32_t*>(&v);
}

__device__ __forceinline__ double pow2(int e) {   // 2^e for e in the normal range
  e = e < -1022 ? -1022 : (e > 1023 ? 1023 : e);
  return __longlong_as_double((long long)(e + 1023) << 52);
}

// ------------------------------------------------------------------------------------------ exponent bounds
// E[c] = smallest e with max_r |M[r, c]| < 2^e (kNoExp for a zero line). Each block reduces a slice of lines and
// merges its bound with atomicMax (the bound is monotone in the maximum), so a column of n rows is read by many
// CTAs at once; E must hold kNoExp beforehand (fill_exp_kernel). NaN entries are ignored.
__device__ __forceinline__ int exp_bound(double mx) {
  const long long b = __double_as_longlong(mx);
  const int ex = (int)((b >> 52) & 0x7FF);
  return (mx == 0.0 || ex == 0) ? kNoExp : ex - 1022;     // mx in [2^(ex-1023), 2^(ex-1022))
}

__global__ void fill_exp_kernel(int* E, int count) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) E[i] = kNoExp;
}

constexpr int kExpRows = 4096;    // rows per block of the column bound

// grid (cols, ceil(rows / kExpRows)); 256 threads stride over the block's rows of column blockIdx.x
__global__ void __launch_bounds__(256)
col_exp_kernel(const double* __restrict__ M, int64_t ld, int64_t rows, int* __restrict__ E) {
  const int col = blockIdx.x;
  const int64_t r0 = (int64_t)blockIdx.y * kExpRows;
  const int64_t r1 = min(rows, r0 + kExpRows);
  const double* c = M + (int64_t)col * ld;
  double mx = 0.0;
  for (int64_t r = r0 + threadIdx.x; r < r1; r += blockDim.x) mx = fmax(mx, fabs(__ldg(c + r)));
  for (int off = 16; off > 0; off >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, off));
  __shared__ double red[8];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x / 32] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x / 32); ++w) mx = fmax(mx, red[w]);
    const int e = exp_bound(mx);
    if (e != kNoExp) atomicMax(E + col, e);
  }
}

constexpr int kExpCols = 32;      // columns per block of the row bound

// E[r] = smallest e with max_c |M[r, c]| < 2^e; grid (ceil(rows / 256), ceil(cols / kExpCols)), one thread per row
__global__ void row_exp_kernel(const double* __restrict__ M, int64_t ld, int64_t rows, int cols, int* __restrict__ E) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= rows) return;
  const int c0 = blockIdx.y * kExpCols;
  const int c1 = min(cols, c0 + kExpCols);
  double mx = 0.0;
  for (int c = c0; c < c1; ++c) mx = fmax(mx, fabs(__ldg(M + r + (int64_t)c * ld)));
  const int e = exp_bound(mx);
  if (e != kNoExp) atomicMax(E + r, e);
}

cudaError_t col_exps(const double* M, int64_t ld, int64_t rows, int cols, int* E, cudaStream_t s) {
  fill_exp_kernel<<<(unsigned)ceil_div(cols, 256), 256, 0, s>>>(E, cols);
  col_exp_kernel<<<dim3((unsigned)cols, (unsigned)ceil_div(rows, kExpRows)), 256, 0, s>>>(M, ld, rows, E);
  count_launch(2);
  return cudaGetLastError();
}

cudaError_t row_exps(const double* M, int64_t ld, int64_t rows, int cols, int* E, cudaStream_t s) {
  const int64_t b = ceil_div(rows, 256);
  fill_exp_kernel<<<(unsigned)(b < 4096 ? b : 4096), 256, 0, s>>>(E, (int)rows);
  row_exp_kernel<<<dim3((unsigned)b, (unsigned)ceil_div(cols, kExpCols)), 256, 0, s>>>(M, ld, rows, cols, E);
  count_launch(2);
  return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------ shared machinery
struct OzSmem {
  uint64_t mbar[2];
  uint32_t tmem_slot;
  int ok;
  int Ea[kM];
  int Eb[kN];
};

__device__ void oz_setup(OzSmem& sm) {
  if (threadIdx.x == 0) {
    mbar_init(smem_u32(&sm.mbar[0]), 1);
    mbar_init(smem_u32(&sm.mbar[1]), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncwarp();
  if (threadIdx.x / 32 == 0) tmem_alloc(smem_u32(&sm.tmem_slot), 512);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
}

__device__ void oz_teardown(OzSmem& sm, uint32_t tmem, bool ok, int gstage, int* flag) {
  if (!ok && threadIdx.x == 0) {
    atomicOr(flag, kFlagTimeout);
    if (gstage > 0) mbar_wait(smem_u32(&sm.mbar[(gstage - 1) & 1]), (uint32_t)(((gstage - 1) >> 1) & 1));
  }
  tc_fence_before();
  __syncthreads();
  if (threadIdx.x / 32 == 0) {
    __syncwarp();
    tc_fence_after();
    tmem_dealloc(tmem, 512);
  }
}

// the 72 MMAs of one stage: for g = j + l, both K halves of the stage
__device__ __forceinline__ void issue_stage(uint32_t tmem, uint8_t* stage, bool first_stage_of_chunk) {
  const uint32_t a0 = smem_u32(stage), b0 = a0 + kDig * kAPlane;
  constexpr uint32_t idesc = idesc_bf16(kM, kN);
#pragma unroll
  for (int g = 0; g < kGroups; ++g) {
#pragma unroll
    for (int j = 0; j <= g; ++j) {
      const int l = g - j;
#pragma unroll
      for (int ks = 0; ks < kBK / 16; ++ks) {
        const uint32_t acc = (first_stage_of_chunk && j == 0 && ks == 0) ? 0u : 1u;
        mma_bf16(tmem + (uint32_t)(g * kN), smem_desc_nosw(a0 + j * kAPlane + ks * 2 * kLBO, kLBO, kSBO),
                 smem_desc_nosw(b0 + l * kBPlane + ks * 2 * kLBO, kLBO, kSBO), idesc, acc);
      }
    }
  }
}

// fold the 8 group accumulators of this warp's 32 lanes x 32 columns into (hi, lo)
__device__ __forceinline__ void fold_groups(uint32_t tmem, int q, int h, float (&hi)[32], float (&lo)[32]) {
#pragma unroll 1
  for (int g = kGroups - 1; g >= 0; --g) {
    float v[32];
    tmem_ld32(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(g * kN + 32 * h), v);
    const float w = __int_as_float((127 - 7 * g) << 23);   // 2^(-7 g), exact
#pragma unroll
    for (int i = 0; i < 32; ++i) {
      const float x = v[i] * w;
      const float s = hi[i] + x;
      const float bb = s - hi[i];
      lo[i] += (hi[i] - (s - bb)) + (x - bb);
      hi[i] = s;
    }
  }
}

// per-thread staging registers: A core matrices (8 rows x 8 k, 2 elements per lane) and B core matrices
constexpr int kACm = (kM / 8) * (kBK / 8) / (kThreads / 32);   // 8
constexpr int kBCm = (kN / 8) * (kBK / 8) / (kThreads / 32);   // 4
struct Regs {
  double a[kACm][2];
  double b[kBCm][2];
};

// ------------------------------------------------------------------------------------------ C = A^T B partials
// grid (tiles_m * tiles_n, nsplit); A: n x ma, B: n x mb; Ea/Eb column exponent bounds over all n rows
__global__ void __launch_bounds__(kThreads, 1)
oz_gram_kernel(const double* __restrict__ A, int64_t lda, const double* __restrict__ B, int64_t ldb, int64_t n,
               int ma, int mb, int tiles_n, int64_t rows_per_split, const int* __restrict__ Ea,
               const int* __restrict__ Eb, double* __restrict__ part, int symmetric, int* flag) {
  extern __shared__ __align__(1024) uint8_t dyn[];
  __shared__ OzSmem sm;
  const int tm = blockIdx.x / tiles_n, tn = blockIdx.x % tiles_n;
  const int m0 = tm * kM, n0 = tn * kN;
  if (symmetric && n0 + kN <= m0) return;        // entirely below the diagonal: the reduce reads only i <= j
  const int64_t r_begin = (int64_t)blockIdx.y * rows_per_split;
  const int64_t r_end = min(n, r_begin + rows_per_split);
  for (int i = threadIdx.x; i < kM; i += kThreads) sm.Ea[i] = (m0 + i < ma) ? Ea[m0 + i] : kNoExp;
  for (int i = threadIdx.x; i < kN; i += kThreads) sm.Eb[i] = (n0 + i < mb) ? Eb[n0 + i] : kNoExp;
  oz_setup(sm);
  const uint32_t tmem = sm.tmem_slot;
  const int warp = threadIdx.x / 32, lane = threadIdx.x & 31;
  const int rr = lane >> 2, kp = lane & 3;       // inside a core matrix: row rr, k = 2 kp, 2 kp + 1
  const int q = warp & 3, h = warp >> 2;
  float hi[32], lo[32];
#pragma unroll
  for (int i = 0; i < 32; ++i) { hi[i] = 0.f; lo[i] = 0.f; }
  Regs reg;
  auto load = [&](int64_t k0, int64_t kend) {
#pragma unroll
    for (int i = 0; i < kACm; ++i) {
      const int cm = warp + i * (kThreads / 32);
      const int g8 = cm / (kBK / 8), c8 = cm % (kBK / 8);
      const int col = m0 + 8 * g8 + rr;
      const int64_t r = k0 + 8 * c8 + 2 * kp;
      const double* p = A + r + (int64_t)col * lda;
      reg.a[i][0] = (col < ma && r < kend) ? __ldg(p) : 0.0;
      reg.a[i][1] = (col < ma && r + 1 < kend) ? __ldg(p + 1) : 0.0;
    }
#pragma unroll
    for (int i = 0; i < kBCm; ++i) {
      const int cm = warp + i * (kThreads / 32);
      const int g8 = cm / (kBK / 8), c8 = cm % (kBK / 8);
      const int col = n0 + 8 * g8 + rr;
      const int64_t r = k0 + 8 * c8 + 2 * kp;
      const double* p = B + r + (int64_t)col * ldb;
      reg.b[i][0] = (col < mb && r < kend) ? __ldg(p) : 0.0;
      reg.b[i][1] = (col < mb && r + 1 < kend) ? __ldg(p + 1) : 0.0;
    }
  };
  auto store = [&](uint8_t* stage) {
#pragma unroll
    for (int i = 0; i < kACm; ++i) {
      const int cm = warp + i * (kThreads / 32);
      const int g8 = cm / (kBK / 8), c8 = cm % (kBK / 8);
      const int E = sm.Ea[8 * g8 + rr];
      const unsigned long long t0 = biased_digits(reg.a[i][0], E), t1 = biased_digits(reg.a[i][1], E);
      const uint32_t off = tile_off(8 * g8 + rr, 8 * c8 + 2 * kp);
#pragma unroll
      for (int j = 0; j < kDig; ++j)
        *reinterpret_cast<uint32_t*>(stage + j * kAPlane + off) = digit_pair(t0, t1, j);
    }
    uint8_t* bst = stage + kDig * kAPlane;
#pragma unroll
    for (int i = 0; i < kBCm; ++i) {
      const int cm = warp + i * (kThreads / 32);
      const int g8 = cm / (kBK / 8), c8 = cm % (kBK / 8);
      const int E = sm.Eb[8 * g8 + rr];
      const unsigned long long t0 = biased_digits(reg.b[i][0], E), t1 = biased_digits(reg.b[i][1], E);
      const uint32_t off = tile_off(8 * g8 + rr, 8 * c8 + 2 * kp);
#pragma unroll
      for (int j = 0; j < kDig; ++j)
        *reinterpret_cast<uint32_t*>(bst + j * kBPlane + off) = digit_pair(t0, t1, j);
    }
  };
  int gstage = 0;
  bool ok = true;
  for (int64_t c0 = r_begin; c0 < r_end && ok; c0 += kChunk) {
    const int64_t cend = min(r_end, c0 + kChunk);
    const int nk = (int)ceil_div(cend - c0, kBK);
    load(c0, cend);
    for (int kb = 0; kb < nk; ++kb, ++gstage) {
      const int s = gstage & 1;
      uint8_t* stage = dyn + s * kStageBytes;
      if (gstage >= 2) {
        if (threadIdx.x == 0) sm.ok = mbar_wait(smem_u32(&sm.mbar[s]), (uint32_t)(((gstage - 2) >> 1) & 1)) ? 1 : 0;
        __syncthreads();
        if (!sm.ok) { ok = false; break; }
      }
      store(stage);
      if (kb + 1 < nk) load(c0 + (int64_t)(kb + 1) * kBK, cend);
      fence_async_smem();
      __syncthreads();
      if (threadIdx.x == 0) {
        tc_fence_after();
        issue_stage(tmem, stage, kb == 0);
        mma_commit(smem_u32(&sm.mbar[s]));
      }
    }
    if (!ok) break;
    if (threadIdx.x == 0) sm.ok = mbar_wait(smem_u32(&sm.mbar[(gstage - 1) & 1]), (uint32_t)(((gstage - 1) >> 1) & 1)) ? 1 : 0;
    __syncthreads();
    if (!sm.ok) { ok = false; break; }
    tc_fence_after();
    fold_groups(tmem, q, h, hi, lo);
    tc_fence_before();
    __syncthreads();
  }
  if (ok) {
    double* out = part + (int64_t)blockIdx.y * ma * mb;
    const int ri = 32 * q + lane;
    const int gi = m0 + ri;
    if (gi < ma) {
      const int Ei = sm.Ea[ri];
#pragma unroll
      for (int i = 0; i < 32; ++i) {
        const int cj = 32 * h + i;
        const int gj = n0 + cj;
        if (gj >= mb) continue;
        const int Ej = sm.Eb[cj];
        const double v = (Ei == kNoExp || Ej == kNoExp) ? 0.0 : (widen(hi[i]) + widen(lo[i])) * pow2(Ei + Ej - 10);
        out[gi + (int64_t)gj * ma] = v;
      }
    }
  }
  oz_teardown(sm, tmem, ok, gstage, flag);
}

// ------------------------------------------------------------------------------------------ Y = Y -/+ A G
// grid (ceil(n / 128), ceil(p / 64)); A: n x m, G: m x p; Er: row exponents of A, Fc: column exponents of G
__global__ void __launch_bounds__(kThreads, 1)
oz_update_kernel(const double* __restrict__ A, int64_t lda, const double* __restrict__ G, int ldg, int64_t n, int m,
                 int p, double* Y, int64_t ldy, int mode, const int* __restrict__ Er, const int* __restrict__ Fc,
                 int* flag) {
  extern __shared__ __align__(1024) uint8_t dyn[];
  __shared__ OzSmem sm;
  const int64_t r0 = (int64_t)blockIdx.x * kM;
  const int c0 = blockIdx.y * kN;
  for (int i = threadIdx.x; i < kM; i += kThreads) sm.Ea[i] = (r0 + i < n) ? Er[r0 + i] : kNoExp;
  for (int i = threadIdx.x; i < kN; i += kThreads) sm.Eb[i] = (c0 + i < p) ? Fc[c0 + i] : kNoExp;
  oz_setup(sm);
  const uint32_t tmem = sm.tmem_slot;
  const int warp = threadIdx.x / 32, lane = threadIdx.x & 31;
  const int rr = lane >> 2, kp = lane & 3;
  const int q = warp & 3, h = warp >> 2;
  float hi[32], lo[32];
#pragma unroll
  for (int i = 0; i < 32; ++i) { hi[i] = 0.f; lo[i] = 0.f; }
  Regs reg;
  // A tile: rows of A x k (columns of A); B tile: columns of G x k (rows of G)
  auto load = [&](int k0, int kend) {
#pragma unroll
    for (int i = 0; i < kACm; ++i) {
      const int cm = warp + i * (kThreads / 32);
      const int g8 = cm / (kBK / 8), c8 = cm % (kBK / 8);
      const int64_t row = r0 + 8 * g8 + rr;
      const int k = k0 + 8 * c8 + 2 * kp;
      reg.a[i][0] = (row < n && k < kend) ? __ldg(A + row + (int64_t)k * lda) : 0.0;
      reg.a[i][1] = (row < n && k + 1 < kend) ? __ldg(A + row + (int64_t)(k + 1) * lda) : 0.0;
    }
#pragma unroll
    for (int i = 0; i < kBCm; ++i) {
      const int cm = warp + i * (kThreads / 32);
      const int g8 = cm / (kBK / 8), c8 = cm % (kBK / 8);
      const int col = c0 + 8 * g8 + rr;
      const int k = k0 + 8 * c8 + 2 * kp;
      const double* pp = G + k + (int64_t)col * ldg;
      reg.b[i][0] = (col < p && k < kend) ? __ldg(pp) : 0.0;
      reg.b[i][1] = (col < p && k + 1 < kend) ? __ldg(pp + 1) : 0.0;
    }
  };
  auto store = [&](uint8_t* stage) {
#pragma unroll
    for (int i = 0; i < kACm; ++i) {
      const int cm = warp + i * (kThreads / 32);
      const int g8 = cm / (kBK / 8), c8 = cm % (kBK / 8);
      const int E = sm.Ea[8 * g8 + rr];
      const unsigned long long t0 = biased_digits(reg.a[i][0], E), t1 = biased_digits(reg.a[i][1], E);
      const uint32_t off = tile_off(8 * g8 + rr, 8 * c8 + 2 * kp);
#pragma unroll
      for (int j = 0; j < kDig; ++j)
        *reinterpret_cast<uint32_t*>(stage + j * kAPlane + off) = digit_pair(t0, t1, j);
    }
    uint8_t* bst = stage + kDig * kAPlane;
#pragma unroll
    for (int i = 0; i < kBCm; ++i) {
      const int cm = warp + i * (kThreads / 32);
      const int g8 = cm / (kBK / 8), c8 = cm % (kBK / 8);
      const int E = sm.Eb[8 * g8 + rr];
      const unsigned long long t0 = biased_digits(reg.b[i][0], E), t1 = biased_digits(reg.b[i][1], E);
      const uint32_t off = tile_off(8 * g8 + rr, 8 * c8 + 2 * kp);
#pragma unroll
      for (int j = 0; j < kDig; ++j)
        *reinterpret_cast<uint32_t*>(bst + j * kBPlane + off) = digit_pair(t0, t1, j);
    }
  };
  int gstage = 0;
  bool ok = true;
  for (int k0 = 0; k0 < m && ok; k0 += kChunk) {
    const int kend = min(m, k0 + kChunk);
    const int nk = (int)ceil_div(kend - k0, kBK);
    load(k0, kend);
    for (int kb = 0; kb < nk; ++kb, ++gstage) {
      const int s = gstage & 1;
      uint8_t* stage = dyn + s * kStageBytes;
      if (gstage >= 2) {
        if (threadIdx.x == 0) sm.ok = mbar_wait(smem_u32(&sm.mbar[s]), (uint32_t)(((gstage - 2) >> 1) & 1)) ? 1 : 0;
        __syncthreads();
        if (!sm.ok) { ok = false; break; }
      }
      store(stage);
      if (kb + 1 < nk) load(k0 + (kb + 1) * kBK, kend);
      fence_async_smem();
      __syncthreads();
      if (threadIdx.x == 0) {
        tc_fence_after();
        issue_stage(tmem, stage, kb == 0);
        mma_commit(smem_u32(&sm.mbar[s]));
      }
    }
    if (!ok) break;
    if (threadIdx.x == 0) sm.ok = mbar_wait(smem_u32(&sm.mbar[(gstage - 1) & 1]), (uint32_t)(((gstage - 1) >> 1) & 1)) ? 1 : 0;
    __syncthreads();
    if (!sm.ok) { ok = false; break; }
    tc_fence_after();
    fold_groups(tmem, q, h, hi, lo);
    tc_fence_before();
    __syncthreads();
  }
  if (ok) {
    const int ri = 32 * q + lane;
    const int64_t gr = r0 + ri;
    if (gr < n) {
      const int Ei = sm.Ea[ri];
      double yv[32];
#pragma unroll
      for (int i = 0; i < 32; ++i) {
        const int gc = c0 + 32 * h + i;
        yv[i] = (mode != (int)Epi::Store && gc < p) ? Y[gr + (int64_t)gc * ldy] : 0.0;
      }
#pragma unroll
      for (int i = 0; i < 32; ++i) {
        const int cj = 32 * h + i;
        const int gc = c0 + cj;
        if (gc >= p) continue;
        const int Ej = sm.Eb[cj];
        const double v = (Ei == kNoExp || Ej == kNoExp) ? 0.0 : (widen(hi[i]) + widen(lo[i])) * pow2(Ei + Ej - 10);
        Y[gr + (int64_t)gc * ldy] = mode == (int)Epi::Store ? v : yv[i] - v;
      }
    }
  }
  oz_teardown(sm, tmem, ok, gstage, flag);
}

// ------------------------------------------------------------------------------------------ pre-sliced Grams
// The Gram's operands are sliced once, by a streaming kernel, into "digit images": for every 128-column tile t and
// every 16-row block b of the operand, 8 planes (one per digit), each the exact shared-memory image of a 128-row x
// 16-K operand tile in the canonical K-major layout (core matrices of 8 rows x 16 bytes; 128 B between core matrices
// along K, 256 B between 8-row groups). The 8 planes of a (t, b) pair are contiguous, so one bulk asynchronous copy
// (cp.async.bulk) per operand and stage moves them into shared memory through an mbarrier ring: no digit arithmetic
// sits in the product's main loop and every operand element is sliced once instead of once per output tile.
//
// Output tiles are 128 x 128. The 8 group accumulators of a 128 x 128 tile would need 1024 TMEM columns, so the
// product runs every exact-accumulation chunk twice: pass 0 accumulates groups g = 0..3 (digit planes 0..3 of
// both operands), pass 1 groups g = 4..7 (all planes), each in 4 accumulators of 128 columns (all 512 TMEM
// columns), and each pass is folded at the chunk's end. Against 128 x 64 tiles with all 8 groups resident, every
// MMA is twice as wide, so the tensor cores read half as many operand bytes from shared memory per product.
// A buffer holds one pass-1 stage (all 8 planes of both operands, 26 MMAs) or two pass-0 stages (planes 0..3, 20
// MMAs), so that every wait on a buffer is followed by at least 20 MMAs.
constexpr int kSK = 16;                                   // K per stage
constexpr uint32_t kSSBO = (kSK / 8) * 128;              // 256 B between 8-row groups
constexpr uint32_t kSAPlane = (128 / 8) * kSSBO;         // 4 KB: one 128-row plane
constexpr uint32_t kImgBlk = kDig * kSAPlane;            // 32 KB: the 8 planes of one (tile, 16-row block)
constexpr uint32_t kHalf = kImgBlk / 2;                  // 16 KB: planes 0..3 of one (tile, 16-row block)
constexpr uint32_t kStage2 = 2 * kImgBlk;                // 64 KB: both operands, all planes
constexpr int kSBuf = 3;
constexpr int kN2 = 128;                                 // output columns per tile of the image-fed product
constexpr int kSChunkBlocks = kChunk / kSK;             // 32 stages per exact-accumulation chunk

__device__ __forceinline__ uint32_t tile_off16(int row, int k) {
  return (uint32_t)(row >> 3) * kSSBO + (uint32_t)(row & 7) * 16u + (uint32_t)(k >> 3) * 128u + (uint32_t)(k & 7) * 2u;
}

// One CTA per (TW-column tile, 16-row block): 16 TW elements, 8 digit planes of 32 TW bytes. Warp w stages core
// matrices w, w + 8, ... (row group g8 = cm / 2, K group c8 = cm % 2); lane (rr, kp) holds rows 2 kp, 2 kp + 1 of
// column rr of its core matrix.
template <int TW>
__global__ void __launch_bounds__(256)
oz_slice_kernel(const double* __restrict__ M, int64_t ld, int64_t nrows, int ncols, const int* __restrict__ E,
                uint8_t* __restrict__ img, int nkb) {
  constexpr uint32_t plane = (TW / 8) * kSSBO;
  const int tile = blockIdx.x / nkb, kb = blockIdx.x % nkb;
  const int warp = threadIdx.x / 32, lane = threadIdx.x & 31;
  const int rr = lane >> 2, kp = lane & 3;
  uint8_t* out = img + ((size_t)tile * nkb + kb) * kDig * plane;
#pragma unroll
  for (int i = 0; i < TW / 32; ++i) {
    const int cm = warp + 8 * i;
    const int g8 = cm >> 1, c8 = cm & 1;
    const int col = tile * TW + 8 * g8 + rr;
    const int64_t r = (int64_t)kb * kSK + 8 * c8 + 2 * kp;
    const bool cok = col < ncols;
    const double* p = M + r + (int64_t)col * ld;
    const double x0 = (cok && r < nrows) ? __ldg(p) : 0.0;
    const double x1 = (cok && r + 1 < nrows) ? __ldg(p + 1) : 0.0;
    const int Ec = cok ? __ldg(E + col) : kNoExp;
    const unsigned long long t0 = biased_digits(x0, Ec), t1 = biased_digits(x1, Ec);
    const uint32_t off = tile_off16(8 * g8 + rr, 8 * c8 + 2 * kp);
#pragma unroll
    for (int j = 0; j < kDig; ++j) *reinterpret_cast<uint32_t*>(out + j * plane + off) = digit_pair(t0, t1, j);
  }
}

struct OzImgSmem {
  uint64_t full[kSBuf];
  uint64_t empty[kSBuf];
  uint32_t tmem_slot;
  int ok;
  int issued, consumed;
  int Ea[kM];
  int Eb[kN2];
};

// Image-fed product. Gram (UPD = false): out = the split's FP64 partial of A^T B (ma x mb, leading dimension ma),
// A/B the column images; Ea/Eb column exponents. Update (UPD = true): out = Y (ma = n rows, mb = p columns,
// leading dimension ldo) receives A G (mode Store) or Y - A G (mode Sub), A the row image of the n x m operand
// (row exponents Ea), B the column image of G (column exponents Eb). grid (tiles_m * tiles_n, nsplit); the split
// covers 16-row (16-column for the update) blocks [y * kb_per_split, min(nkb, (y + 1) * kb_per_split)).
struct ImgArgs {
  const uint8_t* imgA;
  const uint8_t* imgB;
  int nkb, ma, mb, tiles_n, kb_per_split;
  const int* Ea;
  const int* Eb;
  double* out;
  int64_t ldo;
  int symmetric, mode;
  int upper;        // update: G upper triangular, so column tile [n0, n0 + 128) needs only its rows < n0 + 128
  int* flag;
};

// fold the 4 accumulators of pass p (groups 4 p .. 4 p + 3) of this warp's 32 lanes x 64 columns into (hi, lo)
__device__ __forceinline__ void fold_pass(uint32_t tmem, int q, int h, int pass, float (&hi)[64], float (&lo)[64]) {
#pragma unroll 1
  for (int gl = 3; gl >= 0; --gl) {
    const int g = 4 * pass + gl;
    const float w = __int_as_float((127 - 7 * g) << 23);   // 2^(-7 g), exact
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      float v[32];
      tmem_ld32(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(gl * kN2 + 64 * h + 32 * c), v);
#pragma unroll
      for (int i = 0; i < 32; ++i) {
        const float x = v[i] * w;
        const float sm = hi[32 * c + i] + x;
        const float bb = sm - hi[32 * c + i];
        lo[32 * c + i] += (hi[32 * c + i] - (sm - bb)) + (x - bb);
        hi[32 * c + i] = sm;
      }
    }
  }
}

template <bool UPD>
__global__ void __launch_bounds__(kThreads, 1) oz_img_kernel(ImgArgs a) {
  extern __shared__ __align__(1024) uint8_t dyn[];
  __shared__ OzImgSmem sm;
  const int tm = blockIdx.x / a.tiles_n, tn = blockIdx.x % a.tiles_n;
  const int m0 = tm * kM, n0 = tn * kN2;
  if (!UPD && a.symmetric && n0 + kN2 <= m0) return;   // entirely below the diagonal: the reduce reads only i <= j
  const int kb0 = blockIdx.y * a.kb_per_split;
  int kb1 = min(a.nkb, kb0 + a.kb_per_split);
  if (UPD && a.upper) kb1 = min(kb1, (n0 + kN2 + kSK - 1) / kSK);   // the rows of G below are zero in this tile
  const int nst = kb1 > kb0 ? kb1 - kb0 : 0;
  const int tid = threadIdx.x;
  for (int i = tid; i < kM; i += kThreads) sm.Ea[i] = (m0 + i < a.ma) ? a.Ea[m0 + i] : kNoExp;
  for (int i = tid; i < kN2; i += kThreads) sm.Eb[i] = (n0 + i < a.mb) ? a.Eb[n0 + i] : kNoExp;
  if (tid == 0) {
    for (int b = 0; b < kSBuf; ++b) {
      mbar_init(smem_u32(&sm.full[b]), 1);
      mbar_init(smem_u32(&sm.empty[b]), 1);
    }
    sm.ok = 1;
    sm.issued = 0;
    sm.consumed = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncwarp();
  if (tid / 32 == 0) tmem_alloc(smem_u32(&sm.tmem_slot), 512);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = sm.tmem_slot;
  const int warp = tid / 32, lane = tid & 31;
  const int q = warp & 3, h = warp >> 2;
  const uint8_t* srcA = a.imgA + (size_t)tm * a.nkb * kImgBlk;
  const uint8_t* srcB = a.imgB + (size_t)tn * a.nkb * kImgBlk;
  // Items fill buffers in consumption order. Chunk ci (CB = kSChunkBlocks stages, the last chunk possibly shorter,
  // len stages) takes ceil(len / 2) pass-0 items, each the low planes of two stages, then len pass-1 items, one
  // stage each. Thread 0 of warp 0 produces (bulk copies into a free buffer), thread 0 of warp 1 consumes (MMAs,
  // then a commit that frees the buffer); both run ahead independently within a (chunk, pass) block, and all warps
  // meet at its end to fold its 4 group accumulators. issued / consumed live in shared memory for the timeout path.
  constexpr int kCI = kSChunkBlocks / 2 + kSChunkBlocks;   // items of a full chunk
  const int nchunk = (int)ceil_div(nst, kSChunkBlocks);
  const int last_len = nst - (nchunk - 1) * kSChunkBlocks;
  const int nit = nchunk == 0 ? 0 : (nchunk - 1) * kCI + (last_len + 1) / 2 + last_len;
  auto issue = [&](int t) {                       // item t into buffer t % kSBuf
    const int ci = t / kCI, c0 = ci * kSChunkBlocks;
    const int len = min(kSChunkBlocks, nst - c0), n0 = (len + 1) / 2, r = t - kCI * ci;
    const int b = t % kSBuf;
    const uint32_t dst = smem_u32(dyn + b * kStage2);
    const uint32_t fb = smem_u32(&sm.full[b]);
    if (r < n0) {                                 // pass 0: planes 0..3 of stages c0 + 2 r (and c0 + 2 r + 1)
      const int st = c0 + 2 * r, ns = min(2, c0 + len - st);
      mbar_expect_tx(fb, 2u * (uint32_t)ns * kHalf);
      for (int u = 0; u < ns; ++u) {
        bulk_g2s(dst + u * kHalf, srcA + (size_t)(kb0 + st + u) * kImgBlk, kHalf, fb);
        bulk_g2s(dst + kImgBlk + u * kHalf, srcB + (size_t)(kb0 + st + u) * kImgBlk, kHalf, fb);
      }
    } else {                                      // pass 1: all planes of stage c0 + r - n0
      const int st = c0 + r - n0;
      mbar_expect_tx(fb, 2 * kImgBlk);
      bulk_g2s(dst, srcA + (size_t)(kb0 + st) * kImgBlk, kImgBlk, fb);
      bulk_g2s(dst + kImgBlk, srcB + (size_t)(kb0 + st) * kImgBlk, kImgBlk, fb);
    }
  };
  float hi[64], lo[64];
#pragma unroll
  for (int i = 0; i < 64; ++i) { hi[i] = 0.f; lo[i] = 0.f; }
  constexpr uint32_t idesc = idesc_bf16(kM, kN2);
  bool ok = true;
  int issued = 0, consumed = 0;                   // thread 0 / thread 32 only
  for (int ci = 0; ci < nchunk && ok; ++ci) {
    const int len = min(kSChunkBlocks, nst - ci * kSChunkBlocks), n0 = (len + 1) / 2;
    for (int pass = 0; pass < 2; ++pass) {
      const int tb0 = kCI * ci + (pass ? n0 : 0), tb1 = tb0 + (pass ? len : n0);
      if (tid == 0) {
        // keep up to kSBuf items in flight: this block's and the first ones of the next
        const int upto = min(nit, tb1 + kSBuf - 1);
        for (int t = issued; t < upto && sm.ok; ++t) {
          if (t >= kSBuf && !mbar_wait(smem_u32(&sm.empty[t % kSBuf]), (uint32_t)((t / kSBuf - 1) & 1))) {
            sm.ok = 0;
            break;
          }
          issue(t);
          issued = t + 1;
          sm.issued = issued;
        }
      } else if (tid == 32) {
        for (int t = tb0; t < tb1 && sm.ok; ++t) {
          const int b = t % kSBuf;
          if (!mbar_wait(smem_u32(&sm.full[b]), (uint32_t)((t / kSBuf) & 1))) {
            sm.ok = 0;
            break;
          }
          tc_fence_after();
          const uint32_t a0 = smem_u32(dyn + b * kStage2), b0 = a0 + kImgBlk;
          const bool first = t == tb0;
          if (pass == 0) {
            const int ns = min(2, len - 2 * (t - tb0));
            for (int u = 0; u < ns; ++u) {
#pragma unroll
              for (int g = 0; g < 4; ++g) {
                for (int j = 0; j <= g; ++j) {       // digit pairs (j, g - j), planes 0..3
                  mma_bf16(tmem + (uint32_t)(g * kN2), smem_desc_nosw(a0 + u * kHalf + j * kSAPlane, 128, kSSBO),
                           smem_desc_nosw(b0 + u * kHalf + (g - j) * kSAPlane, 128, kSSBO), idesc,
                           (first && u == 0 && j == 0) ? 0u : 1u);
                }
              }
            }
          } else {
#pragma unroll
            for (int gl = 0; gl < 4; ++gl) {
              const int g = 4 + gl;
              for (int j = 0; j <= g; ++j) {         // digit pairs (j, g - j), both at most 7 since g <= 7
                mma_bf16(tmem + (uint32_t)(gl * kN2), smem_desc_nosw(a0 + j * kSAPlane, 128, kSSBO),
                         smem_desc_nosw(b0 + (g - j) * kSAPlane, 128, kSSBO), idesc, (first && j == 0) ? 0u : 1u);
              }
            }
          }
          mma_commit(smem_u32(&sm.empty[b]));
          consumed = t + 1;
          sm.consumed = consumed;
        }
        // the block's products are complete once its last commit has arrived
        if (sm.ok && consumed == tb1 &&
            !mbar_wait(smem_u32(&sm.empty[(tb1 - 1) % kSBuf]), (uint32_t)(((tb1 - 1) / kSBuf) & 1)))
          sm.ok = 0;
      }
      __syncthreads();
      if (!sm.ok) { ok = false; break; }
      tc_fence_after();
      fold_pass(tmem, q, h, pass, hi, lo);
      tc_fence_before();
      __syncthreads();
    }
  }
  if (ok) {
    const int ri = 32 * q + lane;
    const int gi = m0 + ri;
    if (gi < a.ma) {
      const int Ei = sm.Ea[ri];
      double* row = UPD ? a.out + gi : a.out + (int64_t)blockIdx.y * a.ma * a.mb + gi;
      const int64_t ld = UPD ? a.ldo : a.ma;
#pragma unroll
      for (int i = 0; i < 64; ++i) {            // fully unrolled: hi / lo stay in registers
        const int cj = 64 * h + i;
        const int gj = n0 + cj;
        if (gj >= a.mb) continue;
        const int Ej = sm.Eb[cj];
        const double v = (nst == 0 || Ei == kNoExp || Ej == kNoExp) ? 0.0
                                                                    : (widen(hi[i]) + widen(lo[i])) * pow2(Ei + Ej - 10);
        double* o = row + (int64_t)gj * ld;
        *o = (UPD && a.mode != (int)Epi::Store) ? *o - v : v;
      }
    }
  }
  if (tid == 0 && !ok) {
    atomicOr(a.flag, kFlagTimeout);
    // wait (bounded) for the copies and MMAs still in flight before the CTA gives its memory back
    const int iss = sm.issued, con = sm.consumed;
    for (int t = con; t < iss; ++t)
      mbar_wait(smem_u32(&sm.full[t % kSBuf]), (uint32_t)((t / kSBuf) & 1));
    if (con > 0) mbar_wait(smem_u32(&sm.empty[(con - 1) % kSBuf]), (uint32_t)(((con - 1) / kSBuf) & 1));
  }
  tc_fence_before();
  __syncthreads();
  if (tid / 32 == 0) {
    __syncwarp();
    tc_fence_after();
    tmem_dealloc(tmem, 512);
  }
}

// Row image of an n x m operand for the update's A role: element (r, c) sits at M-row r, K index c; one CTA per
// (128-row tile, 16-column block); row exponents Er.
__global__ void __launch_bounds__(256)
oz_slice_rows_kernel(const double* __restrict__ M, int64_t ld, int64_t nrows, int ncols, const int* __restrict__ Er,
                     uint8_t* __restrict__ img, int nkb) {
  const int tile = blockIdx.x / nkb, kb = blockIdx.x % nkb;
  const int warp = threadIdx.x / 32, lane = threadIdx.x & 31;
  const int rr = lane >> 2, kp = lane & 3;
  uint8_t* out = img + ((size_t)tile * nkb + kb) * kDig * kSAPlane;
#pragma unroll
  for (int i = 0; i < kM / 32; ++i) {
    const int cm = warp + 8 * i;
    const int g8 = cm >> 1, c8 = cm & 1;
    const int64_t r = (int64_t)tile * kM + 8 * g8 + rr;
    const int c = kb * kSK + 8 * c8 + 2 * kp;
    const bool rok = r < nrows;
    const double x0 = (rok && c < ncols) ? __ldg(M + r + (int64_t)c * ld) : 0.0;
    const double x1 = (rok && c + 1 < ncols) ? __ldg(M + r + (int64_t)(c + 1) * ld) : 0.0;
    const int Ei = rok ? __ldg(Er + r) : kNoExp;
    const unsigned long long t0 = biased_digits(x0, Ei), t1 = biased_digits(x1, Ei);
    const uint32_t off = tile_off16(8 * g8 + rr, 8 * c8 + 2 * kp);
#pragma unroll
    for (int j = 0; j < kDig; ++j) *reinterpret_cast<uint32_t*>(out + j * kSAPlane + off) = digit_pair(t0, t1, j);
  }
}

size_t oz_img_smem() { return (size_t)kSBuf * kStage2 + 1024; }

size_t oz_smem() { return 2 * (size_t)kStageBytes + 1024; }

int sm_count() {
  static const int sms = [] {               // initialised once, thread-safe (concurrent batched solves)
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    return v > 0 ? v : 1;
  }();
  return sms;
}

// one CTA per SM: the kernels allocate all 512 TMEM columns
cudaError_t prep(const void* fn) {
  const size_t smem = oz_smem();
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kThreads, smem);
  if (e != cudaSuccess) return e;
  return per_sm <= 1 ? cudaSuccess : cudaErrorInvalidConfiguration;
}

}  // namespace

size_t oz_exp_elems(int64_t n, int cols) { return (size_t)(n > cols ? n : cols) + (size_t)cols + 64; }

// one CTA per SM: the image kernels allocate all 512 TMEM columns
cudaError_t prep_img(const void* fn) {
  const size_t smem = oz_img_smem();
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kThreads, smem);
  if (e != cudaSuccess) return e;
  return per_sm <= 1 ? cudaSuccess : cudaErrorInvalidConfiguration;
}

size_t oz_img_bytes(int64_t n, int cols) {   // the images of both operands (128-column tiles each)
  const size_t nkb = (size_t)ceil_div(n, kSK);
  return 2 * (size_t)ceil_div(cols, 128) * kImgBlk * nkb;
}

cudaError_t oz_gram(const double* A, int64_t lda, const double* B, int64_t ldb, int64_t n, int ma, int mb, double* C,
                    int ldc, bool symmetric, double* part, size_t part_capacity, int* exps, uint8_t* img,
                    size_t img_bytes, int* flag, cudaStream_t s) {
  if (ma <= 0 || mb <= 0) return cudaSuccess;
  if ((size_t)ma * mb > part_capacity) return cudaErrorInvalidValue;
  int* Ea = exps;
  int* Eb = exps + ma;
  const bool same = symmetric && A == B;
  cudaError_t e0 = col_exps(A, lda, n, ma, Ea, s);
  if (e0 != cudaSuccess) return e0;
  if (!same) {
    e0 = col_exps(B, ldb, n, mb, Eb, s);
    if (e0 != cudaSuccess) return e0;
  } else {
    Eb = Ea;
  }
  const int tiles_m = (int)ceil_div(ma, kM), tiles_n = (int)ceil_div(mb, kN);
  const int tiles = tiles_m * tiles_n;
  const int64_t nkb64 = ceil_div(n, kSK);
  const size_t bytesA = (size_t)ceil_div(ma, 128) * kImgBlk * nkb64;
  const size_t bytesB = (size_t)ceil_div(mb, 128) * kImgBlk * nkb64;
  if (img && img_bytes >= bytesA + bytesB && mb > kN) {
    // several column tiles of B would each re-slice A: slice each operand once into digit images instead, then
    // run the bulk-copy-fed Gram on 128 x 128 tiles
    const int nkb = (int)ceil_div(n, kSK);
    const int tiles_n2 = (int)ceil_div(mb, kN2);
    const int tiles2 = tiles_m * tiles_n2;
    uint8_t* imgA = img;
    uint8_t* imgB = img + bytesA;
    oz_slice_kernel<128><<<(unsigned)(ceil_div(ma, 128) * nkb), 256, 0, s>>>(A, lda, n, ma, Ea, imgA, nkb);
    oz_slice_kernel<128><<<(unsigned)(ceil_div(mb, 128) * nkb), 256, 0, s>>>(B, ldb, n, mb, Eb, imgB, nkb);
    count_launch(2);
    const size_t smem = oz_img_smem();
    cudaError_t e = prep_img((const void*)oz_img_kernel<false>);
    if (e != cudaSuccess) return e;
    // CTAs that do work (a symmetric Gram skips the tiles below the diagonal); the K split, in whole chunks, is the
    // one with the fewest waves x chunks per CTA (one CTA per SM), the smaller split on ties
    int64_t active = tiles2;
    if (symmetric && ma == mb) active = (int64_t)tiles_m * (tiles_m + 1) / 2;
    const int64_t nchunks = ceil_div(nkb, kSChunkBlocks);
    const int64_t cap_mem = std::max<int64_t>(1, (int64_t)(part_capacity / ((size_t)ma * mb)));
    const int64_t sms = sm_count();
    int64_t cps = nchunks;                        // chunks per split
    int64_t best = ceil_div(active, sms) * nchunks;
    for (int64_t c = nchunks - 1; c >= 1; --c) {
      const int64_t ns = ceil_div(nchunks, c);
      if (ns > cap_mem) break;
      const int64_t cost = ceil_div(active * ns, sms) * c;
      if (cost < best) {
        best = cost;
        cps = c;
      }
    }
    const int kps = (int)(cps * kSChunkBlocks);
    const int nsp = (int)ceil_div(nkb, kps);
    const ImgArgs args{imgA, imgB, nkb, ma, mb, tiles_n2, kps, Ea, Eb, part, ma, symmetric ? 1 : 0, 0, 0, flag};
    oz_img_kernel<false><<<dim3(tiles2, nsp), kThreads, smem, s>>>(args);
    count_launch();
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return gram_reduce_partials(part, nsp, ma, mb, C, ldc, symmetric, s);
  }
  cudaError_t e = prep((const void*)oz_gram_kernel);
  if (e != cudaSuccess) return e;
  int64_t nsplit = ceil_div(sm_count(), tiles);
  const int64_t cap_rows = ceil_div(n, kChunk);
  const int64_t cap_mem = (int64_t)(part_capacity / ((size_t)ma * mb));
  nsplit = std::max<int64_t>(1, std::min(nsplit, std::min(cap_rows, cap_mem)));
  const int64_t rows = ceil_div(ceil_div(n, nsplit), kChunk) * kChunk;
  const int nsp = (int)ceil_div(n, rows);
  oz_gram_kernel<<<dim3(tiles, nsp), kThreads, oz_smem(), s>>>(A, lda, B, ldb, n, ma, mb, tiles_n, rows, Ea, Eb,
                                                                  part, symmetric ? 1 : 0, flag);
  count_launch();
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return gram_reduce_partials(part, nsp, ma, mb, C, ldc, symmetric, s);
}

cudaError_t oz_update(const double* A, int64_t lda, const double* G, int ldg, int64_t n, int m, int p, double* Y,
                      int64_t ldy, Epi mode, int* exps, uint8_t* img, size_t img_bytes, int* flag, cudaStream_t s,
                      bool g_upper) {
  if (p <= 0 || n <= 0) return cudaSuccess;
  int* Er = exps;
  int* Fc = exps + n;
  cudaError_t e = row_exps(A, lda, n, m, Er, s);
  if (e != cudaSuccess) return e;
  e = col_exps(G, ldg, m, p, Fc, s);
  if (e != cudaSuccess) return e;
  const int tiles_m = (int)ceil_div(n, kM), tiles_n = (int)ceil_div(p, kN2);
  const int nkb = (int)ceil_div(m, kSK);
  const size_t bytesA = (size_t)tiles_m * nkb * kImgBlk;
  const size_t bytesB = (size_t)tiles_n * nkb * kImgBlk;
  if (img && img_bytes >= bytesA + bytesB && p > kN) {
    // several column tiles of G would each re-slice A: slice it once (row image) and feed the tensor cores by
    // bulk copies, on 128 x 128 tiles
    uint8_t* imgA = img;
    uint8_t* imgB = img + bytesA;
    oz_slice_rows_kernel<<<(unsigned)((int64_t)tiles_m * nkb), 256, 0, s>>>(A, lda, n, m, Er, imgA, nkb);
    oz_slice_kernel<128><<<(unsigned)(tiles_n * nkb), 256, 0, s>>>(G, ldg, m, p, Fc, imgB, nkb);
    count_launch(2);
    e = prep_img((const void*)oz_img_kernel<true>);
    if (e != cudaSuccess) return e;
    const ImgArgs args{imgA, imgB, nkb, (int)n, p, tiles_n, nkb, Er, Fc, Y, ldy, 0, (int)mode, g_upper ? 1 : 0,
                       flag};
    oz_img_kernel<true><<<dim3((unsigned)((int64_t)tiles_m * tiles_n), 1), kThreads, oz_img_smem(), s>>>(args);
    count_launch();
    return cudaGetLastError();
  }
  e = prep((const void*)oz_update_kernel);
  if (e != cudaSuccess) return e;
  oz_update_kernel<<<dim3((unsigned)ceil_div(n, kM), (unsigned)ceil_div(p, kN)), kThreads, oz_smem(), s>>>(
      A, lda, G, ldg, n, m, p, Y, ldy, (int)mode, Er, Fc, flag);
  count_launch();
  return cudaGetLastError();
}

}  // namespace ppcg
