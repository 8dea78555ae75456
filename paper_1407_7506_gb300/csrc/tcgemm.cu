// Tensor-core (tcgen05, TF32 or BF16 inputs, FP32 accumulation in TMEM) versions of the tall-skinny GEMMs whose
// rounding only perturbs search directions: the projections of steps 9-10 (G = X^T W, W <- W - X G) and the
// Gram of the first CholeskyQR pass (its error changes only the conditioning of R, not span(X), because
// X R^{-1} is applied in FP64). These are the mixed-precision forms of the method's workload: kind::tf32 with
// K = 8 per instruction, or kind::f16 with BF16 operands and K = 16 per instruction. Both stage 128 bytes of K per
// tile row (32 TF32 or 64 BF16 values), so the shared-memory layout, the descriptors and the four instructions per
// stage are the same; only the conversion and the element packing differ.
//
// The blocks are FP64 in HBM, which TMA cannot convert, so the operand tiles are staged by the threads: FP64
// loads, conversion to TF32 (round to nearest, by integer operations on the upper word), and stores into shared memory in the K-major layout with the
// 128-byte swizzle: a stage holds K = 32 TF32 values (128 B) per tile row, rows 128 B apart, and the 16-byte chunk
// c of row r sits at chunk position c ^ (r mod 8). The swizzle is what lets the loads follow the FP64 data: a warp
// reads 32 consecutive elements of one column (256 contiguous bytes, two cache lines per request) and still writes
// 32 distinct banks. One thread issues tcgen05.mma (M = 128, N = NT, K = 8 per instruction, the descriptor start
// advanced by 32 B inside the 128-byte atom) into a TMEM accumulator and commits to an mbarrier per stage; two
// stages overlap staging with the MMAs. The epilogue reads TMEM with tcgen05.ld (each warp its 32-lane quadrant);
// the Gram writes FP32 partials, the update subtracts in FP64.
//
//   tc_gram    C = A^T B split over row chunks into FP32 partials, summed in FP32 by tc_reduce_kernel and widened
//   tc_update  Y = Y - A G (or Y = A G)
//
// Every mbarrier wait is bounded; on timeout the CTA records kFlagTimeout, waits (bounded) once more for its
// MMAs, frees its TMEM and returns.
#include "ppcg_internal.h"
#include "tc_util.cuh"

#include <algorithm>

namespace ppcg {

namespace {

using namespace tc;

constexpr int kM = 128;           // MMA M: rows of the accumulator = TMEM lanes
constexpr int kBK = 32;           // TF32 K elements staged per stage (4 MMAs of K = 8): one 128-byte swizzle atom
template <bool BF>
constexpr int kbk() { return BF ? 64 : 32; }   // K elements per stage: 128 bytes of TF32 or BF16
constexpr int kThreads = 512;     // 16 warps: 4 per scheduler, to hide the latency of the integer conversions
constexpr int kWarps = kThreads / 32;
constexpr uint32_t kRowB = 128;   // bytes per tile row (kBK TF32 values)
constexpr uint32_t kSBO = 1024;   // bytes between 8-row groups

// byte offset of element (row, k) of a stage tile: row-major 128-byte rows, 16-byte chunks XOR-swizzled by row mod 8
__device__ __forceinline__ uint32_t tile_off(int row, int k) {
  return (uint32_t)row * kRowB + ((uint32_t)((k >> 2) ^ (row & 7)) << 4) + (uint32_t)(k & 3) * 4u;
}
// the same for 2-byte (BF16) elements: 8 per 16-byte chunk
__device__ __forceinline__ uint32_t tile_off_bf(int row, int k) {
  return (uint32_t)row * kRowB + ((uint32_t)((k >> 3) ^ (row & 7)) << 4) + (uint32_t)(k & 7) * 2u;
}

// shared-memory descriptor of a K-major tile with the 128-byte swizzle (layout code 2 in bits 61-63); the tile is
// 1024-byte aligned, so the base offset is 0, and the leading byte offset is unused for this layout
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)((kSBO >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;          // descriptor version of tcgen05
  d |= (uint64_t)2 << 61;          // 128-byte swizzle
  return d;
}

__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// FP32 bit pattern of the TF32 value nearest to the double whose upper 32-bit word is hi, ties away from zero (the
// rounding of cvt.rna.tf32). The upper word holds the sign, the exponent and the leading 20 mantissa bits: the 10
// that TF32 keeps and the first one it drops, which alone decides this rounding. The exponent is rebiased in place
// (1023 -> 127) with integer operations only, so the conversion stays off GB300's narrow FP64 pipe. The magnitude is
// first clamped to [2^-127, 2^128] (two min/max operations instead of compares and selects on the busy integer
// pipe): below that range the result is zero, inside the FP32 subnormal range the rounded subnormal, and at or
// above 2^128 infinity; infinities and NaNs become infinity (the result is non-finite either way).
__device__ __forceinline__ uint32_t tf32_from_hi(uint32_t hi) {
  const uint32_t mag = min(max(hi & 0x7FFFFFFFu, 0x38000000u), 0x47F00000u);
  return ((((mag - 0x38000000u) << 3) + 0x1000u) & 0xFFFFE000u) | (hi & 0x80000000u);
}

// BF16 bit pattern of the value nearest to the double whose upper word is hi, ties away from zero: the same clamp
// and integer rebias to the FP32 layout, then the FP32 pattern rounded to its upper 16 bits (8 significant bits;
// the upper word keeps 20 mantissa bits, enough to decide this rounding). Below 2^-127: zero; at or above 2^128,
// and for infinities and NaNs: infinity.
__device__ __forceinline__ uint32_t bf16_from_hi(uint32_t hi) {
  const uint32_t mag = min(max(hi & 0x7FFFFFFFu, 0x38000000u), 0x47F00000u);
  return (((((mag - 0x38000000u) << 3) + 0x8000u) >> 16) & 0x7FFFu) | ((hi >> 16) & 0x8000u);
}

__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// upper 32-bit word of a double in global memory (little-endian: at byte offset 4)
__device__ __forceinline__ uint32_t ld_hi(const double* p) {
  return __ldg(reinterpret_cast<const uint32_t*>(p) + 1);
}

struct TcSmem {
  uint64_t mbar[2];
  uint32_t tmem_slot;
  int ok;
};

// Shared machinery: K loop over nk stages of kBK. `load(kb, r)` issues the global loads of stage kb into the
// register set r, `store(a_tile, b_tile, r)` converts r and writes the stage tiles; thread 0 issues the MMAs. Two
// register sets alternate, and the loads of stage kb+1 are issued before stage kb is converted, so their memory
// latency overlaps the conversion, the barrier and the MMA issue of stage kb.
// Returns false (uniformly) if a bounded wait gave up; TMEM is still allocated on return (caller frees it).
// The A tile has MT halves of 128 rows, each with its own accumulator of NT TMEM columns (at column h NT), and
// every staged B tile feeds all of them.
template <class Regs, int MT, int NT, bool BF, class LoadFn, class StoreFn>
__device__ bool tc_mainloop(int nk, uint8_t* tiles, uint32_t a_bytes, uint32_t b_bytes, TcSmem& sm, uint32_t tmem,
                            uint32_t idesc, LoadFn load, StoreFn store) {
  const int tid = threadIdx.x;
  const uint32_t stage_bytes = a_bytes + b_bytes;
  Regs r0, r1;
  auto step = [&](int kb, Regs& cur, Regs& nxt) -> bool {
    const int s = kb & 1;
    uint8_t* a_tile = tiles + s * stage_bytes;
    uint8_t* b_tile = a_tile + a_bytes;
    if (kb + 1 < nk) load(kb + 1, nxt);
    if (kb >= 2) {
      // the MMAs of step kb-2 used this stage: wait for their commit (completion number (kb-2)/2)
      if (tid == 0) sm.ok = mbar_wait(smem_u32(&sm.mbar[s]), (uint32_t)(((kb - 2) >> 1) & 1)) ? 1 : 0;
      __syncthreads();
      if (!sm.ok) return false;
    }
    store(a_tile, b_tile, cur);
    fence_async_smem();
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
      const uint32_t a0 = smem_u32(a_tile), b0 = smem_u32(b_tile);
#pragma unroll
      for (int j = 0; j < 4; ++j)                    // 32 bytes of K per instruction (8 TF32 or 16 BF16)
#pragma unroll
        for (int h = 0; h < MT; ++h) {
          const uint64_t ad = smem_desc(a0 + h * kM * kRowB + j * 32), bd = smem_desc(b0 + j * 32);
          const uint32_t acc = (kb > 0 || j > 0) ? 1u : 0u;
          if (BF) mma_bf16(tmem + (uint32_t)(h * NT), ad, bd, idesc, acc);
          else mma_tf32(tmem + (uint32_t)(h * NT), ad, bd, idesc, acc);
        }
      mma_commit(smem_u32(&sm.mbar[s]));
    }
    return true;
  };
  if (nk > 0) load(0, r0);
  for (int kb = 0; kb < nk; kb += 2) {
    if (!step(kb, r0, r1)) return false;
    if (kb + 1 < nk && !step(kb + 1, r1, r0)) return false;
  }
  if (nk > 0) {
    const int last = nk - 1;
    if (tid == 0) sm.ok = mbar_wait(smem_u32(&sm.mbar[last & 1]), (uint32_t)((last >> 1) & 1)) ? 1 : 0;
    __syncthreads();
    if (!sm.ok) return false;
  }
  tc_fence_after();
  return true;
}

__device__ void tc_setup(TcSmem& sm, uint32_t ncols) {
  if (threadIdx.x == 0) {
    mbar_init(smem_u32(&sm.mbar[0]), 1);
    mbar_init(smem_u32(&sm.mbar[1]), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncwarp();
  if (threadIdx.x / 32 == 0) tmem_alloc(smem_u32(&sm.tmem_slot), ncols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
}

__device__ void tc_teardown(TcSmem& sm, uint32_t tmem, uint32_t ncols, bool ok, int nk, int* flag) {
  if (!ok) {
    // a bounded wait gave up: record it and give the in-flight MMAs one more bounded wait before freeing TMEM
    if (threadIdx.x == 0) {
      atomicOr(flag, kFlagTimeout);
      if (nk > 0) mbar_wait(smem_u32(&sm.mbar[(nk - 1) & 1]), (uint32_t)(((nk - 1) >> 1) & 1));
    }
  }
  tc_fence_before();
  __syncthreads();
  if (threadIdx.x / 32 == 0) {
    __syncwarp();
    tc_fence_after();
    tmem_dealloc(tmem, ncols);
  }
}

// Per-thread register staging: all global loads of a stage are issued before any is converted and stored, and the
// next stage's loads are issued while the MMAs run.
template <int NT, int MT, bool BF>
struct Stage {
  static constexpr int kA = MT * kM * kbk<BF>() / kThreads;    // elements of A per thread
  static constexpr int kB = NT * kbk<BF>() / kThreads;         // elements of B per thread
  uint32_t a[kA];   // upper words of the FP64 elements
  uint32_t b[kB];
};

// 1024-byte aligned start of the stage tiles inside the dynamic shared memory (its size includes 1024 B of slack)
__device__ __forceinline__ uint8_t* align_tiles(uint8_t* dyn) {
  return dyn + ((1024u - (smem_u32(dyn) & 1023u)) & 1023u);
}

// ------------------------------------------------------------------------------------------ C = A^T B partials
// grid (tiles_m * tiles_n, nsplit); tile rows m0 = tm * 128 MT (columns of A), cols n0 = tn * NT (columns of B)
template <int NT, int MT, bool BF>
__global__ void __launch_bounds__(kThreads, 1)
tc_gram_kernel(const double* __restrict__ A, int64_t lda, const double* __restrict__ B, int64_t ldb, int64_t n,
               int ma, int mb, int tiles_n, int64_t rows_per_split, float* __restrict__ part, int* flag) {
  using Regs = Stage<NT, MT, BF>;
  constexpr int BK = kbk<BF>();
  extern __shared__ __align__(1024) uint8_t dyn[];
  __shared__ TcSmem sm;
  const int tm = blockIdx.x / tiles_n, tn = blockIdx.x % tiles_n;
  const int m0 = tm * kM * MT, n0 = tn * NT;
  const int64_t r_begin = (int64_t)blockIdx.y * rows_per_split;
  const int64_t r_end = min(n, r_begin + rows_per_split);
  const int nk = r_end > r_begin ? (int)ceil_div(r_end - r_begin, BK) : 0;
  constexpr uint32_t a_bytes = MT * kM * kRowB, b_bytes = (uint32_t)NT * kRowB;
  constexpr uint32_t ncols = (uint32_t)(MT * NT);
  tc_setup(sm, ncols);
  const uint32_t tmem = sm.tmem_slot;
  const int warp = threadIdx.x / 32, lane = threadIdx.x & 31;
  // TF32: lane = k (a row of A and B), warp w takes tile rows w, w + 16, ...: 256 contiguous bytes per warp load.
  // BF16: lane = the pair of rows k = 2 lane, 2 lane + 1 (512 contiguous bytes per warp), packed into one word.
  constexpr int P = BF ? 2 : 1;
  auto load = [&](int kb, Regs& reg) {
    const int64_t r = r_begin + (int64_t)kb * BK + P * lane;
#pragma unroll
    for (int i = 0; i < Regs::kA / P; ++i) {
      const int col = m0 + warp + kWarps * i;
#pragma unroll
      for (int e = 0; e < P; ++e)
        reg.a[P * i + e] = (r + e < r_end && col < ma) ? ld_hi(A + r + e + (int64_t)col * lda) : 0u;
    }
#pragma unroll
    for (int i = 0; i < Regs::kB / P; ++i) {
      const int col = n0 + warp + kWarps * i;
#pragma unroll
      for (int e = 0; e < P; ++e)
        reg.b[P * i + e] = (r + e < r_end && col < mb) ? ld_hi(B + r + e + (int64_t)col * ldb) : 0u;
    }
  };
  auto store = [&](uint8_t* a_tile, uint8_t* b_tile, const Regs& reg) {
    if (BF) {
#pragma unroll
      for (int i = 0; i < Regs::kA / 2; ++i)
        *reinterpret_cast<uint32_t*>(a_tile + tile_off_bf(warp + kWarps * i, 2 * lane)) =
            bf16_from_hi(reg.a[2 * i]) | (bf16_from_hi(reg.a[2 * i + 1]) << 16);
#pragma unroll
      for (int i = 0; i < Regs::kB / 2; ++i)
        *reinterpret_cast<uint32_t*>(b_tile + tile_off_bf(warp + kWarps * i, 2 * lane)) =
            bf16_from_hi(reg.b[2 * i]) | (bf16_from_hi(reg.b[2 * i + 1]) << 16);
    } else {
#pragma unroll
      for (int i = 0; i < Regs::kA; ++i)
        *reinterpret_cast<uint32_t*>(a_tile + tile_off(warp + kWarps * i, lane)) = tf32_from_hi(reg.a[i]);
#pragma unroll
      for (int i = 0; i < Regs::kB; ++i)
        *reinterpret_cast<uint32_t*>(b_tile + tile_off(warp + kWarps * i, lane)) = tf32_from_hi(reg.b[i]);
    }
  };
  const bool ok = tc_mainloop<Regs, MT, NT, BF>(nk, align_tiles(dyn), a_bytes, b_bytes, sm, tmem,
                                                BF ? idesc_bf16(kM, NT) : idesc_tf32(kM, NT), load, store);
  if (ok) {
    // epilogue: warp w reads TMEM lanes 32 (w % 4).. (its quadrant) of every half, 16-column chunks w / 4, + 4, ...
    float* out = part + (int64_t)blockIdx.y * ma * mb;
    const int q = warp & 3, h = warp >> 2;
#pragma unroll 1
    for (int half = 0; half < MT; ++half) {
      const int gi = m0 + half * kM + 32 * q + lane;
#pragma unroll 1
      for (int c0 = 16 * h; c0 < NT; c0 += 16 * (kWarps / 4)) {
        float v[16];
        if (nk > 0) tmem_ld16(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(half * NT + c0), v);
        else
#pragma unroll
          for (int i = 0; i < 16; ++i) v[i] = 0.f;
        if (gi < ma) {
#pragma unroll
          for (int i = 0; i < 16; ++i) {
            const int gj = n0 + c0 + i;
            if (gj < mb) out[gi + (int64_t)gj * ma] = v[i];
          }
        }
      }
    }
  }
  tc_teardown(sm, tmem, ncols, ok, nk, flag);
}

// C = sum over the nsplit FP32 partials, summed in FP32 (their rounding, ~nsplit 2^-24 relative, is far below the
// 2^-11 of the TF32 inputs) and widened to FP64; a symmetric C takes its lower triangle from the upper one.
__global__ void tc_reduce_kernel(const float* __restrict__ part, int nsplit, int ma, int mb, double* __restrict__ C,
                                 int ldc, int symmetric) {
  const int64_t total = (int64_t)ma * mb;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % ma), j = (int)(e / ma);
    const int64_t o = (symmetric && i > j) ? j + (int64_t)i * ma : e;
    float s0 = 0.f, s1 = 0.f;
    int q = 0;
    for (; q + 1 < nsplit; q += 2) {
      s0 += __ldg(part + (int64_t)q * total + o);
      s1 += __ldg(part + (int64_t)(q + 1) * total + o);
    }
    if (q < nsplit) s0 += __ldg(part + (int64_t)q * total + o);
    C[i + (int64_t)j * ldc] = widen(s0 + s1);
  }
}

// ------------------------------------------------------------------------------------------ Y = Y - A G / Y = A G
// grid (ceil(n / (128 MT)), ceil(p / NT)); A: n x m, G: m x p, Y: n x p
template <int NT, int MT, bool BF>
__global__ void __launch_bounds__(kThreads, 1)
tc_update_kernel(const double* __restrict__ A, int64_t lda, const double* __restrict__ G, int ldg, int64_t n, int m,
                 int p, double* Y, int64_t ldy, int subtract, int* flag) {
  using Regs = Stage<NT, MT, BF>;
  constexpr int BK = kbk<BF>();
  extern __shared__ __align__(1024) uint8_t dyn[];
  __shared__ TcSmem sm;
  const int64_t r0 = (int64_t)blockIdx.x * kM * MT;
  const int c0 = blockIdx.y * NT;
  const int nk = (int)ceil_div(m, BK);
  constexpr uint32_t a_bytes = MT * kM * kRowB, b_bytes = (uint32_t)NT * kRowB;
  constexpr uint32_t ncols = (uint32_t)(MT * NT);
  constexpr int kRows = MT * kM;
  tc_setup(sm, ncols);
  const uint32_t tmem = sm.tmem_slot;
  const int warp = threadIdx.x / 32, lane = threadIdx.x & 31;
  // A: thread items (row, 16-byte chunk of k: 4 TF32 or 8 BF16 values); lanes run down 32 consecutive rows of X (256
  // contiguous bytes per load) and each item is one 16-byte store, conflict-free under the swizzle.
  // B (G, contiguous along k): lane = k (TF32) or the pair k = 2 lane, 2 lane + 1 (BF16).
  constexpr int E = BF ? 8 : 4;                    // elements per 16-byte chunk
  constexpr int P = BF ? 2 : 1;
  auto load = [&](int kb, Regs& reg) {
    const int k0 = kb * BK;
#pragma unroll
    for (int i = 0; i < Regs::kA / E; ++i) {
      const int it = threadIdx.x + kThreads * i;
      const int row = it % kRows, c = it / kRows;
      const int64_t gr = r0 + row;
#pragma unroll
      for (int j = 0; j < E; ++j) {
        const int gk = k0 + E * c + j;
        reg.a[E * i + j] = (gr < n && gk < m) ? ld_hi(A + gr + (int64_t)gk * lda) : 0u;
      }
    }
    const int gk = k0 + P * lane;
#pragma unroll
    for (int i = 0; i < Regs::kB / P; ++i) {
      const int gc = c0 + warp + kWarps * i;
#pragma unroll
      for (int e = 0; e < P; ++e)
        reg.b[P * i + e] = (gk + e < m && gc < p) ? ld_hi(G + gk + e + (int64_t)gc * ldg) : 0u;
    }
  };
  auto store = [&](uint8_t* a_tile, uint8_t* b_tile, const Regs& reg) {
#pragma unroll
    for (int i = 0; i < Regs::kA / E; ++i) {
      const int it = threadIdx.x + kThreads * i;
      const int row = it % kRows, c = it / kRows;
      uint4 v;
      if (BF) {
        v.x = bf16_from_hi(reg.a[E * i + 0]) | (bf16_from_hi(reg.a[E * i + 1]) << 16);
        v.y = bf16_from_hi(reg.a[E * i + 2]) | (bf16_from_hi(reg.a[E * i + 3]) << 16);
        v.z = bf16_from_hi(reg.a[E * i + 4]) | (bf16_from_hi(reg.a[E * i + 5]) << 16);
        v.w = bf16_from_hi(reg.a[E * i + 6]) | (bf16_from_hi(reg.a[E * i + 7]) << 16);
        *reinterpret_cast<uint4*>(a_tile + tile_off_bf(row, E * c)) = v;
      } else {
        v.x = tf32_from_hi(reg.a[E * i + 0]);
        v.y = tf32_from_hi(reg.a[E * i + 1]);
        v.z = tf32_from_hi(reg.a[E * i + 2]);
        v.w = tf32_from_hi(reg.a[E * i + 3]);
        *reinterpret_cast<uint4*>(a_tile + tile_off(row, E * c)) = v;
      }
    }
#pragma unroll
    for (int i = 0; i < Regs::kB / P; ++i) {
      const uint32_t word = BF ? (bf16_from_hi(reg.b[2 * i]) | (bf16_from_hi(reg.b[2 * i + 1]) << 16))
                               : tf32_from_hi(reg.b[i]);
      *reinterpret_cast<uint32_t*>(b_tile + (BF ? tile_off_bf(warp + kWarps * i, 2 * lane)
                                                : tile_off(warp + kWarps * i, lane))) = word;
    }
  };
  const bool ok = tc_mainloop<Regs, MT, NT, BF>(nk, align_tiles(dyn), a_bytes, b_bytes, sm, tmem,
                                                BF ? idesc_bf16(kM, NT) : idesc_tf32(kM, NT), load, store);
  if (ok) {
    const int q = warp & 3, h = warp >> 2;         // TMEM lane quadrant; 16-column chunks h, h + kWarps/4, ...
#pragma unroll 1
    for (int half = 0; half < MT; ++half) {
      const int64_t gr = r0 + half * kM + 32 * q + lane;
#pragma unroll 1
      for (int cc = 16 * h; cc < NT; cc += 16 * (kWarps / 4)) {
        float v[16];
        if (nk > 0) tmem_ld16(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(half * NT + cc), v);
        else
#pragma unroll
          for (int i = 0; i < 16; ++i) v[i] = 0.f;
        if (gr < n) {
          double y[16];
#pragma unroll
          for (int i = 0; i < 16; ++i) {
            const int gc = c0 + cc + i;
            y[i] = (subtract && gc < p) ? Y[gr + (int64_t)gc * ldy] : 0.0;
          }
#pragma unroll
          for (int i = 0; i < 16; ++i) {
            const int gc = c0 + cc + i;
            if (gc < p) Y[gr + (int64_t)gc * ldy] = subtract ? (y[i] - widen(v[i])) : widen(v[i]);
          }
        }
      }
    }
  }
  tc_teardown(sm, tmem, ncols, ok, nk, flag);
}

int pick_nt(int cols) {
  if (cols <= 32) return 32;
  if (cols <= 64) return 64;
  if (cols <= 128) return 128;
  return 256;
}

size_t tc_smem_bytes(int NT, int MT) { return 2 * ((size_t)MT * kM * kRowB + (size_t)NT * kRowB) + 1024; }

// Sets the dynamic shared memory of fn to at least `bytes`, padded so that no more CTAs than 512 / cols can be
// resident on one SM: tcgen05.alloc waits for free TMEM columns, and the SM has 512.
cudaError_t set_smem(const void* fn, size_t& bytes, int cols) {
  const int max_ctas = 512 / cols;
  for (int tries = 0; tries < 8; ++tries) {
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kThreads, bytes);
    if (e != cudaSuccess) return e;
    if (per_sm <= max_ctas) return cudaSuccess;
    bytes = std::min<size_t>(bytes * 2, 200 * 1024);
  }
  return cudaErrorInvalidConfiguration;
}

int sm_count() {
  static const int sms = [] {               // initialised once, thread-safe (concurrent batched solves)
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    return v > 0 ? v : 1;
  }();
  return sms;
}


template <int NT, int MT, bool BF>
cudaError_t launch_gram(dim3 grid, const double* A, int64_t lda, const double* B, int64_t ldb, int64_t n, int ma,
                        int mb, int tiles_n, int64_t rows, float* part, int* flag, cudaStream_t s) {
  size_t smem = tc_smem_bytes(NT, MT);
  cudaError_t e = set_smem((const void*)tc_gram_kernel<NT, MT, BF>, smem, NT * MT);
  if (e != cudaSuccess) return e;
  tc_gram_kernel<NT, MT, BF><<<grid, kThreads, smem, s>>>(A, lda, B, ldb, n, ma, mb, tiles_n, rows, part, flag);
  count_launch();
  return cudaGetLastError();
}

template <int MT, bool BF>
cudaError_t launch_gram_nt(int NT, dim3 grid, const double* A, int64_t lda, const double* B, int64_t ldb, int64_t n,
                           int ma, int mb, int tiles_n, int64_t rows, float* part, int* flag, cudaStream_t s) {
  switch (NT) {
    case 32: return launch_gram<32, MT, BF>(grid, A, lda, B, ldb, n, ma, mb, tiles_n, rows, part, flag, s);
    case 64: return launch_gram<64, MT, BF>(grid, A, lda, B, ldb, n, ma, mb, tiles_n, rows, part, flag, s);
    case 128: return launch_gram<128, MT, BF>(grid, A, lda, B, ldb, n, ma, mb, tiles_n, rows, part, flag, s);
    default: return launch_gram<256, MT, BF>(grid, A, lda, B, ldb, n, ma, mb, tiles_n, rows, part, flag, s);
  }
}

template <int NT, int MT, bool BF>
cudaError_t launch_update(const double* A, int64_t lda, const double* G, int ldg, int64_t n, int m, int p, double* Y,
                          int64_t ldy, bool subtract, int* flag, cudaStream_t s) {
  size_t smem = tc_smem_bytes(NT, MT);
  cudaError_t e = set_smem((const void*)tc_update_kernel<NT, MT, BF>, smem, NT * MT);
  if (e != cudaSuccess) return e;
  tc_update_kernel<NT, MT, BF><<<dim3((unsigned)ceil_div(n, (int64_t)kM * MT), (unsigned)ceil_div(p, NT)), kThreads,
                                 smem, s>>>(A, lda, G, ldg, n, m, p, Y, ldy, subtract ? 1 : 0, flag);
  count_launch();
  return cudaGetLastError();
}

template <int MT, bool BF>
cudaError_t launch_update_nt(int NT, const double* A, int64_t lda, const double* G, int ldg, int64_t n, int m, int p,
                             double* Y, int64_t ldy, bool subtract, int* flag, cudaStream_t s) {
  switch (NT) {
    case 32: return launch_update<32, MT, BF>(A, lda, G, ldg, n, m, p, Y, ldy, subtract, flag, s);
    case 64: return launch_update<64, MT, BF>(A, lda, G, ldg, n, m, p, Y, ldy, subtract, flag, s);
    case 128: return launch_update<128, MT, BF>(A, lda, G, ldg, n, m, p, Y, ldy, subtract, flag, s);
    default: return launch_update<256, MT, BF>(A, lda, G, ldg, n, m, p, Y, ldy, subtract, flag, s);
  }
}

}  // namespace

cudaError_t tc_gram(const double* A, int64_t lda, const double* B, int64_t ldb, int64_t n, int ma, int mb, double* C,
                    int ldc, bool symmetric, double* part, size_t part_capacity, int* flag, cudaStream_t s, bool bf16) {
  if (ma <= 0 || mb <= 0) return cudaSuccess;
  if ((size_t)ma * mb > part_capacity) return cudaErrorInvalidValue;
  // BF16 stages twice as many K values per tile row, so its register staging keeps one 128-row accumulator and at
  // most 128 columns
  const int NT = bf16 ? std::min(pick_nt(mb), 128) : pick_nt(mb);
  const int MT = (!bf16 && ma > kM) ? 2 : 1;       // two accumulators share each converted B tile
  const int BK = bf16 ? kbk<true>() : kbk<false>();
  const int tiles_m = (int)ceil_div(ma, kM * MT), tiles_n = (int)ceil_div(mb, NT);
  const int tiles = tiles_m * tiles_n;
  // The K split: the smallest whose waves per unit of K work come within 3% of the fewest (a CTA holds all of its
  // SM's TMEM when MT NT = 512, so one CTA per SM is resident; otherwise 512 / (MT NT)), while the FP32 partials
  // (written, then read by the reduce; mostly L2-resident) stay below half of the input bytes
  const int64_t cap_traffic = (n * (int64_t)(ma + mb)) / (2LL * ma * mb) + 1;
  const int64_t cap_rows = ceil_div(n, 4 * BK);
  const int64_t cap_mem = (int64_t)(2 * part_capacity / ((size_t)ma * mb));   // FP32 partials in FP64 space
  const int64_t cap = std::max<int64_t>(1, std::min(cap_traffic, std::min(cap_rows, cap_mem)));
  const int64_t slots = (int64_t)sm_count() * std::max(1, 512 / (NT * MT));
  const int64_t ns_max = std::min<int64_t>(cap, 4 * slots);
  auto cost = [&](int64_t ns) { return (double)ceil_div((int64_t)tiles * ns, slots) / (double)ns; };
  double best = cost(1);
  for (int64_t ns = 2; ns <= ns_max; ++ns) best = std::min(best, cost(ns));
  int64_t nsplit = 1;
  while (nsplit < ns_max && cost(nsplit) > 1.03 * best) ++nsplit;
  const int64_t rows = ceil_div(ceil_div(n, nsplit), BK) * BK;
  const int nsp = (int)ceil_div(n, rows);
  const dim3 grid(tiles, nsp);
  float* fpart = reinterpret_cast<float*>(part);     // FP32 partials in the FP64 partial buffer (half its bytes)
  cudaError_t e;
  if (bf16) e = launch_gram_nt<1, true>(NT, grid, A, lda, B, ldb, n, ma, mb, tiles_n, rows, fpart, flag, s);
  else if (MT == 2) e = launch_gram_nt<2, false>(NT, grid, A, lda, B, ldb, n, ma, mb, tiles_n, rows, fpart, flag, s);
  else e = launch_gram_nt<1, false>(NT, grid, A, lda, B, ldb, n, ma, mb, tiles_n, rows, fpart, flag, s);
  if (e != cudaSuccess) return e;
  const int64_t blocks = ceil_div((int64_t)ma * mb, 256);
  tc_reduce_kernel<<<(unsigned)(blocks < 8192 ? blocks : 8192), 256, 0, s>>>(fpart, nsp, ma, mb, C, ldc,
                                                                            symmetric ? 1 : 0);
  count_launch();
  return cudaGetLastError();
}

cudaError_t tc_update(const double* A, int64_t lda, const double* G, int ldg, int64_t n, int m, int p, double* Y,
                      int64_t ldy, bool subtract, int* flag, cudaStream_t s, bool bf16) {
  if (p <= 0 || n <= 0) return cudaSuccess;
  if (bf16) return launch_update_nt<1, true>(std::min(pick_nt(p), 128), A, lda, G, ldg, n, m, p, Y, ldy, subtract,
                                             flag, s);
  const int NT = pick_nt(p);
  // 256-row tiles (two accumulators sharing each converted G tile) unless that leaves more than half the SMs idle
  const bool two = 2 * ceil_div(n, (int64_t)2 * kM) * ceil_div(p, NT) >= sm_count();
  return two ? launch_update_nt<2, false>(NT, A, lda, G, ldg, n, m, p, Y, ldy, subtract, flag, s)
             : launch_update_nt<1, false>(NT, A, lda, G, ldg, n, m, p, Y, ldy, subtract, flag, s);
}

}  // namespace ppcg
