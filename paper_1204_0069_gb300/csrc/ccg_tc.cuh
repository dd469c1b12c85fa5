// ccg_tc.cuh -- device primitives for the tensor-core block product:
// mbarriers, TMA tensor loads, tcgen05 MMA / commit / fences, tensor-memory
// loads, the shared-memory and instruction descriptors, and the stream-K
// work split.  Shared by the standalone low-precision block product and the
// persistent solver.  Internal header.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>

namespace ccg {
namespace tc {

// Kinds of quantised A: BF16; FP8 E4M3 with row scales (operand as two E4M3
// terms); FP32 multiplied from TF32 halves, (A_hi + A_lo)(D_hi + D_lo) (the
// low parts split off in shared memory / at conversion); FP64 split without
// error into kSlices FP8 slices of small integers (KIND_SLICED, see
// ccg_lowp.cu): every slice product is exact in the FP32 accumulator.
enum Kind : int { KIND_BF16 = 0, KIND_FP8 = 1, KIND_TF32X3 = 2, KIND_SLICED = 3 };

// Slices of the error-free FP64 split: 4 bits each (integers in [-15, 15],
// exact in E4M3), 56 bits in all.
constexpr int kSlices = 14;

// Error-free 4-bit slicing of x = v 2^-e (|v| < 2^e) with integer operations:
// X = |x| 2^56 rounded to the nearest integer (halves away from zero; the
// dropped remainder is at most 2^-57 and has no sign bias, where truncation
// would shrink every entry toward zero), digit s = bits 55 - 4s .. 52 - 4s
// of X, so that x = sign(v) sum_s digit_s 16^-(s+1) + r, |r| <= 2^-57.
// X stays below 2^56: rounding happens only when v has bits below 2^(e-56),
// i.e. |v| < 2^(e-3).  Each digit is
// written as FP8 E4M3 of sign(v) digit: for d = 2^k (1 + M/8), k = floor(log2
// d), the code is (k + 7) << 3 | M (exponent bias 7, three mantissa bits),
// exact for d <= 15.
__device__ __forceinline__ uint32_t e4m3_digit(uint32_t d, uint32_t neg) {
  if (d == 0u) return 0u;
  const uint32_t k = 31u - (uint32_t)__clz(d);
  return (((k + 7u) << 3) | ((d << (3u - k)) - 8u)) | (neg << 7);
}
__device__ __forceinline__ uint64_t slice_bits(double v, int e, uint32_t* neg) {
  const uint64_t b = (uint64_t)__double_as_longlong(v);
  *neg = (uint32_t)(b >> 63);
  const int be = (int)((b >> 52) & 0x7FF);
  if (be == 0) return 0ull;  // zero or subnormal: below 2^-1022, below any slice here
  const uint64_t m = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);  // v = m 2^(be - 1075)
  const int sh = be - 1075 + 56 - e;  // X = m 2^sh
  if (sh >= 0) return m << sh;        // sh <= 3 since |v| < 2^e
  if (-sh > 60) return 0ull;           // |x| 2^56 < 2^-7: rounds to zero
  return ((m >> (-sh - 1)) + 1ull) >> 1;
}

__host__ __device__ constexpr int pow2_at_least(int v) {
  int r = 32;
  while (r < v) r <<= 1;
  return r;
}

constexpr int kBM = 128;          // rows per tile (MMA M)
constexpr int kRowBytes = 128;    // K bytes per stage = one 128-byte swizzle atom
constexpr int kStages = 6;        // ring depth of the BF16 / FP8 kinds
constexpr int kTileABytes = kBM * kRowBytes;  // 16 KB

template <int KIND, int NP>
struct Shape {
  // B rows: NP (BF16), hi and lo (FP8, TF32), kSlices slices per column
  // (sliced FP64, padded to the MMA's N granularity of 16)
  static constexpr int NB = (KIND == KIND_BF16)     ? NP
                            : (KIND == KIND_SLICED) ? (kSlices * NP + 15) / 16 * 16
                                                    : 2 * NP;
  // FP32 stages also hold the low halves of A: five fit next to the solver's
  // serial scratch for N <= 16 operand columns, four for 32; the sliced
  // operand tile is large for 16 columns
  static constexpr int kStagesK = (KIND == KIND_TF32X3)   ? ((NP <= 16) ? 5 : 4)
                                  : (KIND == KIND_SLICED) ? ((NP >= 16) ? 4 : kStages)
                                                          : kStages;
  static constexpr int kTileBBytes = NB * kRowBytes;
  static constexpr int kTileA2Bytes = (KIND == KIND_TF32X3) ? kTileABytes : 0;  // A_lo
  static constexpr int kStageBytes = kTileABytes + kTileBBytes;  // bytes one TMA stage brings
  // one MMA covers all operand rows (hi and lo, or all slices) at once
  // (N = NB); the epilogue combines the parts of the accumulator
  static constexpr int NMMA = NB;
  static constexpr int kTmemCols = pow2_at_least(2 * NMMA);  // two accumulators
  static constexpr int kRingBytes = kStagesK * (kTileABytes + kTileA2Bytes + kTileBBytes);
  static constexpr int kElemBytes = (KIND == KIND_BF16) ? 2 : (KIND == KIND_TF32X3) ? 4 : 1;
  static_assert(NMMA % 16 == 0 && NMMA <= 256, "MMA N for M = 128");
  static_assert(kTmemCols <= 512, "tensor memory columns");
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// ---- mbarrier --------------------------------------------------------------
__device__ __forceinline__ void mbar_init(uint32_t a, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t a, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(a), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t a) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(a) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t a, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok) : "r"(a), "r"(parity) : "memory");
  return ok != 0;
}
// Bounded wait: false (and the error flag set) after timeout_ns.
__device__ inline bool mbar_wait(uint32_t a, uint32_t parity, long long timeout_ns, int* err) {
  for (int i = 0; i < 128; ++i)
    if (mbar_try(a, parity)) return true;
  const unsigned long long t0 = gtimer();
  while (!mbar_try(a, parity)) {
    if (*(volatile int*)err != 0) return false;
    if (gtimer() - t0 > (unsigned long long)timeout_ns) {
      atomicCAS(err, 0, -5);
      return false;
    }
    __nanosleep(64);
  }
  return true;
}

// ---- TMA -------------------------------------------------------------------
// 2-D tiled TMA load with an L2 eviction policy (createpolicy): the streamed matrix tiles are
// read once per pass and marked evict-first, so the pass does not push the
// small operand and vector blocks the other phases of an iteration re-read
// out of L2; the operand tiles, read by every CTA, are marked evict-last.
__device__ __forceinline__ void tma_load_2d_hint(uint32_t dst, const CUtensorMap* tm, int x, int y,
                                                 uint32_t mbar, uint64_t policy) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint"
      " [%0], [%1, {%2, %3}], [%4], %5;" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(tm)), "r"(x), "r"(y), "r"(mbar), "l"(policy)
      : "memory");
}
__device__ __forceinline__ uint64_t l2_policy_evict_first() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ uint64_t l2_policy_evict_last() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}

// ---- tcgen05 ---------------------------------------------------------------
// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, rows of
// 128 bytes, 8-row groups 1024 bytes apart.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);  // start address
  d |= (uint64_t)1 << 16;                    // leading byte offset (unused here)
  d |= (uint64_t)(1024 >> 4) << 32;          // stride byte offset
  d |= (uint64_t)1 << 46;                    // descriptor version
  d |= (uint64_t)2 << 61;                    // 128-byte swizzle
  return d;
}
template <int KIND>
__device__ __forceinline__ void mma(uint32_t dtmem, uint64_t ad, uint64_t bd, uint32_t idesc,
                                    uint32_t accum) {
  if constexpr (KIND == KIND_TF32X3) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(dtmem),
        "l"(ad), "l"(bd), "r"(idesc), "r"(accum)
        : "memory");
  } else if constexpr (KIND == KIND_BF16) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(dtmem),
        "l"(ad), "l"(bd), "r"(idesc), "r"(accum)
        : "memory");
  } else {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}" ::"r"(dtmem),
        "l"(ad), "l"(bd), "r"(idesc), "r"(accum)
        : "memory");
  }
}
__device__ __forceinline__ void mma_commit(uint32_t mbar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
      : "memory");
}
__device__ __forceinline__ void fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}

// Instruction descriptor: FP32 accumulator, K-major A and B, M = 128, N.
template <int KIND>
__host__ __device__ constexpr uint32_t idesc(int N) {
  return (1u << 4)                                  // D format F32
         | ((KIND == KIND_BF16 ? 1u : KIND == KIND_TF32X3 ? 2u : 0u) << 7)   // A: BF16 / TF32 / E4M3
         | ((KIND == KIND_BF16 ? 1u : KIND == KIND_TF32X3 ? 2u : 0u) << 10)  // B: same
         | ((uint32_t)(N >> 3) << 17)               // N / 8
         | ((uint32_t)(kBM >> 4) << 24);            // M / 16
}

// 32 lanes x N columns of FP32 from tensor memory.
template <int N>
__device__ __forceinline__ void tmem_ld(uint32_t taddr, float (&v)[N]) {
  uint32_t r[N];
  if constexpr (N == 16) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
        "%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
  } else if constexpr (N == 64) {
    tmem_ld<32>(taddr, *reinterpret_cast<float(*)[32]>(&v[0]));
    tmem_ld<32>(taddr + 32u, *reinterpret_cast<float(*)[32]>(&v[32]));
    return;
  } else {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
        "%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
          "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
          "=r"(r[31])
        : "r"(taddr));
  }
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < N; ++i) v[i] = __uint_as_float(r[i]);
}

// Stream-K range of CTA c over U units on G CTAs.
__host__ __device__ __forceinline__ int64_t unit_begin(int64_t U, int G, int c) {
  return (U * c) / G;
}

}  // namespace tc
}  // namespace ccg
