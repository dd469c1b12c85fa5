// ccg_lowp.cu -- low-precision block product W = A_lp D (Table 1, row 1) on
// the 5th-generation tensor cores, for the mixed-precision solver.
//
// A is stored once in BF16, or in FP8 E4M3 with one FP32 scale per row
// (A_ij ~= s_i q_ij).  The agents' block D is fed as BF16, or, next to an FP8
// A, as a pair of E4M3 blocks hi + lo with one scale per column
// (D_kj ~= sigma_j (hi_kj + lo_kj)), which keeps D to about BF16 accuracy
// without converting A.  Products accumulate in FP32 in tensor memory:
//
//   W_ij = s_i sigma_j sum_k q_ik (hi_kj + lo_kj)      (FP8)
//   W_ij = sum_k bf16(A_ik) bf16(D_kj)                 (BF16)
//
// Kernel shape (one CTA per SM, 192 threads):
//   warp 0    TMA producer: 128 x 128-byte tiles of A and the matching
//             N x 128-byte tile of D^T into a 6-stage ring (128-byte swizzle)
//   warp 1    tcgen05.mma issuer (M = 128, N = 16 or 32, FP32 accumulators in
//             TMEM, double-buffered so the epilogue overlaps the next tile)
//   warps 2-5 epilogue: tcgen05.ld of the 128 x N accumulator, FP32 partial
//             tile to global memory
// Work is split stream-K: the T x KC (row tile, k-chunk) units are divided
// evenly over the CTAs in tile-major order, so every SM streams the same
// number of A bytes.  A second kernel sums, for each row, the partial tiles of
// the CTAs that touched its tile, in CTA order (deterministic), and applies the
// scales.  Every mbarrier wait gives up after a time limit and sets an error
// flag; the kernel then drains its own copies and MMAs and frees TMEM.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "ccg_lowp.h"
#include "ccg_tc.cuh"

namespace ccg {
namespace lp {
namespace {

using namespace ccg::tc;
constexpr int kThreadsLp = 192;

// ---- the block-product kernel ----------------------------------------------
template <int KIND, int NP>
__global__ void __launch_bounds__(kThreadsLp, 1)
    lp_apass_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                    const __grid_constant__ LpRun run) {
  constexpr int NB = (KIND == KIND_FP8) ? 2 * NP : NP;  // B rows per stage (hi + lo for FP8)
  constexpr int kTileBBytes = NB * kRowBytes;
  constexpr int kStageBytes = kTileABytes + kTileBBytes;
  constexpr int NM = NB;  // one MMA covers hi and lo rows; the epilogue adds the halves
  constexpr uint32_t kIdesc = idesc<KIND>(NM);
  constexpr int kTmemCols = (2 * NM < 32) ? 32 : 2 * NM;  // two accumulator buffers

  extern __shared__ __align__(1024) uint8_t smem_raw[];
  // 1024-byte alignment for the swizzled tiles
  uint8_t* smem = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* sA = smem;
  uint8_t* sB = smem + kStages * kTileABytes;
  uint64_t* bars = reinterpret_cast<uint64_t*>(sB + kStages * kTileBBytes);
  uint64_t* full = bars;                 // [kStages]
  uint64_t* empty = bars + kStages;      // [kStages]
  uint64_t* accf = bars + 2 * kStages;   // [2]
  uint64_t* acce = bars + 2 * kStages + 2;  // [2]
  uint64_t* drain = bars + 2 * kStages + 4;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * kStages + 5);

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const int G = gridDim.x;
  const int c = blockIdx.x;
  const int64_t U = run.units;
  const int kc = run.kc;
  const int64_t u0 = unit_begin(U, G, c);
  const int64_t u1 = unit_begin(U, G, c + 1);
  int* err = run.error;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(smem_u32(&full[s]), 1);
      mbar_init(smem_u32(&empty[s]), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(smem_u32(&accf[b]), 1);
      mbar_init(smem_u32(&acce[b]), 4);
    }
    mbar_init(smem_u32(drain), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    // ---------------- TMA producer ----------------
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      int64_t u_issued = u0;
      const uint64_t pol_a = l2_policy_evict_first(), pol_b = l2_policy_evict_last();
      for (int64_t u = u0; u < u1; ++u) {
        if (!mbar_wait(smem_u32(&empty[stage]), phase ^ 1u, run.timeout_ns, err)) break;
        u_issued = u + 1;
        const int t = (int)(u / kc);
        const int k = (int)(u % kc);
        const uint32_t fb = smem_u32(&full[stage]);
        mbar_expect_tx(fb, kStageBytes);
        tma_load_2d_hint(smem_u32(sA + stage * kTileABytes), &tmA, k * run.k_elems, t * kBM, fb,
                         pol_a);
        tma_load_2d_hint(smem_u32(sB + stage * kTileBBytes), &tmB, k * run.k_elems, 0, fb, pol_b);
        if (++stage == kStages) { stage = 0; phase ^= 1u; }
      }
      // drain: the last copy issued on every stage has landed before the CTA
      // may exit (immediate when the MMA warp already consumed it)
      const int64_t issued = u_issued - u0;
      for (int s2 = 0; s2 < kStages && s2 < issued; ++s2) {
        const int64_t last = u0 + issued - 1 - s2;             // most recent issue
        const int st = (int)((last - u0) % kStages);
        const uint32_t ph = (uint32_t)(((last - u0) / kStages) & 1);
        mbar_wait(smem_u32(&full[st]), ph, run.timeout_ns, err);
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      int seg = 0;
      bool ok = true;
      bool issued_any = false;
      for (int64_t u = u0; u < u1 && ok; ++u) {
        const int k = (int)(u % kc);
        const bool first = (u == u0) || (k == 0);
        const bool last = (u == u1 - 1) || (k == kc - 1);
        const int b = seg & 1;
        if (first) {
          ok = mbar_wait(smem_u32(&acce[b]), (((uint32_t)seg >> 1) & 1u) ^ 1u, run.timeout_ns, err);
          if (!ok) break;
          fence_after();
        }
        ok = mbar_wait(smem_u32(&full[stage]), phase, run.timeout_ns, err);
        if (!ok) break;
        fence_after();
        const uint32_t dt = tmem + (uint32_t)(b * NM);
        const uint64_t ad = sdesc(smem_u32(sA + stage * kTileABytes));
        const uint64_t bd = sdesc(smem_u32(sB + stage * kTileBBytes));
#pragma unroll
        for (int kk = 0; kk < kRowBytes / 32; ++kk) {
          // advance 32 bytes along K inside the swizzle atom
          mma<KIND>(dt, ad + 2u * kk, bd + 2u * kk, kIdesc, (first && kk == 0) ? 0u : 1u);
        }
        issued_any = true;
        mma_commit(smem_u32(&empty[stage]));
        if (last) {
          mma_commit(smem_u32(&accf[b]));
          ++seg;
        }
        if (++stage == kStages) { stage = 0; phase ^= 1u; }
      }
      // all MMAs issued by this thread complete before TMEM is released
      if (issued_any) {
        mma_commit(smem_u32(drain));
        mbar_wait(smem_u32(drain), 0u, run.timeout_ns, err);
      }
    }
  } else {
    // ---------------- epilogue (warps 2..5) ----------------
    const int quad = warp & 3;  // TMEM lane quadrant this warp may access
    const int row = quad * 32 + lane;
    int seg = 0;
    if (u0 < u1) {
      const int t0 = (int)(u0 / kc);
      const int t1 = (int)((u1 - 1) / kc);
      for (int t = t0; t <= t1; ++t, ++seg) {
        const int b = seg & 1;
        if (!mbar_wait(smem_u32(&accf[b]), ((uint32_t)seg >> 1) & 1u, run.timeout_ns, err)) break;
        fence_after();
        float v[NM];
        tmem_ld<NM>(tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(b * NM), v);
        if constexpr (NM != NP) {
#pragma unroll
          for (int j = 0; j < NP; ++j) v[j] += v[NP + j];  // hi + lo halves
        }
        float* dst = run.part + ((size_t)(c + t) * kBM + row) * NP;
#pragma unroll
        for (int j = 0; j < NP; j += 4)
          *reinterpret_cast<float4*>(dst + j) = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
        fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_u32(&acce[b]));
      }
    }
  }
  fence_before();
  __syncthreads();
  fence_after();
  if (warp == 1) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(kTmemCols)
                 : "memory");
  }
}

// ---- fixup: sum partial tiles per row (CTA order), apply scales -----------
// One block of kBM threads per row tile: the CTA range of the tile is found
// once, then each thread sums its row's partial rows four columns at a time.
__global__ void lp_fixup_kernel(LpRun run, int NP, int q, double* __restrict__ W, int ldw) {
  __shared__ int s_c[2];
  const int64_t n = run.n;
  const int t = blockIdx.x;
  const int64_t U = run.units;
  const int G = run.ctas;
  if (threadIdx.x == 0) {
    const int64_t lo = (int64_t)t * run.kc, hi = lo + run.kc;
    // first CTA whose range ends after lo, last whose range starts before hi
    int c0 = (int)((lo * G) / U);
    while (c0 > 0 && unit_begin(U, G, c0) > lo) --c0;
    while (unit_begin(U, G, c0 + 1) <= lo) ++c0;
    int c1 = c0;
    while (c1 + 1 < G && unit_begin(U, G, c1 + 1) < hi) ++c1;
    s_c[0] = c0;
    s_c[1] = c1;
  }
  __syncthreads();
  const int r = threadIdx.x;
  const int64_t i = (int64_t)t * kBM + r;
  if (i >= n) return;
  const bool some_empty = U < G;  // with U >= G every CTA holds a unit
  const double rs = run.row_scale ? (double)run.row_scale[i] : 1.0;
  for (int j0 = 0; j0 < q; j0 += 4) {
    double sv[4] = {0.0, 0.0, 0.0, 0.0};
    for (int c = s_c[0]; c <= s_c[1]; ++c) {
      if (some_empty && unit_begin(U, G, c + 1) <= unit_begin(U, G, c)) continue;
      const float4 a = *reinterpret_cast<const float4*>(run.part + ((size_t)(c + t) * kBM + r) * NP + j0);
      sv[0] += (double)a.x;
      sv[1] += (double)a.y;
      sv[2] += (double)a.z;
      sv[3] += (double)a.w;
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int j = j0 + u;
      if (j >= q) break;
      double v = sv[u];
      if (run.row_scale) v *= rs;
      if (run.col_scale) v *= (double)run.col_scale[j];
      W[i * ldw + j] = v;
    }
  }
}

// ---- conversions -------------------------------------------------------------
// A (FP64, row-major, lda) -> BF16 rows of ldq elements.
__global__ void quant_bf16_kernel(const double* __restrict__ A, int64_t lda, int64_t n,
                                  __nv_bfloat16* __restrict__ Q, int64_t ldq) {
  const int64_t i = blockIdx.x;
  for (int64_t k = threadIdx.x; k < ldq; k += blockDim.x)
    Q[i * ldq + k] = (k < n) ? __double2bfloat16(A[i * lda + k]) : __double2bfloat16(0.0);
}

// A (FP64) -> FP32 rows of ldq elements (round to nearest).
__global__ void quant_f32_kernel(const double* __restrict__ A, int64_t lda, int64_t n,
                                 float* __restrict__ Q, int64_t ldq) {
  const int64_t i = blockIdx.x;
  for (int64_t k = threadIdx.x; k < ldq; k += blockDim.x)
    Q[i * ldq + k] = (k < n) ? (float)A[i * lda + k] : 0.f;
}

// A -> FP8 E4M3 with a per-row scale s_i = max_k |A_ik| / 448.
__global__ void quant_fp8_kernel(const double* __restrict__ A, int64_t lda, int64_t n,
                                 uint8_t* __restrict__ Q, int64_t ldq, float* __restrict__ scale) {
  __shared__ double red[32];
  const int64_t i = blockIdx.x;
  double m = 0.0;
  for (int64_t k = threadIdx.x; k < n; k += blockDim.x) m = fmax(m, fabs(A[i * lda + k]));
  for (int o = 16; o >= 1; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x < 32) {
    m = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0.0;
    for (int o = 16; o >= 1; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (threadIdx.x == 0) red[0] = m;
  }
  __syncthreads();
  const double s = red[0] > 0.0 ? red[0] / 448.0 : 1.0;
  const float sf = (float)s;
  if (threadIdx.x == 0) scale[i] = sf;
  const double inv = 1.0 / (double)sf;
  for (int64_t k = threadIdx.x; k < ldq; k += blockDim.x) {
    const double v = (k < n) ? A[i * lda + k] * inv : 0.0;
    Q[i * ldq + k] = (uint8_t)__nv_cvt_double_to_fp8(v, __NV_SATFINITE, __NV_E4M3);
  }
}

// Bound on the largest eigenvalue of a quantised copy A_q of A (Gershgorin):
// max_i [(1 + rel) sum_k |A_ik| + n absf max_k |A_ik|], where every entry of
// A_q satisfies |A_q,ik| <= (1 + rel) |A_ik| + absf max_k |A_ik| (rel: the
// format's relative rounding, absf: its absolute rounding below the normal
// range relative to the row scale).  Folded into *out with atomicMax on the
// bits of the non-negative double (they order as the values).  One block per
// row.
__global__ void eig_bound_kernel(const double* __restrict__ A, int64_t lda, int64_t n,
                                 double rel, double absf, unsigned long long* __restrict__ out) {
  __shared__ double red[2][32];
  const int64_t i = blockIdx.x;
  double t = 0.0, m = 0.0;
  for (int64_t k = threadIdx.x; k < n; k += blockDim.x) {
    const double a = fabs(A[i * lda + k]);
    t += a;
    m = fmax(m, a);
  }
  for (int o = 16; o >= 1; o >>= 1) {
    t += __shfl_xor_sync(0xffffffffu, t, o);
    m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = t;
    red[1][threadIdx.x >> 5] = m;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double r = 0.0, mx = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      r += red[0][w];
      mx = fmax(mx, red[1][w]);
    }
    // the sum of n non-negative terms is at most (1 + n 2^-52) too small
    const double b = ((1.0 + rel) * r + (double)n * absf * mx) * (1.0 + (double)n * 0x1.0p-51);
    atomicMax(out, (unsigned long long)__double_as_longlong(b));
  }
}

// A (FP64) -> kSlices FP8 slices without rounding error (the error-free
// splitting of Ozaki, Ogita, Oishi and Rump, "Error-free transformations of
// matrix multiplication by using fast routines of matrix multiplication and
// its applications", Numer. Algorithms 59, 2012, with 4-bit slices).  With e_i
// the binary exponent of the row's largest |A_ij| (so |A_ij| 2^-e_i < 1),
// x = A_ij 2^-e_i is written as sign(x) sum_s q_s 16^-(s+1) + r with the hex
// digits q_s in [0, 15] of |x| (taken from the significand bits, see
// slice_bits); the remainder |r| < 16^-kSlices is dropped.  sign(x) q_s is
// exact in E4M3, so the tensor cores multiply slices exactly.  Slice s of row
// i lands in row s * srows + i; scale[i] = 2^e_i.
__global__ void slice_fp64_kernel(const double* __restrict__ A, int64_t lda, int64_t n,
                                  uint8_t* __restrict__ Q, int64_t ldq, int64_t srows,
                                  float* __restrict__ scale) {
  __shared__ double red[32];
  const int64_t i = blockIdx.x;
  double m = 0.0;
  for (int64_t k = threadIdx.x; k < n; k += blockDim.x) m = fmax(m, fabs(A[i * lda + k]));
  for (int o = 16; o >= 1; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x < 32) {
    m = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0.0;
    for (int o = 16; o >= 1; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (threadIdx.x == 0) red[0] = m;
  }
  __syncthreads();
  int e = 0;
  if (red[0] > 0.0) frexp(red[0], &e);
  if (threadIdx.x == 0) scale[i] = ldexpf(1.f, e);
  for (int64_t k = threadIdx.x; k < n; k += blockDim.x) {
    uint32_t neg;
    const uint64_t X = slice_bits(A[i * lda + k], e, &neg);
#pragma unroll
    for (int sl = 0; sl < kSlices; ++sl)
      Q[((int64_t)sl * srows + i) * ldq + k] =
          (uint8_t)e4m3_digit((uint32_t)(X >> (52 - 4 * sl)) & 15u, neg);
  }
}

// Column max |V[:, j]| (for the FP8 column scales), as float bits.
__global__ void colmax_kernel(const double* __restrict__ V, int64_t n, int q,
                              unsigned int* __restrict__ out) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n * q) return;
  const int j = (int)(idx % q);
  const float a = (float)fabs(V[idx]);
  atomicMax(out + j, __float_as_uint(a));
}

// V (FP64, n x q row-major) -> operand rows (K contiguous, ldk elements):
// BF16: Vt[j][k] = bf16(V[k][j]); FP8: hi/lo E4M3 pair with column scale.
__global__ void convert_v_kernel(const double* __restrict__ V, int64_t n, int q, int NP,
                                 int kind, int64_t ldk, void* __restrict__ Vt,
                                 const unsigned int* __restrict__ cmax,
                                 float* __restrict__ col_scale) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y;
  if (k >= ldk) return;
  const double v = (k < n && j < q) ? V[k * q + j] : 0.0;
  if (kind == KIND_BF16) {
    reinterpret_cast<__nv_bfloat16*>(Vt)[(int64_t)j * ldk + k] = __double2bfloat16(v);
  } else {
    const float mx = (j < q) ? __uint_as_float(cmax[j]) : 0.f;
    const float sg = mx > 0.f ? mx / 448.f : 1.f;
    if (k == 0 && j < q) col_scale[j] = sg;
    const double x = v / (double)sg;
    const __nv_fp8_storage_t h = __nv_cvt_double_to_fp8(x, __NV_SATFINITE, __NV_E4M3);
    const double hv = (double)__half2float(__half(__nv_cvt_fp8_to_halfraw(h, __NV_E4M3)));
    const __nv_fp8_storage_t l = __nv_cvt_double_to_fp8(x - hv, __NV_SATFINITE, __NV_E4M3);
    uint8_t* o = reinterpret_cast<uint8_t*>(Vt);
    o[(int64_t)j * ldk + k] = (uint8_t)h;
    o[(int64_t)(NP + j) * ldk + k] = (uint8_t)l;
  }
}

template <int KIND, int NP>
size_t lp_smem_bytes() {
  constexpr int NB = (KIND == KIND_FP8) ? 2 * NP : NP;
  return 1024 + (size_t)kStages * (kTileABytes + NB * kRowBytes) + (2 * kStages + 6) * 8 + 64;
}

template <int KIND, int NP>
cudaError_t launch_apass_t(const CUtensorMap& tA, const CUtensorMap& tB, const LpRun& run,
                           cudaStream_t s) {
  const size_t smem = lp_smem_bytes<KIND, NP>();
  cudaError_t e = cudaFuncSetAttribute(lp_apass_kernel<KIND, NP>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  lp_apass_kernel<KIND, NP><<<run.ctas, kThreadsLp, smem, s>>>(tA, tB, run);
  return cudaGetLastError();
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

// 2-D tensor map over a rows x cols operand (K contiguous, ld elements), box
// of box_rows x 128 bytes, 128-byte swizzle.
bool make_map(CUtensorMap* m, const void* base, int kind, int64_t rows, int64_t cols,
              int64_t ld, int box_rows) {
  auto fn = encode_fn();
  if (!fn) return false;
  const int esz = (kind == KIND_BF16) ? 2 : (kind == KIND_TF32X3) ? 4 : 1;
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)(ld * esz)};
  cuuint32_t box[2] = {(cuuint32_t)(kRowBytes / esz), (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  const CUtensorMapDataType dt = kind == KIND_BF16    ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                 : kind == KIND_TF32X3 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                                       : CU_TENSOR_MAP_DATA_TYPE_UINT8;
  CUresult r = fn(m, dt,
                  2, const_cast<void*>(base), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

}  // namespace

bool make_tensor_map(CUtensorMap* m, const void* base, int kind, int64_t rows, int64_t cols,
                     int64_t ld, int box_rows) {
  return make_map(m, base, kind, rows, cols, ld, box_rows);
}

int64_t ld_elems(int64_t n) { return (n + 127) / 128 * 128; }

size_t part_floats(int64_t n, int ctas, int NP) {
  const int64_t T = (n + kBM - 1) / kBM;
  return (size_t)(ctas + T) * kBM * NP;
}

int64_t slice_rows(int64_t n) { return (n + kBM - 1) / kBM * kBM; }

cudaError_t eig_bound(int kind, const double* A, int64_t lda, int64_t n,
                      unsigned long long* out, cudaStream_t s) {
  // relative rounding of the format and its absolute rounding below the
  // normal range (FP8 E4M3 with row scale s_i = max/448: half the smallest
  // subnormal step, 2^-10 s_i < 2^-18 max)
  const double rel = kind == KIND_FP8 ? 0x1.0p-4 : kind == KIND_BF16 ? 0x1.0p-8 : 0x1.0p-20;
  const double absf = kind == KIND_FP8 ? 0x1.0p-18 : 0.0;
  cudaError_t e = cudaMemsetAsync(out, 0, sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  eig_bound_kernel<<<(unsigned)n, 256, 0, s>>>(A, lda, n, rel, absf, out);
  return cudaGetLastError();
}
static_assert(kSlicesHost == kSlices, "slice count");

cudaError_t quantize(int kind, const double* A, int64_t lda, int64_t n, void* Q, int64_t ldq,
                     float* row_scale, cudaStream_t s) {
  if (kind == KIND_SLICED) {
    // padding rows and columns of every slice stay zero
    const int64_t srows = slice_rows(n);
    cudaError_t e = cudaMemsetAsync(Q, 0, (size_t)kSlices * srows * ldq, s);
    if (e != cudaSuccess) return e;
    slice_fp64_kernel<<<(unsigned)n, 256, 0, s>>>(A, lda, n, reinterpret_cast<uint8_t*>(Q), ldq,
                                                   srows, row_scale);
    return cudaGetLastError();
  }
  if (kind == KIND_BF16)
    quant_bf16_kernel<<<(unsigned)n, 256, 0, s>>>(A, lda, n, reinterpret_cast<__nv_bfloat16*>(Q), ldq);
  else if (kind == KIND_TF32X3)
    quant_f32_kernel<<<(unsigned)n, 256, 0, s>>>(A, lda, n, reinterpret_cast<float*>(Q), ldq);
  else
    quant_fp8_kernel<<<(unsigned)n, 256, 0, s>>>(A, lda, n, reinterpret_cast<uint8_t*>(Q), ldq,
                                                  row_scale);
  return cudaGetLastError();
}

cudaError_t convert_operand(int kind, const double* V, int64_t n, int q, int NP, void* Vt,
                            int64_t ldk, unsigned int* cmax, float* col_scale, cudaStream_t s) {
  if (kind == KIND_FP8) {
    cudaMemsetAsync(cmax, 0, sizeof(unsigned int) * 32, s);
    const int64_t tot = n * q;
    colmax_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(V, n, q, cmax);
  }
  dim3 grid((unsigned)((ldk + 255) / 256), (unsigned)NP);
  convert_v_kernel<<<grid, 256, 0, s>>>(V, n, q, NP, kind, ldk, Vt, cmax, col_scale);
  return cudaGetLastError();
}

cudaError_t block_product(int kind, int NP, const void* Q, int64_t ldq, const void* Vt,
                          int64_t ldk, LpRun run, int q, double* W, cudaStream_t s,
                          cudaEvent_t ev0, cudaEvent_t ev1) {
  const int64_t n = run.n;
  const int k_elems = (kind == KIND_BF16) ? kRowBytes / 2 : kRowBytes;
  run.k_elems = k_elems;
  run.kc = (int)((n + k_elems - 1) / k_elems);
  const int64_t T = (n + kBM - 1) / kBM;
  run.units = T * run.kc;
  CUtensorMap tA, tB;
  const int NB = (kind == KIND_FP8) ? 2 * NP : NP;
  if (!make_map(&tA, Q, kind, n, n, ldq, kBM)) return cudaErrorInvalidValue;
  if (!make_map(&tB, Vt, kind, NB, n, ldk, NB)) return cudaErrorInvalidValue;
  if (ev0) cudaEventRecord(ev0, s);
  cudaError_t e;
  if (kind == KIND_BF16)
    e = (NP == 16) ? launch_apass_t<KIND_BF16, 16>(tA, tB, run, s)
                   : launch_apass_t<KIND_BF16, 32>(tA, tB, run, s);
  else
    e = (NP == 16) ? launch_apass_t<KIND_FP8, 16>(tA, tB, run, s)
                   : launch_apass_t<KIND_FP8, 32>(tA, tB, run, s);
  if (e != cudaSuccess) return e;
  lp_fixup_kernel<<<(unsigned)T, kBM, 0, s>>>(run, NP, q, W, q);
  if (ev1) cudaEventRecord(ev1, s);
  return cudaGetLastError();
}

}  // namespace lp
}  // namespace ccg
