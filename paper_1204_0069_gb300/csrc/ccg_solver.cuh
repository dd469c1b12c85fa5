// ccg_solver.cuh -- the persistent solver kernel for the cooperative conjugate
// gradient method (cCG, Algorithm 2 of arXiv:1204.0069) with the deflation of
// Algorithm 3 (mcCG) and the stopping rule of Algorithm 4.
//
// One cooperative launch runs a whole solve.  CTA c owns rows
// [c n / G, (c+1) n / G) of A, X, R, D and W = A D.  Each iteration is the
// sequence of Table 1 with its two exchange points, plus one barrier before
// the next block product:
//
//   A-pass   W = A D_k (own rows; A streamed once per iteration), and the
//            per-CTA partials of M = D'W, G = R'D           (Table 1, rows 1-3)
//   sync #1  cross-CTA sums of the partials (spread over all CTAs when there
//            are many), then in the last-arriving CTA the scaled Cholesky of
//            M with the rank test of Algorithm 3 and alpha_k
//   update   X += D alpha^T, R += W alpha^T (recurrence, proof of Thm. 2);
//            partials of H = R_{k+1}'W and ||R_{k+1} e_j||^2  (Table 1, rows 5-7)
//   sync #2  cross-CTA sums, then in the last-arriving CTA beta_k and the stop
//            test min_j ||R e_j|| <= tol ||b||
//   D-update D_{k+1} = R_{k+1} + D_k beta^T                  (Table 1, row 9)
//   barrier
//
// The p x p Grams and the norms are inner products that the method treats as
// exact (Sec. 4 works in exact arithmetic); they decide the matrix stepsizes
// and the stop test, so each lane sums its terms exactly in a long integer
// accumulator (ccg_xacc.h) and the lanes and CTAs are combined with
// error-free transformations (Dot2 arithmetic of Ogita, Rump and Oishi 2005:
// TwoSum for the running sum).  Every sum runs in an order
// fixed by the grid alone, so a solve is bitwise reproducible for a fixed
// grid.  (The inner solves of the mixed-precision path, whose operator is
// itself a rounded copy of A, accumulate their Grams in plain FP64.)  On
// GB300 a single SM retires about two FP64 operations per clock, so the
// serial steps keep their dependent chains short: sums over CTAs are warp
// trees, and large sets are spread over all CTAs.  Every wait on another CTA
// gives up
// after Params::timeout_ns and sets CCG_ERR_TIMEOUT; all CTAs then return.
#pragma once

#include <cstdint>
#include <type_traits>
#include <cuda_runtime.h>

#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include "ccg_internal.h"
#include "ccg_tc.cuh"
#include "ccg_xacc.h"

namespace ccg {
namespace {

// --------------------------------------------------------------------------
// Memory-model helpers
// --------------------------------------------------------------------------
__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_u32(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned atom_add_acqrel_u32(unsigned* p, unsigned v) {
  unsigned old;
  asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;"
               : "=r"(old) : "l"(p), "r"(v) : "memory");
  return old;
}
__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Cross-CTA data produced inside the launch is read through L2 only.
__device__ __forceinline__ double ldcg(const double* p) { return __ldcg(p); }
__device__ __forceinline__ int ldcg(const int* p) { return __ldcg(p); }

__device__ void set_error(DevState* st, int code, int where) {
  if (atomicCAS(&st->error, 0, code) == 0) st->err_where = where;
}

// Compensated accumulation (Dot2) on DSum pairs (ccg_xacc.h).  The
// intrinsics keep the compiler from contracting the error-free
// transformations into FMAs.
__device__ __forceinline__ void two_sum(double a, double b, double& s, double& e) {
  s = __dadd_rn(a, b);
  const double z = __dsub_rn(s, a);
  e = __dadd_rn(__dsub_rn(a, __dsub_rn(s, z)), __dsub_rn(b, z));
}
__device__ __forceinline__ void dsum_fma(DSum& t, double x, double y) {
  const double p = __dmul_rn(x, y);
  const double pe = fma(x, y, -p);  // exact product error
  double s, e;
  two_sum(t.hi, p, s, e);
  t.hi = s;
  t.lo = __dadd_rn(t.lo, __dadd_rn(pe, e));
}
__device__ __forceinline__ void dsum_add(DSum& t, double hi, double lo) {
  double s, e;
  two_sum(t.hi, hi, s, e);
  t.hi = s;
  t.lo = __dadd_rn(t.lo, __dadd_rn(lo, e));
}
// Warp-wide compensated sum in a fixed butterfly order; all lanes get it.
__device__ __forceinline__ DSum dsum_warp(DSum t) {
#pragma unroll
  for (int m = 16; m >= 1; m >>= 1) {
    const double oh = __shfl_xor_sync(0xffffffffu, t.hi, m);
    const double ol = __shfl_xor_sync(0xffffffffu, t.lo, m);
    // combine in lane order so both partners compute the same value
    const bool low = (threadIdx.x & m) == 0;
    DSum a = low ? t : DSum{oh, ol};
    const DSum b = low ? DSum{oh, ol} : t;
    dsum_add(a, b.hi, b.lo);
    t = a;
  }
  return t;
}

// --------------------------------------------------------------------------
// Grid synchronisation with an optional serial step.
//   grid_arrive: 1 = this CTA arrived last and must run the serial step and
//   then grid_release; 0 = released (serial step complete and visible);
//   -1 = an error is set or the wait timed out: leave the kernel.
// --------------------------------------------------------------------------
struct SyncShared {
  unsigned gen;
  int flag;
};

// Size of the group of CTAs solving one system and this CTA's rank in it.
__device__ __forceinline__ int grp_size(const Params& prm) {
  return prm.group_ctas ? prm.group_ctas : (int)gridDim.x;
}
__device__ __forceinline__ int grp_rank(const Params& prm) {
  return prm.group_ctas ? prm.group_rank : (int)blockIdx.x;
}

__device__ int grid_arrive(const Params& prm, SyncShared* ss) {
  __syncthreads();
  if (prm.expected_ctas == 1u) {
    // a group of one CTA: the CTA barrier is the whole synchronisation
    if (threadIdx.x == 0) ss->flag = 1;
    __syncthreads();
    return 1;
  }
  if (threadIdx.x == 0) {
    DevState* st = prm.st;
    __threadfence();
    const unsigned gen = ld_acquire_u32(&st->bar_gen);
    const unsigned arrived = atom_add_acqrel_u32(&st->bar_count, 1u);
    int flag;
    if (arrived == prm.expected_ctas - 1u) {
      flag = 1;
      __threadfence();
    } else {
      flag = 0;
      const unsigned long long t0 = globaltimer_ns();
      unsigned polls = 0;
      // tight spin on the generation word (one thread per CTA); the error
      // word and the time limit are looked at every 16th poll
      while (ld_acquire_u32(&st->bar_gen) == gen) {
        if ((++polls & 15u) != 0u) continue;
        if (*(volatile int*)&st->error != 0) { flag = -1; break; }
        if (globaltimer_ns() - t0 > (unsigned long long)prm.timeout_ns) {
          set_error(st, ST_ERR_TIMEOUT, 100);
          flag = -1;
          break;
        }
      }
      __threadfence();
    }
    if (flag == 0 && *(volatile int*)&st->error != 0) flag = -1;
    ss->gen = gen;
    ss->flag = flag;
  }
  __syncthreads();
  return ss->flag;
}

__device__ void grid_release(const Params& prm, SyncShared* ss) {
  __syncthreads();
  if (prm.expected_ctas == 1u) return;
  if (threadIdx.x == 0) {
    __threadfence();
    atomicExch(&prm.st->bar_count, 0u);
    st_release_u32(&prm.st->bar_gen, ss->gen + 1u);
  }
  __syncthreads();
}

// Error state broadcast to the whole CTA (one read, uniform decision).
__device__ __forceinline__ bool cta_error(const DevState* st, int* s_err) {
  __syncthreads();
  if (threadIdx.x == 0) *s_err = *(volatile const int*)&st->error;
  __syncthreads();
  return *s_err != 0;
}

// Plain barrier; false = leave the kernel.  A released CTA has read the
// error word after its wake-up (grid_arrive); only the releasing CTA reads it
// again.
__device__ bool grid_barrier(const Params& prm, SyncShared* ss, int* s_err) {
  const int f = grid_arrive(prm, ss);
  if (f < 0) return false;
  if (f == 0) return true;
  grid_release(prm, ss);
  return !cta_error(prm.st, s_err);
}

// --------------------------------------------------------------------------
// Block product tile shapes.  Lanes of a warp split the k range of one row
// of A (two consecutive k per lane, 16-byte loads); a k-chunk of the operand
// V (BK x P) is staged transposed in shared memory and shared by the CTA's 8
// rows of the pass.  The next chunk's A values (registers) and V values
// (registers, then the second shared buffer) are fetched while the current
// chunk is multiplied, so each chunk costs one CTA barrier and the memory
// latency hides behind the FP64 pipe.  NS independent accumulator sets keep
// >= 8 FMA chains per lane.
// --------------------------------------------------------------------------
template <int P>
struct Tile {
  static constexpr int BK = (2048 / P < 512) ? 2048 / P : 512;
  static constexpr int VSTR = BK + 2;          // padded shared row (16-byte aligned)
  static constexpr int NS = (P >= 8) ? 1 : 8 / P;
  static constexpr int NLD = BK / 64;          // double2 loads of A per lane per chunk
  static constexpr int NV = BK * P / kThreads; // staged V values per thread per chunk
  static constexpr int LOGP = (P == 1) ? 0 : (P == 2) ? 1 : (P == 4) ? 2
                             : (P == 8) ? 3 : (P == 16) ? 4 : 5;
  static_assert(NV >= 1 && NV * kThreads == BK * P, "chunk must tile the CTA");
};

// Reduce-scatter over the 32 lanes: afterwards v[0] holds, in every lane, the
// full sum of column (lane >> (5 - log2 P)).
template <int CNT, int M>
struct ReduceScatter {
  __device__ __forceinline__ static void run(double* v, int lane) {
    if constexpr (CNT > 1) {
      constexpr int H = CNT / 2;
      const bool up = (lane & M) != 0;
#pragma unroll
      for (int i = 0; i < H; ++i) {
        const double send = up ? v[i] : v[i + H];
        const double keep = up ? v[i + H] : v[i];
        v[i] = keep + __shfl_xor_sync(0xffffffffu, send, M);
      }
      if constexpr (M > 1) ReduceScatter<H, M / 2>::run(v, lane);
    } else {
      v[0] += __shfl_xor_sync(0xffffffffu, v[0], M);
      if constexpr (M > 1) ReduceScatter<1, M / 2>::run(v, lane);
    }
  }
};

template <int P>
__device__ __forceinline__ void load_v_chunk(const double* __restrict__ V, int ldv, int coff,
                                             int pk, int64_t n, int64_t k0, double (&v)[Tile<P>::NV]) {
#pragma unroll
  for (int t = 0; t < Tile<P>::NV; ++t) {
    const int idx = threadIdx.x + t * kThreads;
    const int kk = idx >> Tile<P>::LOGP;
    const int c = idx & (P - 1);
    const int64_t k = k0 + kk;
    v[t] = (c < pk && k < n) ? ldcg(V + k * ldv + coff + c) : 0.0;
  }
}

template <int P>
__device__ __forceinline__ void store_v_chunk(double* Vb, const double (&v)[Tile<P>::NV]) {
#pragma unroll
  for (int t = 0; t < Tile<P>::NV; ++t) {
    const int idx = threadIdx.x + t * kThreads;
    Vb[(idx & (P - 1)) * Tile<P>::VSTR + (idx >> Tile<P>::LOGP)] = v[t];
  }
}

template <int P, bool VEC>
__device__ __forceinline__ void load_a_chunk(const double* Arow, int64_t n, int64_t k0, int lane,
                                             bool valid, double2 (&a)[Tile<P>::NLD]) {
#pragma unroll
  for (int j = 0; j < Tile<P>::NLD; ++j) {
    const int64_t k = k0 + j * 64 + 2 * lane;
    double2 v = make_double2(0.0, 0.0);
    if (valid) {
      if (VEC && k + 1 < n) {
        v = __ldcs(reinterpret_cast<const double2*>(Arow + k));
      } else {
        if (k < n) v.x = __ldcs(Arow + k);
        if (k + 1 < n) v.y = __ldcs(Arow + k + 1);
      }
    }
    a[j] = v;
  }
}

// Narrow block product (few operand columns, which fit in L1): every warp
// streams its own rows with U independent 16-byte loads in flight per lane
// (a step covers 64 U columns) and reads the operand through L1; no CTA
// barrier per k-chunk.  The operand was written before the last grid barrier,
// whose acquire makes L1 reads fresh.  U = 2 suits short rows (small batched
// systems), where wider steps would be mostly masked lanes.
template <int P, bool VEC, int U = 8>
__device__ void apass_narrow(const Params& prm, const double* __restrict__ V, int ldv,
                             int coff, int pk, double* __restrict__ Y, int ldy,
                             bool sub_b, int64_t r0, int64_t r1) {
  constexpr int NS = 4;                 // accumulator sets
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int64_t n = prm.n;
  const int64_t lda = prm.lda;
  const int64_t nr = r1 - r0;
  const int64_t w0 = r0 + (nr * warp) / kWarps;
  const int64_t w1 = r0 + (nr * (warp + 1)) / kWarps;
  for (int64_t row = w0; row < w1; ++row) {
    const double* Arow = prm.A + row * lda;
    double acc[NS][P];
#pragma unroll
    for (int s = 0; s < NS; ++s)
#pragma unroll
      for (int c = 0; c < P; ++c) acc[s][c] = 0.0;
    for (int64_t k0 = 0; k0 < n; k0 += 64 * U) {
      double2 a[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int64_t k = k0 + 64 * u + 2 * lane;
        double2 t = make_double2(0.0, 0.0);
        if (VEC && k + 1 < n) {
          t = __ldcs(reinterpret_cast<const double2*>(Arow + k));
        } else {
          if (k < n) t.x = __ldcs(Arow + k);
          if (k + 1 < n) t.y = __ldcs(Arow + k + 1);
        }
        a[u] = t;
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int64_t k = k0 + 64 * u + 2 * lane;
#pragma unroll
        for (int c = 0; c < P; ++c) {
          const bool in0 = c < pk && k < n, in1 = c < pk && k + 1 < n;
          const double vx = in0 ? __ldca(V + k * ldv + coff + c) : 0.0;
          const double vy = in1 ? __ldca(V + (k + 1) * ldv + coff + c) : 0.0;
          acc[(2 * u) % NS][c] = fma(a[u].x, vx, acc[(2 * u) % NS][c]);
          acc[(2 * u + 1) % NS][c] = fma(a[u].y, vy, acc[(2 * u + 1) % NS][c]);
        }
      }
    }
    double tot[P];
#pragma unroll
    for (int c = 0; c < P; ++c) tot[c] = (acc[0][c] + acc[1][c]) + (acc[2][c] + acc[3][c]);
    ReduceScatter<P, 16>::run(tot, lane);
    const int c = lane >> (5 - Tile<P>::LOGP);
    const bool owner = (lane & ((32 >> Tile<P>::LOGP) - 1)) == 0;
    if (owner && c < pk) {
      double y = tot[0];
      if (sub_b) y -= prm.b[row];
      Y[row * ldy + c] = y;
    }
  }
  __syncthreads();
}

// Y[row, c] = sum_k A[row, k] V[k, coff + c] (- b[row]) for the rows
// [r0, r1) and c < pk.  Vs: shared scratch of 2 * P * VSTR doubles.
// VARIANTS (the batched kernels only): prm.apass_variant, chosen per size
// bucket by the host's autotuner, selects 0 tiled (narrow with 8 loads per
// step for P <= 2), 1 narrow with 8 loads per step, 2 narrow with 2 loads.
template <int P, bool VEC, bool VARIANTS = false>
__device__ void apass(const Params& prm, const double* __restrict__ V, int ldv,
                      int coff, int pk, double* __restrict__ Y, int ldy,
                      bool sub_b, int64_t r0, int64_t r1, double* Vs) {
  if constexpr (P <= 2) {
    if (VARIANTS && prm.apass_variant == 2)
      apass_narrow<P, VEC, 2>(prm, V, ldv, coff, pk, Y, ldy, sub_b, r0, r1);
    else
      apass_narrow<P, VEC, 8>(prm, V, ldv, coff, pk, Y, ldy, sub_b, r0, r1);
    return;
  } else if constexpr (VARIANTS && P <= 8) {
    if (prm.apass_variant == 1) {
      apass_narrow<P, VEC, 8>(prm, V, ldv, coff, pk, Y, ldy, sub_b, r0, r1);
      return;
    }
    if (prm.apass_variant == 2) {
      apass_narrow<P, VEC, 2>(prm, V, ldv, coff, pk, Y, ldy, sub_b, r0, r1);
      return;
    }
  }
  using T = Tile<P>;
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int64_t n = prm.n;
  const int64_t lda = prm.lda;
  const int64_t nr = r1 - r0;
  const int64_t w0 = r0 + (nr * warp) / kWarps;
  const int64_t w1 = r0 + (nr * (warp + 1)) / kWarps;
  const int64_t passes = (nr + kWarps - 1) / kWarps;
  const int64_t nch = (n + T::BK - 1) / T::BK;
  const double* __restrict__ A = prm.A;

  for (int64_t ps = 0; ps < passes; ++ps) {
    const int64_t row = w0 + ps;
    const bool valid = row < w1;
    const double* Arow = A + (valid ? row : r0) * lda;
    double acc[T::NS][P];
#pragma unroll
    for (int s = 0; s < T::NS; ++s)
#pragma unroll
      for (int c = 0; c < P; ++c) acc[s][c] = 0.0;

    double vreg[T::NV];
    double2 acur[T::NLD], anxt[T::NLD];
    load_v_chunk<P>(V, ldv, coff, pk, n, 0, vreg);
    load_a_chunk<P, VEC>(Arow, n, 0, lane, valid, acur);
    store_v_chunk<P>(Vs, vreg);
    __syncthreads();
    for (int64_t ch = 0; ch < nch; ++ch) {
      const bool more = ch + 1 < nch;
      if (more) {
        load_v_chunk<P>(V, ldv, coff, pk, n, (ch + 1) * T::BK, vreg);
        load_a_chunk<P, VEC>(Arow, n, (ch + 1) * T::BK, lane, valid, anxt);
      }
      const double* Vb = Vs + (ch & 1) * (P * T::VSTR);
      if (valid) {
#pragma unroll
        for (int j = 0; j < T::NLD; ++j) {
          const int kk = j * 64 + 2 * lane;
#pragma unroll
          for (int c = 0; c < P; ++c) {
            const double2 v = *reinterpret_cast<const double2*>(Vb + c * T::VSTR + kk);
            acc[(2 * j) % T::NS][c] = fma(acur[j].x, v.x, acc[(2 * j) % T::NS][c]);
            acc[(2 * j + 1) % T::NS][c] = fma(acur[j].y, v.y, acc[(2 * j + 1) % T::NS][c]);
          }
        }
      }
      if (more) store_v_chunk<P>(Vs + ((ch + 1) & 1) * (P * T::VSTR), vreg);
      __syncthreads();
#pragma unroll
      for (int j = 0; j < T::NLD; ++j) acur[j] = anxt[j];
    }
    double tot[P];
#pragma unroll
    for (int c = 0; c < P; ++c) {
      double t = acc[0][c];
#pragma unroll
      for (int s = 1; s < T::NS; ++s) t += acc[s][c];
      tot[c] = t;
    }
    ReduceScatter<P, 16>::run(tot, lane);
    const int c = lane >> (5 - T::LOGP);
    const bool owner = (lane & ((32 >> T::LOGP) - 1)) == 0;
    if (valid && owner && c < pk) {
      double y = tot[0];
      if (sub_b) y -= prm.b[row];
      Y[row * ldy + c] = y;
    }
  }
  __syncthreads();
}

// Per-CTA partial Grams over the rows [r0, r1) of blocks with leading
// dimension ld:  out[g0 + a*kMaxP + c] = sum_i U0[i,a] V0[i,c]  (U0 != NULL)
//                out[g1 + a*kMaxP + c] = sum_i U1[i,a] V1[i,c]  (U1 != NULL)
//                out[kSlotVec + a]    = sum_i S[i,a]^2          (S != NULL)
// Each entry is summed by a group of T lanes (T = 32 for a few entries, 1
// when they fill the CTA): lane q of the group takes rows r0 + q, r0 + q + T,
// ... in order, then the group combines in a fixed butterfly.  COMP: each
// lane's sum exact in a long accumulator, the group's in Dot2 arithmetic (hi
// at [slot], lo at [kPartHalf + slot]); otherwise a plain FP64 sum (lo 0).
template <bool COMP>
__device__ __forceinline__ void grp_combine(DSum& t, int T) {
  for (int m = T >> 1; m >= 1; m >>= 1) {
    const double oh = __shfl_xor_sync(0xffffffffu, t.hi, m);
    if constexpr (COMP) {
      const double ol = __shfl_xor_sync(0xffffffffu, t.lo, m);
      const bool low = (threadIdx.x & m) == 0;
      DSum a = low ? t : DSum{oh, ol};
      const DSum b = low ? DSum{oh, ol} : t;
      dsum_add(a, b.hi, b.lo);
      t = a;
    } else {
      t.hi = t.hi + oh;
    }
  }
}

template <bool COMP>
__device__ void partial_grams(const double* U0, const double* V0, const double* U1,
                              const double* V1, const double* S, int ld, int pk,
                              int64_t r0, int64_t r1, double* out, double* stage = nullptr,
                              int stage_doubles = 0) {
  const int sq = pk * pk;
  const int n0 = U0 ? sq : 0, n1 = U1 ? sq : 0, n2 = S ? pk : 0;
  const int E = n0 + n1 + n2;
  int T = 1;
  while (T < 32 && E * T * 2 <= kThreads) T <<= 1;
  const int groups = kThreads / T;
  const int gi = threadIdx.x / T, q = threadIdx.x % T;
  // When they fit, the CTA's rows of the operand blocks (first pk columns)
  // are read once, coalesced, into shared memory (U0 V0 U1 V1 S in order).
  // The exact sums stage each value decoded for the accumulator (one word of
  // significand and sign, a 16-bit exponent): every value enters pk products.
  const int64_t nr = r1 - r0;
  const int64_t blk = nr * pk;
  const int nblk = (U0 ? 2 : 0) + (U1 ? 2 : 0) + (S ? 1 : 0);
  constexpr int kStageBytesPer = COMP ? 10 : 8;
  const bool staged =
      stage != nullptr && nblk * blk * kStageBytesPer <= (int64_t)stage_doubles * 8;
  unsigned long long* st_m = reinterpret_cast<unsigned long long*>(stage);
  short* st_e = staged ? reinterpret_cast<short*>(st_m + nblk * blk) : nullptr;
  const int oU1 = U0 ? 2 * (int)blk : 0;
  const int oS = oU1 + (U1 ? 2 * (int)blk : 0);
  if (staged) {
    // all blocks in one pass, eight loads in flight per thread
    const int tot = nblk * (int)blk;
    for (int g0 = threadIdx.x; g0 < tot; g0 += 8 * kThreads) {
      double v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int g = g0 + u * kThreads;
        v[u] = 0.0;
        if (g < tot) {
          int b = g / (int)blk;
          const int idx = g - b * (int)blk;
          const double* B = S;
          if (U0 && b < 2) B = b == 0 ? U0 : V0;
          else if (U1 && (b -= U0 ? 2 : 0) < 2) B = b == 0 ? U1 : V1;
          const int rr = idx / pk;
          v[u] = ldcg(B + (r0 + rr) * ld + (idx - rr * pk));
        }
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int g = g0 + u * kThreads;
        if (g < tot) {
          if constexpr (COMP) {
            int e;
            xacc_decode(v[u], st_m[g], e);
            st_e[g] = (short)e;
          } else {
            stage[g] = v[u];
          }
        }
      }
    }
    __syncthreads();
  }
  for (int base = 0; base < E; base += groups) {  // same trip count in every warp
    const int e = base + gi;
    const bool act = e < E;
    const double* U = S;
    const double* Vv = S;
    int slot = 0, a = 0, c = 0;
    if (act) {
      if (e < n0) {
        U = U0; Vv = V0; a = e / pk; c = e - a * pk; slot = kSlotGram0 + a * kMaxP + c;
      } else if (e < n0 + n1) {
        const int f = e - n0;
        U = U1; Vv = V1; a = f / pk; c = f - a * pk; slot = kSlotGram1 + a * kMaxP + c;
      } else {
        a = c = e - n0 - n1; slot = kSlotVec + a;
      }
    }
    DSum t{0.0, 0.0};
    if (act && staged) {
      const int ou = e < n0 ? 0 : e < n0 + n1 ? oU1 : oS;
      const int ov = e < n0 + n1 ? ou + (int)blk : oS;
      if constexpr (COMP) {
        const unsigned long long* Um = st_m + ou + a;
        const unsigned long long* Vm = st_m + ov + c;
        const short* Ue = st_e + ou + a;
        const short* Ve = st_e + ov + c;
        XAcc x;
        xacc_init(x);
        int K = 2;  // anchor: the largest exponent sum of the entry's terms
#pragma unroll 8
        for (int rr = q; rr < (int)nr; rr += T) K = max(K, (int)Ue[rr * pk] + (int)Ve[rr * pk]);
        x.K = K;
#pragma unroll 4
        for (int rr = q; rr < (int)nr; rr += T)
          xacc_fma_kd(x, Um[rr * pk], Vm[rr * pk], (int)Ue[rr * pk] + (int)Ve[rr * pk]);
        t = xacc_value(x);
      } else {
        const double* Us = stage + ou + a;
        const double* Vs = stage + ov + c;
#pragma unroll 4
        for (int rr = q; rr < (int)nr; rr += T) t.hi = fma(Us[rr * pk], Vs[rr * pk], t.hi);
      }
    } else if (act) {
      XAcc x;
      xacc_init(x);
      int64_t i = r0 + q;
      // blocks of 8 of this lane's rows: 16 independent loads in flight, then
      // the sum in row order
      for (; i + 7 * T < r1; i += 8 * T) {
        double u[8], v[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          u[k] = ldcg(U + (i + k * T) * ld + a);
          v[k] = ldcg(Vv + (i + k * T) * ld + c);
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          if constexpr (COMP) xacc_fma(x, u[k], v[k]);
          else t.hi = fma(u[k], v[k], t.hi);
        }
      }
      for (; i < r1; i += T) {
        const double uu = ldcg(U + i * ld + a), vv = ldcg(Vv + i * ld + c);
        if constexpr (COMP) xacc_fma(x, uu, vv);
        else t.hi = fma(uu, vv, t.hi);
      }
      if constexpr (COMP) t = xacc_value(x);
    }
    grp_combine<COMP>(t, T);
    if (act && q == 0) {
      out[slot] = t.hi;
      out[kPartHalf + slot] = COMP ? t.lo : 0.0;
    }
  }
  if (staged) __syncthreads();  // the staging area is shared scratch
}

// Per-CTA compensated sum of squares of x[i * ld] over the rows [r0, r1)
// by warp 0, into `slot` (default: the scalar slot).
__device__ void partial_sumsq(const double* x, int ld, int64_t r0, int64_t r1, double* out,
                              int slot = kSlotScalar) {
  if (threadIdx.x < 32) {
    DSum t{0.0, 0.0};
    for (int64_t i = r0 + threadIdx.x; i < r1; i += 32) {
      const double v = ldcg(x + i * ld);
      dsum_fma(t, v, v);
    }
    t = dsum_warp(t);
    if (threadIdx.x == 0) {
      out[slot] = t.hi;
      out[kPartHalf + slot] = t.lo;
    }
  }
}

// --------------------------------------------------------------------------
// Serial steps (run by the last-arriving CTA only).
// --------------------------------------------------------------------------
constexpr int kLd = kMaxP + 1;  // padded stride of the p x p smem matrices
struct SerialSmem {
  double m[kMaxP * kLd];
  double g[kMaxP * kLd];
  double l[kMaxP * kLd];
  double y[kMaxP * kLd];
  double sc[kMaxP];
  double s2[kMaxP];
  double sv[kMaxP];
  int keep[kMaxP];
  int flag[4];
  int chol_m;
  int chol_fail;
};
// Every kernel's dynamic shared memory holds a SerialSmem; outside the serial
// steps the Gram partials use it to stage their operand rows.
constexpr int kStageDoubles = (int)(sizeof(SerialSmem) / sizeof(double));

// Cross-CTA sums.  A serial step needs the group's sum of some slot entries
// ("reduction set").  Each entry is summed by one warp: lane l takes the
// partials of CTAs l, l+32, ... in order (compensated), the lanes combine in
// the fixed butterfly of dsum_warp, and the rounded sum goes to st->red at the
// entry's slot offset.  The result of an entry does not depend on which warp
// or CTA sums it.  Small sets are summed by the serial CTA itself; larger
// ones are spread over the warps of every CTA of the group between two grid
// barriers, so no single SM carries E x G compensated additions.
enum RedSet : int {
  RED_M_G = 0,   // Gram0 and Gram1, q x q each
  RED_H_S = 1,   // Gram0 (q x q) and the vector slot (q)
  RED_S = 2,     // vector slot (q)
  RED_SCALAR = 3,
  RED_B_R = 4    // vector slot entry 0 and the scalar slot
};
constexpr int kRedLocalMax = 16;  // sets up to this size stay in the serial CTA

__device__ __forceinline__ int red_count(int set, int q) {
  switch (set) {
    case RED_M_G: return 2 * q * q;
    case RED_H_S: return q * q + q;
    case RED_S: return q;
    case RED_SCALAR: return 1;
    default: return 2;
  }
}

__device__ __forceinline__ int red_slot(int set, int q, int e) {
  const int sq = q * q;
  switch (set) {
    case RED_M_G: {
      const int f = e < sq ? e : e - sq;
      const int a = f / q;
      return (e < sq ? kSlotGram0 : kSlotGram1) + a * kMaxP + (f - a * q);
    }
    case RED_H_S: {
      if (e >= sq) return kSlotVec + (e - sq);
      const int a = e / q;
      return kSlotGram0 + a * kMaxP + (e - a * q);
    }
    case RED_S: return kSlotVec + e;
    case RED_SCALAR: return kSlotScalar;
    default: return e == 0 ? kSlotVec : kSlotScalar;
  }
}

// The butterfly skips the levels whose partner lanes hold no partial (G <= 16
// leaves lanes >= G empty; adding their zeros is exact), so lane 0's sum is
// the same as with all five levels.  The result is valid in lane 0.
template <bool COMP>
__device__ __forceinline__ double warp_sum_parts(const Params& prm, int off) {
  const int G = grp_size(prm);
  const int lane = threadIdx.x & 31;
  DSum t{0.0, 0.0};
  int g0 = 0;
  // up to 8 partials per lane with all loads in flight, then summed in order
  for (; g0 < G; g0 += 8 * 32) {
    double h[8], l[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int g = g0 + lane + 32 * k;
      const double* pp = prm.part + (size_t)g * kPartStride;
      h[k] = g < G ? ldcg(pp + off) : 0.0;
      l[k] = g < G ? ldcg(pp + kPartHalf + off) : 0.0;
    }
#pragma unroll
    for (int k = 0; k < 8; ++k)
      if (g0 + lane + 32 * k < G) {
        if constexpr (COMP) dsum_add(t, h[k], l[k]);
        else t.hi += h[k] + l[k];
      }
  }
  int top = 1;
  while (top < G && top < 32) top <<= 1;
  for (int m = top >> 1; m >= 1; m >>= 1) {
    const double oh = __shfl_xor_sync(0xffffffffu, t.hi, m);
    if constexpr (COMP) {
      const double ol = __shfl_xor_sync(0xffffffffu, t.lo, m);
      const bool low = (threadIdx.x & m) == 0;
      DSum a = low ? t : DSum{oh, ol};
      const DSum b = low ? DSum{oh, ol} : t;
      dsum_add(a, b.hi, b.lo);
      t = a;
    } else {
      t.hi += oh;
    }
  }
  return COMP ? __dadd_rn(t.hi, t.lo) : t.hi;
}

// Entries w0 + j * wstride (j = 0, 1, ...) of the set, one per warp of the
// first nw warps of this CTA.  COMP: compensated (FP64 solves); plain FP64
// sums for the inner solves of the mixed-precision paths, whose partials are
// plain sums already.
template <bool COMP>
__device__ void reduce_entries(const Params& prm, int set, int q, int w0, int wstride,
                               int nw = kWarps) {
  const int E = red_count(set, q);
  const int w = (int)(threadIdx.x >> 5);
  if (w >= nw) return;
  for (int e = w0 + w; e < E; e += wstride) {
    const int off = red_slot(set, q, e);
    const double v = warp_sum_parts<COMP>(prm, off);
    if ((threadIdx.x & 31) == 0) prm.st->red[off] = v;
  }
}

__device__ __forceinline__ double red_get(const DevState* st, int off) {
  return ldcg(&st->red[off]);
}

// Y <- L^{-T} L^{-1} Y for the m columns of y, L lower (m x m, m <= 32).
// One warp per right-hand side: lane a holds entry a of the column in a
// register; each solved entry is broadcast by a shuffle and applied to the
// remaining rows at once, so the dependent chain per row is a shuffle, a
// multiplication by the pivot reciprocal and an FMA.  The row loops stay
// rolled (a compact body the instruction cache keeps across rows).  rinv:
// shared scratch for the m pivot reciprocals.
__device__ void chol_solve_cols(const double* l, double* y, int m, double* rinv) {
  const int lane = threadIdx.x & 31;
  if ((int)threadIdx.x < m) rinv[threadIdx.x] = 1.0 / l[threadIdx.x * kLd + threadIdx.x];
  __syncthreads();
  for (int c = threadIdx.x >> 5; c < m; c += kWarps) {  // warp-uniform
    double v = lane < m ? y[lane * kLd + c] : 0.0;
#pragma unroll 1
    for (int u = 0; u < m; ++u) {
      const double yu = __shfl_sync(0xffffffffu, v, u) * rinv[u];
      const double lau = (lane > u && lane < m) ? l[lane * kLd + u] : 0.0;
      v = (lane == u) ? yu : (lane > u ? fma(-lau, yu, v) : v);
    }
#pragma unroll 1
    for (int u = m - 1; u >= 0; --u) {
      const double yu = __shfl_sync(0xffffffffu, v, u) * rinv[u];
      const double lua = (lane < u) ? l[u * kLd + lane] : 0.0;
      v = (lane == u) ? yu : (lane < u ? fma(-lua, yu, v) : v);
    }
    if (lane < m) y[lane * kLd + c] = v;
  }
  __syncthreads();
}

__device__ __forceinline__ bool finite(double v) { return isfinite(v); }

// Stop test on the residual norms s2 (squared), shared by the init, beta and
// replacement steps: sets s, jbest, relres_recur and the next ctrl.
__device__ void stop_test(const Params& prm, SerialSmem& S, int pk, int where) {
  DevState* st = prm.st;
  if (threadIdx.x < pk) {
    const double s = sqrt(S.s2[threadIdx.x]);
    S.sv[threadIdx.x] = s;
    st->s[threadIdx.x] = s;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    bool bad = false;
    int jmin = 0;
    for (int j = 0; j < pk; ++j) {
      const double s = S.sv[j];
      if (!finite(s)) bad = true;
      if (j > 0 && s < S.sv[jmin]) jmin = j;
    }
    if (bad) {
      set_error(st, ST_ERR_NUMERICAL, where);
    } else {
      const double smin = S.sv[jmin];
      const double bn = ldcg(&st->bnorm);
      const bool stop = smin <= prm.tol * bn;
      st->jbest = jmin;
      st->relres_recur = smin / bn;
      const bool done = stop || ldcg(&st->k) >= prm.maxit;
      if (done && prm.skip_true_check) {
        // inner solve: the recurrence residual decides (the caller checks the
        // true residual of its own, outer system)
        st->relres_true = smin / bn;
        st->result = stop ? ST_OK : ST_NOT_CONVERGED;
        st->ctrl = CTRL_FINISH;
      } else {
        st->ctrl = done ? CTRL_CHECK : CTRL_LOOP;
      }
    }
  }
  __syncthreads();
}

// Right-looking Cholesky of the unit-diagonal scaled M (lower triangle in
// S.l) by one warp: lane i updates row i of S.l in place, and the
// multipliers of column j are read back from shared memory.  The column loop
// stays rolled: the step runs once per iteration on a single warp, right
// after the product pass has filled the instruction cache with its own code,
// and a compact body is fetched once instead of once per column.  Columns are
// taken in agent order; a column whose pivot is below rank_tol is skipped
// (agent dropped, Algorithm 3), a pivot below -sqrt(rank_tol) means A is not
// SPD.  Leaves the factor in S.l, the kept columns in S.keep, their count in
// S.chol_m and 0 / 2 (not SPD) / 3 (NaN) in S.chol_fail.  Called by warp 0
// only.
template <bool FAST>
__device__ void warp_chol(const Params& prm, SerialSmem& S, int pk) {
  const int lane = threadIdx.x & 31;
  double* row = S.l + lane * kLd;
  const bool mine = lane < pk;
  const double neg_lim = -sqrt(prm.rank_tol);
  int m = 0, fail = 0;
#pragma unroll 1
  for (int j = 0; j < pk; ++j) {
    __syncwarp();
    const double d = S.l[j * kLd + j];
    int decision = 0;  // 0 keep, 1 drop, 2 not SPD, 3 NaN
    if (S.m[j * kLd + j] == 0.0) decision = 1;  // zero direction
    else if (!(d == d)) decision = 3;
    else if (d < neg_lim) decision = 2;
    else if (d < prm.rank_tol) decision = 1;
    if (decision >= 2) {
      fail = decision;
      break;
    }
    if (decision == 1) continue;
    double lij = 0.0;
    if constexpr (FAST) {
      // inner solves: one reciprocal square root per column (shorter
      // dependent chain; the refinement does not see the rounding)
      const double rj = rsqrt(d);
      if (lane == j) row[j] = d * rj;
      else if (lane > j && mine) row[j] = lij = row[j] * rj;
    } else {
      // square root and division as in the textbook factorisation: the
      // iteration count of an ill-conditioned solve follows the rounding of
      // the factor (a reciprocal square root moved it by 9 of 388 at
      // n = 8192, p = 8)
      const double ljj = sqrt(d);
      if (lane == j) row[j] = ljj;
      else if (lane > j && mine) row[j] = lij = row[j] / ljj;
    }
    __syncwarp();
    if (lane > j && mine) {
#pragma unroll 4
      for (int k = j + 1; k <= lane; ++k) row[k] = fma(-lij, S.l[k * kLd + j], row[k]);
    }
    if (lane == 0) S.keep[m] = j;
    ++m;
  }
  __syncwarp();
  if (lane == 0) {
    S.chol_m = m;
    S.chol_fail = fail;
  }
}

// alpha step: M, G -> rank test, factor, alpha_k^T (Algorithm 2 / 3).
template <int NB, bool FAST = false>
__device__ void serial_alpha(const Params& prm, SerialSmem& S) {
  DevState* st = prm.st;
  const int tid = threadIdx.x;
  const int pk = ldcg(&st->pk);
  const int sq = pk * pk;
  if (tid < 4) S.flag[tid] = 0;
  for (int e = tid; e < 2 * sq; e += kThreads) {
    const int f = e < sq ? e : e - sq;
    const int a = f / pk, c = f - a * pk;
    (e < sq ? S.m : S.g)[a * kLd + c] = red_get(st, red_slot(RED_M_G, pk, e));
  }
  __syncthreads();
  // M <- (M + M^T) / 2
  for (int e = tid; e < sq; e += kThreads) {
    const int a = e / pk, c = e - a * pk;
    if (c < a) {
      const double v = 0.5 * (S.m[a * kLd + c] + S.m[c * kLd + a]);
      S.m[a * kLd + c] = v;
      S.m[c * kLd + a] = v;
    }
  }
  __syncthreads();
  for (int e = tid; e < sq; e += kThreads) {
    const int a = e / pk, c = e - a * pk;
    if (!finite(S.m[a * kLd + c]) || !finite(S.g[a * kLd + c])) S.flag[0] = 1;
  }
  if (tid < pk) {
    const double mjj = S.m[tid * kLd + tid];
    if (mjj < 0.0) S.flag[1] = 1;
    S.sc[tid] = mjj > 0.0 ? (FAST ? rsqrt(mjj) : 1.0 / sqrt(mjj)) : 0.0;
  }
  __syncthreads();
  if (S.flag[0] || S.flag[1]) {
    if (tid == 0) set_error(st, S.flag[0] ? ST_ERR_NUMERICAL : ST_ERR_NOT_SPD, 1);
    __syncthreads();
    return;
  }
  // scaled lower triangle, unit diagonal
  for (int e = tid; e < sq; e += kThreads) {
    const int a = e / pk, c = e - a * pk;
    if (c < a) S.l[a * kLd + c] = (S.sc[a] * S.m[a * kLd + c]) * S.sc[c];
    else if (c == a) S.l[a * kLd + a] = 1.0;
  }
  __syncthreads();
  if (tid < 32) warp_chol<FAST>(prm, S, pk);
  __syncthreads();
  const int m = S.chol_m;
  if (S.chol_fail) {
    if (tid == 0) set_error(st, S.chol_fail == 2 ? ST_ERR_NOT_SPD : ST_ERR_NUMERICAL, 2);
    __syncthreads();
    return;
  }
  if (m == 0) {
    if (tid == 0) set_error(st, ST_ERR_NUMERICAL, 3);
    __syncthreads();
    return;
  }
  // restricted factor -> y (as scratch) then st->L; restricted sc
  for (int e = tid; e < m * m; e += kThreads) {
    const int a = e / m, c = e - a * m;
    const double v = (c <= a) ? S.l[S.keep[a] * kLd + S.keep[c]] : 0.0;
    S.y[a * kLd + c] = v;
    st->L[a * kMaxP + c] = v;
  }
  __syncthreads();
  for (int e = tid; e < m * m; e += kThreads) {
    const int a = e / m, c = e - a * m;
    S.m[a * kLd + c] = S.y[a * kLd + c];  // factor
    // right-hand sides: Y[a][c] = sc[a] * G[c][a] on the kept set
    S.l[a * kLd + c] = S.sc[S.keep[a]] * S.g[S.keep[c] * kLd + S.keep[a]];
  }
  __syncthreads();
  chol_solve_cols(S.m, S.l, m, S.sv);
  for (int e = tid; e < m * m; e += kThreads) {
    const int b = e / m, a = e - b * m;
    const double v = -S.sc[S.keep[b]] * S.l[b * kLd + a];
    st->alphaT[b * kMaxP + a] = v;
    if (!finite(v)) S.flag[2] = 1;
  }
  if (tid < m) st->sc[tid] = S.sc[S.keep[tid]];
  __syncthreads();
  if (S.flag[2]) {
    if (tid == 0) set_error(st, ST_ERR_NUMERICAL, 4);
    __syncthreads();
    return;
  }
  if (tid == 0) {
    st->prev_pk = pk;
    st->changed = (m < pk) ? 1 : 0;
    if (m < pk) {
      int old[kMaxP];
      for (int j = 0; j < pk; ++j) {
        old[j] = ldcg(&st->agent[j]);
        st->old_agent[j] = old[j];
      }
      for (int j = 0; j < m; ++j) {
        st->keep[j] = S.keep[j];
        st->agent[j] = old[S.keep[j]];
      }
      st->drops = ldcg(&st->drops) + (pk - m);
      st->pk = m;
    }
  }
  __syncthreads();
}

// beta step: H, s2 -> beta_k^T, iteration count, stop test.
template <int NB>
__device__ void serial_beta(const Params& prm, SerialSmem& S) {
  DevState* st = prm.st;
  const int tid = threadIdx.x;
  const int pk = ldcg(&st->pk);
  const int sq = pk * pk;
  if (tid < 4) S.flag[tid] = 0;
  for (int e = tid; e < sq + pk; e += kThreads) {
    if (e < sq) {
      const int a = e / pk, c = e - a * pk;
      S.g[a * kLd + c] = red_get(st, kSlotGram0 + a * kMaxP + c);
    } else {
      S.s2[e - sq] = red_get(st, kSlotVec + (e - sq));
    }
  }
  for (int e = tid; e < sq; e += kThreads) {
    const int a = e / pk, c = e - a * pk;
    S.m[a * kLd + c] = ldcg(&st->L[a * kMaxP + c]);
  }
  if (tid < pk) S.sc[tid] = ldcg(&st->sc[tid]);
  __syncthreads();
  for (int e = tid; e < sq; e += kThreads) {
    const int a = e / pk, c = e - a * pk;
    if (!finite(S.g[a * kLd + c])) S.flag[0] = 1;
    S.l[a * kLd + c] = S.sc[a] * S.g[c * kLd + a];
  }
  __syncthreads();
  if (S.flag[0]) {
    if (tid == 0) set_error(st, ST_ERR_NUMERICAL, 5);
    __syncthreads();
    return;
  }
  chol_solve_cols(S.m, S.l, pk, S.sv);
  for (int e = tid; e < sq; e += kThreads) {
    const int b = e / pk, a = e - b * pk;
    const double v = -S.sc[b] * S.l[b * kLd + a];
    st->betaT[b * kMaxP + a] = v;
    if (!finite(v)) S.flag[1] = 1;
  }
  if (tid == 0) st->k = ldcg(&st->k) + 1;
  __syncthreads();
  if (S.flag[1]) {
    if (tid == 0) set_error(st, ST_ERR_NUMERICAL, 6);
    __syncthreads();
    return;
  }
  stop_test(prm, S, pk, 7);
}

// Preconditioned solve, after the update of X and R: iteration count and
// stop test on the residual norms (beta_k follows once Z_{k+1} is known).
__device__ void serial_kstop(const Params& prm, SerialSmem& S) {
  DevState* st = prm.st;
  const int pk = ldcg(&st->pk);
  for (int e = threadIdx.x; e < pk; e += kThreads) S.s2[e] = red_get(st, kSlotVec + e);
  if (threadIdx.x == 0) st->k = ldcg(&st->k) + 1;
  __syncthreads();
  stop_test(prm, S, pk, 17);
}

// Preconditioned solve: beta_k^T = -M^{-1} H^T with H = Z_{k+1}' A D_k in the
// Gram0 slot, from the factor of M kept by the alpha step.
template <int NB>
__device__ void serial_beta_pc(const Params& prm, SerialSmem& S) {
  DevState* st = prm.st;
  const int tid = threadIdx.x;
  const int pk = ldcg(&st->pk);
  const int sq = pk * pk;
  if (tid < 4) S.flag[tid] = 0;
  for (int e = tid; e < sq; e += kThreads) {
    const int a = e / pk, c = e - a * pk;
    S.g[a * kLd + c] = red_get(st, kSlotGram0 + a * kMaxP + c);
    S.m[a * kLd + c] = ldcg(&st->L[a * kMaxP + c]);
  }
  if (tid < pk) S.sc[tid] = ldcg(&st->sc[tid]);
  __syncthreads();
  for (int e = tid; e < sq; e += kThreads) {
    const int a = e / pk, c = e - a * pk;
    if (!finite(S.g[a * kLd + c])) S.flag[0] = 1;
    S.l[a * kLd + c] = S.sc[a] * S.g[c * kLd + a];
  }
  __syncthreads();
  if (S.flag[0]) {
    if (tid == 0) set_error(st, ST_ERR_NUMERICAL, 18);
    __syncthreads();
    return;
  }
  chol_solve_cols(S.m, S.l, pk, S.sv);
  for (int e = tid; e < sq; e += kThreads) {
    const int b = e / pk, a = e - b * pk;
    const double v = -S.sc[b] * S.l[b * kLd + a];
    st->betaT[b * kMaxP + a] = v;
    if (!finite(v)) S.flag[1] = 1;
  }
  if (tid == 0) st->pc_stage = PC_NONE;
  __syncthreads();
  if (S.flag[1] && tid == 0) set_error(st, ST_ERR_NUMERICAL, 19);
  __syncthreads();
}

// Preconditioned solve: after a stop test that continues the iteration, wait
// for Z (the launch ends and the preconditioner runs).
__device__ void serial_pc_request(const Params& prm, int stage) {
  if (!prm.precond) return;
  DevState* st = prm.st;
  if (threadIdx.x == 0 && *(volatile int*)&st->error == 0 && ldcg(&st->ctrl) == CTRL_LOOP)
    st->pc_stage = stage;
  __syncthreads();
}
__device__ void serial_pc_clear(const Params& prm) {
  if (prm.precond && threadIdx.x == 0) prm.st->pc_stage = PC_NONE;
  __syncthreads();
}

__device__ void serial_bnorm(const Params& prm, SerialSmem& S) {
  DevState* st = prm.st;
  if (threadIdx.x == 0) {
    const double b2 = red_get(st, kSlotScalar);
    const double bn = sqrt(b2);
    st->bnorm = bn;
    if (!finite(bn)) {
      set_error(st, ST_ERR_NUMERICAL, 8);
    } else if (bn == 0.0) {
      st->zero_rhs = 1;
      st->jbest = 0;
      st->result = ST_OK;
      st->ctrl = CTRL_FINISH;
    } else {
      st->ctrl = CTRL_LOOP;
    }
  }
  __syncthreads();
}

// init / replacement: residual norms of R = A X - b 1^T.
__device__ void serial_norms(const Params& prm, SerialSmem& S, bool replacement) {
  DevState* st = prm.st;
  const int pk = ldcg(&st->pk);
  for (int e = threadIdx.x; e < pk; e += kThreads) S.s2[e] = red_get(st, kSlotVec + e);
  if (threadIdx.x == 0 && replacement) {
    st->replacements = ldcg(&st->replacements) + 1;
    st->k_replaced = ldcg(&st->k);
  }
  __syncthreads();
  stop_test(prm, S, pk, replacement ? 9 : 10);
}

__device__ void serial_check(const Params& prm) {
  DevState* st = prm.st;
  if (threadIdx.x == 0) {
    const double tr = sqrt(red_get(st, kSlotScalar)) / ldcg(&st->bnorm);
    st->relres_true = tr;
    if (!finite(tr)) {
      set_error(st, ST_ERR_NUMERICAL, 11);
    } else if (tr <= prm.tol) {
      st->result = ST_OK;
      st->ctrl = CTRL_FINISH;
    } else if (ldcg(&st->k) >= prm.maxit || !prm.replacement ||
               ldcg(&st->k) == ldcg(&st->k_replaced)) {
      st->result = ST_NOT_CONVERGED;
      st->ctrl = CTRL_FINISH;
    } else {
      st->ctrl = CTRL_REPLACE;
    }
  }
  __syncthreads();
}

__device__ void serial_block_product(const Params& prm, SerialSmem& S) {
  DevState* st = prm.st;
  const int q = prm.q;
  const int sq = q * q;
  for (int e = threadIdx.x; e < 2 * sq; e += kThreads) {
    const int f = e < sq ? e : e - sq;
    const int a = f / q, c = f - a * q;
    (e < sq ? S.m : S.g)[a * kLd + c] = red_get(st, red_slot(RED_M_G, q, e));
  }
  __syncthreads();
  for (int e = threadIdx.x; e < sq; e += kThreads) {
    const int a = e / q, c = e - a * q;
    double v = S.m[a * kLd + c];
    if (c != a) v = 0.5 * (S.m[a * kLd + c] + S.m[c * kLd + a]);
    st->gram_out[a * kMaxP + c] = v;
    st->gram_out[kSq + a * kMaxP + c] = S.g[a * kLd + c];
  }
  if (threadIdx.x == 0) st->result = ST_OK;
  __syncthreads();
}


// FP8 operand: column scales sigma_j = max_i |V_ij| / 448 from the per-CTA
// maxima in the vector slot (hi part).
// Sliced FP64 operand (pow2): sigma_j = 2^e_j with e_j the binary exponent of
// max_i |V_ij| (so |V_ij| / sigma_j < 1), from the same per-CTA maxima.
__device__ void serial_sigma(const Params& prm, int pk, bool pow2 = false) {
  DevState* st = prm.st;
  const int G = gridDim.x;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // one warp per column; the per-CTA maxima are non-negative doubles (or
  // NaN), whose bit patterns order as their values with NaN on top
  for (int j = warp; j < pk; j += kWarps) {
    unsigned long long mb = 0ull;
    for (int g = lane; g < G; g += 32) {
      const unsigned long long v = (unsigned long long)__double_as_longlong(
          ldcg(prm.part + (size_t)g * kPartStride + kSlotVec + j));
      mb = v > mb ? v : mb;
    }
    for (int m = 16; m >= 1; m >>= 1) {
      const unsigned long long o = __shfl_xor_sync(0xffffffffu, mb, m);
      mb = o > mb ? o : mb;
    }
    if (lane != 0) continue;
    const double m = __longlong_as_double((long long)mb);
    if (pow2) {
      int e = 0;
      if (m > 0.0) frexp(m, &e);
      st->sigma[j] = ldexpf(1.f, e);
      if (!(m == m) || isinf(m) || e < -125 || e > 127) set_error(st, ST_ERR_NUMERICAL, 16);
    } else {
      const float mf = (float)m;
      st->sigma[j] = mf > 0.f ? mf / 448.f : 1.f;
      if (!(mf == mf) || isinf(mf)) set_error(st, ST_ERR_NUMERICAL, 12);
    }
  }
  __syncthreads();
}

// Refinement step: ||b|| (vector slot 0) and ||A x - b|| (scalar slot).
__device__ void serial_refine(const Params& prm) {
  DevState* st = prm.st;
  if (threadIdx.x == 0) {
    const double bn = sqrt(red_get(st, kSlotVec));
    const double rn = sqrt(red_get(st, kSlotScalar));
    st->bnorm = bn;
    st->rnorm = rn;
    st->relres_true = bn > 0.0 ? rn / bn : rn;
    if (!finite(rn) || !finite(bn)) set_error(st, ST_ERR_NUMERICAL, 13);
  }
  __syncthreads();
}


// --------------------------------------------------------------------------
// Tensor-core A-pass of the inner low-precision solves (policy != POL_FP64).
// The quantised A (BF16, or FP8 E4M3 with row scales) streams through a TMA
// ring into tcgen05.mma; the operand block is converted to the MMA type by
// the rows' owners first.  Work is split stream-K over (row tile, k-chunk)
// units exactly as in the standalone block product (sliced A: over (row tile,
// slice, k-chunk), so that a CTA sums the slices of a row tile itself); after
// a grid barrier the owner of each row sums the partial tiles that cover it,
// in CTA order, and applies the scales.  The ring position, phases and accumulator-buffer
// counts live in shared memory, so every A-pass resumes where the previous
// one stopped.
// --------------------------------------------------------------------------
struct LpShared {
  int p_stage;
  unsigned p_phase;
  int m_stage;
  unsigned m_phase;
  int m_seg;
  int m_any;
  int e_seg[4];             // per epilogue warp
  int s_stage[2];           // per split warp (TF32x3)
  unsigned s_phase[2];
  unsigned tmem;
  int issued[tc::kStages];  // phase of the last copy issued on each stage, -1 = none
};

template <int POL>
struct LpCfg {
  static constexpr int KIND = (POL == POL_FP8)      ? tc::KIND_FP8
                              : (POL == POL_TF32X3) ? tc::KIND_TF32X3
                              : (POL == POL_SLICED) ? tc::KIND_SLICED
                                                    : tc::KIND_BF16;
};

// Operand columns of the tensor-core pass: 16 or 32 (the MMA's N), or P for
// the sliced FP64 operand, whose kSlices slices per column fill N instead.
template <int P, int POL>
struct LpNP {
  static constexpr int value = (POL == POL_SLICED) ? P : (P <= 16) ? 16 : 32;
};

template <int KIND, int NP>
struct LpLayout {
  using S = tc::Shape<KIND, NP>;
  // full[ST], empty[ST], split[ST], accf[2], acce[2], drain
  static constexpr int kBars = 3 * S::kStagesK + 5;
  static constexpr size_t kBytes = 1024 + S::kRingBytes + kBars * 8 + sizeof(LpShared) + 64;
};

struct LpCtx {
  uint8_t* ring;
  uint64_t* bars;
  LpShared* sh;
};

// Wait without regard to the error flag (teardown drains), bounded.
__device__ void mbar_wait_drain(uint32_t a, uint32_t parity, long long timeout_ns) {
  const unsigned long long t0 = globaltimer_ns();
  while (!tc::mbar_try(a, parity)) {
    if (globaltimer_ns() - t0 > (unsigned long long)timeout_ns) return;
    __nanosleep(64);
  }
}

template <int KIND, int NP>
__device__ void lp_pass(const Params& prm, LpCtx& L) {
  using S = tc::Shape<KIND, NP>;
  constexpr int ST = S::kStagesK;
  constexpr int NM = S::NMMA;
  constexpr uint32_t kIdesc = tc::idesc<KIND>(NM);
  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const int G = gridDim.x;
  const int c = blockIdx.x;
  const int64_t U = prm.lp_units;
  const int kc = prm.lp_kc;
  const int64_t u0 = tc::unit_begin(U, G, c);
  const int64_t u1 = tc::unit_begin(U, G, c + 1);
  uint8_t* sA = L.ring;
  uint8_t* sA2 = L.ring + ST * tc::kTileABytes;           // A_lo tiles (TF32x3)
  uint8_t* sB = sA2 + ST * S::kTileA2Bytes;
  uint64_t* full = L.bars;
  uint64_t* empty = L.bars + ST;
  uint64_t* split = L.bars + 2 * ST;
  uint64_t* accf = L.bars + 3 * ST;
  uint64_t* acce = accf + 2;
  int* err = &prm.st->error;
  const long long to = prm.timeout_ns;

  if (warp == 0) {
    if (lane == 0) {
      // operand rows were written through the generic proxy before the barrier
      asm volatile("fence.proxy.async.global;" ::: "memory");
      int stage = L.sh->p_stage;
      uint32_t phase = L.sh->p_phase;
      const uint64_t pol_a = tc::l2_policy_evict_first(), pol_b = tc::l2_policy_evict_last();
      for (int64_t u = u0; u < u1; ++u) {
        if (!tc::mbar_wait(tc::smem_u32(&empty[stage]), phase ^ 1u, to, err)) break;
        const int t = (int)(u / kc);
        const int k = (int)(u % kc);
        // sliced A: tile t = (row tile tr, slice sl) lies in slice plane sl
        int ty = t;
        if constexpr (KIND == tc::KIND_SLICED) {
          const int tr = t / tc::kSlices;
          ty = (t - tr * tc::kSlices) * (int)prm.lp_tiles + tr;
        }
        const uint32_t fb = tc::smem_u32(&full[stage]);
        tc::mbar_expect_tx(fb, S::kStageBytes);
        tc::tma_load_2d_hint(tc::smem_u32(sA + stage * tc::kTileABytes), &prm.lp_tmA,
                             k * prm.lp_kelems, ty * tc::kBM, fb, pol_a);
        tc::tma_load_2d_hint(tc::smem_u32(sB + stage * S::kTileBBytes), &prm.lp_tmB,
                             k * prm.lp_kelems, 0, fb, pol_b);
        L.sh->issued[stage] = (int)phase;
        if (++stage == ST) { stage = 0; phase ^= 1u; }
      }
      L.sh->p_stage = stage;
      L.sh->p_phase = phase;
    }
  } else if (warp == 1) {
    if (lane == 0) {
      int stage = L.sh->m_stage;
      uint32_t phase = L.sh->m_phase;
      int seg = L.sh->m_seg;
      const uint32_t tmem = L.sh->tmem;
      for (int64_t u = u0; u < u1; ++u) {
        const int k = (int)(u % kc);
        const bool first = (u == u0) || (k == 0);
        const bool last = (u == u1 - 1) || (k == kc - 1);
        const int b = seg & 1;
        if (first) {
          if (!tc::mbar_wait(tc::smem_u32(&acce[b]), (((uint32_t)seg >> 1) & 1u) ^ 1u, to, err)) break;
          tc::fence_after();
        }
        // TF32x3: the split warps signal once the tile has landed and its low
        // part is written; the other kinds wait for the copy itself
        uint64_t* ready = (KIND == tc::KIND_TF32X3) ? &split[stage] : &full[stage];
        if (!tc::mbar_wait(tc::smem_u32(ready), phase, to, err)) break;
        tc::fence_after();
        const uint32_t dt = tmem + (uint32_t)(b * NM);
        const uint64_t ad = tc::sdesc(tc::smem_u32(sA + stage * tc::kTileABytes));
        const uint64_t bd = tc::sdesc(tc::smem_u32(sB + stage * S::kTileBBytes));
#pragma unroll
        for (int kk = 0; kk < tc::kRowBytes / 32; ++kk) {
          // N = NM covers the operand's hi and lo rows (FP8, TF32x3)
          tc::mma<KIND>(dt, ad + 2u * kk, bd + 2u * kk, kIdesc, (first && kk == 0) ? 0u : 1u);
          if constexpr (KIND == tc::KIND_TF32X3) {
            const uint64_t a2 = tc::sdesc(tc::smem_u32(sA2 + stage * tc::kTileABytes));
            tc::mma<KIND>(dt, a2 + 2u * kk, bd + 2u * kk, kIdesc, 1u);
          }
        }
        L.sh->m_any = 1;
        tc::mma_commit(tc::smem_u32(&empty[stage]));
        if (last) {
          tc::mma_commit(tc::smem_u32(&accf[b]));
          ++seg;
        }
        if (++stage == ST) { stage = 0; phase ^= 1u; }
      }
      L.sh->m_stage = stage;
      L.sh->m_phase = phase;
      L.sh->m_seg = seg;
    }
  } else if (warp < 4) {
    if constexpr (KIND == tc::KIND_TF32X3) {
      // split warps: A_lo = A - tf32(A) for every landed FP32 tile, written at
      // the same (swizzled) position of the A_lo ring
      const int w = warp - 2;
      const int t64 = threadIdx.x - 64;
      int stage = L.sh->s_stage[w];
      uint32_t phase = L.sh->s_phase[w];
      for (int64_t u = u0; u < u1; ++u) {
        if (!tc::mbar_wait(tc::smem_u32(&full[stage]), phase, to, err)) break;
        const float4* src = reinterpret_cast<const float4*>(sA + stage * tc::kTileABytes);
        float4* dst = reinterpret_cast<float4*>(sA2 + stage * tc::kTileABytes);
        for (int v = t64; v < tc::kTileABytes / 16; v += 64) {
          float4 a = src[v];
          float4 lo;
          lo.x = a.x - __uint_as_float(__float_as_uint(a.x) & 0xFFFFE000u);
          lo.y = a.y - __uint_as_float(__float_as_uint(a.y) & 0xFFFFE000u);
          lo.z = a.z - __uint_as_float(__float_as_uint(a.z) & 0xFFFFE000u);
          lo.w = a.w - __uint_as_float(__float_as_uint(a.w) & 0xFFFFE000u);
          dst[v] = lo;
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(tc::smem_u32(&split[stage]));
        if (++stage == ST) { stage = 0; phase ^= 1u; }
      }
      __syncwarp();
      if (lane == 0) {
        L.sh->s_stage[w] = stage;
        L.sh->s_phase[w] = phase;
      }
    }
  } else {
    const int quad = warp & 3;
    const int row = quad * 32 + lane;
    int seg = L.sh->e_seg[quad];
    // sliced: FP64 sum over the slices of one row tile that this CTA covers
    double acc[KIND == tc::KIND_SLICED ? NP : 1];
    if (u0 < u1) {
      const int t0 = (int)(u0 / kc);
      const int t1 = (int)((u1 - 1) / kc);
      for (int t = t0; t <= t1; ++t, ++seg) {
        const int b = seg & 1;
        if (!tc::mbar_wait(tc::smem_u32(&accf[b]), ((uint32_t)seg >> 1) & 1u, to, err)) break;
        tc::fence_after();
        const uint32_t tbase = L.sh->tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(b * NM);
        if constexpr (KIND == tc::KIND_SLICED) {
          // accumulator column u NP + j holds the exact integer
          // sum_k qA_s(row, k) qV_u(k, j); its weight is 16^-(s+u+2) (s: slice
          // of A of this tile).  Combined in FP64, largest weight first.
          // weights 16^-(u+2) are compile-time powers of two (one exact FMA per
          // accumulator); 16^-s is applied once per entry.  Tiles run slice-
          // minor, so the slices of a row tile are summed here (slice 0 first)
          // and one partial per (CTA, row tile) is written.
          const int tr = t / tc::kSlices;
          const int sl = t - tr * tc::kSlices;
          double out[NP];
#pragma unroll
          for (int j = 0; j < NP; ++j) out[j] = 0.0;
#pragma unroll
          for (int ch = 0; ch < NM / 16; ++ch) {
            float v[16];
            tc::tmem_ld<16>(tbase + (uint32_t)(ch * 16), v);
#pragma unroll
            for (int q = 0; q < 16; ++q) {
              constexpr double kW[tc::kSlices] = {
                  0x1p-8, 0x1p-12, 0x1p-16, 0x1p-20, 0x1p-24, 0x1p-28, 0x1p-32,
                  0x1p-36, 0x1p-40, 0x1p-44, 0x1p-48, 0x1p-52, 0x1p-56, 0x1p-60};
              const int col = ch * 16 + q;
              const int u = col / NP;
              if (u < tc::kSlices) out[col % NP] = fma((double)v[q], kW[u], out[col % NP]);
            }
          }
          const double ws = __longlong_as_double((int64_t)(1023 - 4 * sl) << 52);  // 16^-s
          const bool open = (t == t0) || (sl == 0);
#pragma unroll
          for (int j = 0; j < NP; ++j) acc[j] = open ? out[j] * ws : fma(out[j], ws, acc[j]);
          if (t == t1 || sl == tc::kSlices - 1) {
            double* dst = reinterpret_cast<double*>(prm.lp_part) + ((size_t)(c + tr) * tc::kBM + row) * NP;
#pragma unroll
            for (int j = 0; j < NP; ++j) dst[j] = acc[j];
          }
        } else {
          float v[NM];
          tc::tmem_ld<NM>(tbase, v);
          if constexpr (NM != NP) {
#pragma unroll
            for (int j = 0; j < NP; ++j) v[j] += v[NP + j];  // hi + lo halves
          }
          float* dst = prm.lp_part + ((size_t)(c + t) * tc::kBM + row) * NP;
#pragma unroll
          for (int j = 0; j < NP; j += 4)
            *reinterpret_cast<float4*>(dst + j) = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
        }
        tc::fence_before();
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(tc::smem_u32(&acce[b]));
      }
    }
    __syncwarp();
    if (lane == 0) L.sh->e_seg[quad] = seg;
  }
  __syncthreads();
}

// Y[:, 0:pk] = A_lp V[:, 0:pk] (- b) on the rows [r0, r1) of this CTA, with the
// operand conversion, the tensor-core pass and the fixup.  false = leave.
// Operand entry (column j of V, row i) in the MMA type: BF16, or the TF32
// halves hi = tf32(v) (low 13 mantissa bits cleared) and lo = v - hi (exact
// in FP32).  FP8 needs the column scales first and is converted in lp_apass.
template <int KIND, int NP>
__device__ __forceinline__ void lp_put(const Params& prm, int j, int64_t i, double v) {
  const int64_t ldk = prm.lp_ldk;
  if constexpr (KIND == tc::KIND_BF16) {
    reinterpret_cast<__nv_bfloat16*>(prm.lp_dq)[(int64_t)j * ldk + i] = __double2bfloat16(v);
  } else if constexpr (KIND == tc::KIND_TF32X3) {
    const float f = (float)v;
    const float hi = __uint_as_float(__float_as_uint(f) & 0xFFFFE000u);
    float* o = reinterpret_cast<float*>(prm.lp_dq);
    o[(int64_t)j * ldk + i] = hi;
    o[(int64_t)(NP + j) * ldk + i] = f - hi;
  }
}

// preconv: the operand rows already hold V in the MMA type (written by the
// D-update, followed by a grid barrier), so the conversion and its barrier
// are skipped.
// The fixup hands finished entries to `epi` four columns at a time:
// epi(i, j0, v, cnt) with v[u] the entry (row i, column j0 + u) of A_lp V, the
// scales applied, u < cnt; lp_apass below stores them (minus b) in Y.
// cmax (FP8 and sliced kinds; nullable): this CTA's column maxima of |V| as
// ordered bit patterns, when the caller has them already (no scan of V).
// VT = float (FP8 kind only): V is an FP32 block; the operand split, the
// fixup sums and the entries handed to epi are FP32, and cmax holds FP32 bit
// patterns.
template <int P, int POL, class Epi, class VT = double>
__device__ bool lp_apass_epi(const Params& prm, const VT* V, int pk, int64_t r0, int64_t r1,
                             LpCtx& L, SyncShared* ss, int* s_err, bool preconv, Epi epi,
                             const unsigned long long* cmax = nullptr) {
  constexpr int KIND = LpCfg<POL>::KIND;
  constexpr int NP = LpNP<P, POL>::value;
  constexpr bool kF32 = std::is_same<VT, float>::value;
  static_assert(!kF32 || KIND == tc::KIND_FP8, "FP32 operand blocks: FP8 kind only");
  DevState* st = prm.st;
  const int p = prm.p;
  const int tid = threadIdx.x;
  const int64_t nr = r1 - r0;
  const int64_t ldk = prm.lp_ldk;
  double* mypart = prm.part + (size_t)blockIdx.x * kPartStride;

  if constexpr (KIND == tc::KIND_FP8 || KIND == tc::KIND_SLICED) {
    // column maxima of |V| over this CTA's rows, as ordered bit patterns
    // (a NaN stays on top and reaches the check of the column scales)
    __shared__ unsigned long long s_cmax[P];
    if (cmax == nullptr) {
      for (int j = tid; j < pk; j += kThreads) s_cmax[j] = 0ull;
      __syncthreads();
      for (int idx = tid; idx < (int)nr * pk; idx += kThreads) {
        const int li = idx / pk;
        const int j = idx - li * pk;
        const VT v = __ldcg(V + (r0 + li) * p + j);
        if constexpr (kF32)
          atomicMax(&s_cmax[j], (unsigned long long)__float_as_uint(fabsf(v)));
        else
          atomicMax(&s_cmax[j], (unsigned long long)__double_as_longlong(fabs(v)));
      }
      __syncthreads();
      cmax = s_cmax;
    }
    for (int j = tid; j < pk; j += kThreads)
      mypart[kSlotVec + j] = kF32 ? (double)__uint_as_float((unsigned)cmax[j])
                                  : __longlong_as_double((long long)cmax[j]);
    const int f = grid_arrive(prm, ss);
    if (f < 0) return false;
    if (f == 1) {
      if (!cta_error(st, s_err)) serial_sigma(prm, pk, KIND == tc::KIND_SLICED);
      grid_release(prm, ss);
      if (cta_error(st, s_err)) return false;
    }
  }
  if constexpr (KIND == tc::KIND_SLICED) {
    // operand row u NP + j holds slice u of column j (x = V_ij / sigma_j,
    // split as in the slicing of A); rows past kSlices NP stay zero
    using Sh = tc::Shape<KIND, NP>;
    uint8_t* o = reinterpret_cast<uint8_t*>(prm.lp_dq);
    for (int64_t idx = tid; idx < (int64_t)NP * nr; idx += kThreads) {
      const int j = (int)(idx / nr);
      const int64_t i = r0 + (idx - (int64_t)j * nr);
      uint64_t X = 0ull;
      uint32_t neg = 0u;
      if (j < pk) {
        int e;
        frexpf(__ldcg(&st->sigma[j]), &e);  // sigma_j = 2^(e - 1)
        X = tc::slice_bits(ldcg(V + i * p + j), e - 1, &neg);
      }
#pragma unroll
      for (int u = 0; u < tc::kSlices; ++u)
        o[(int64_t)(u * NP + j) * ldk + i] =
            (uint8_t)tc::e4m3_digit((uint32_t)(X >> (52 - 4 * u)) & 15u, neg);
    }
    for (int64_t idx = tid; idx < (int64_t)(Sh::NB - tc::kSlices * NP) * nr; idx += kThreads) {
      const int64_t rrow = tc::kSlices * NP + idx / nr;
      o[rrow * ldk + r0 + idx % nr] = 0;
    }
    asm volatile("fence.proxy.async.global;" ::: "memory");
    if (!grid_barrier(prm, ss, s_err)) return false;
  } else if (!preconv) {
    // operand row j (< NP) holds column j of V, zero beyond pk; a thread
    // takes whole rows of V (contiguous reads), the byte rows are written
    // across consecutive threads
    __shared__ VT s_inv[32];  // FP8: 1 / sigma_j
    if constexpr (KIND == tc::KIND_FP8) {
      for (int j = tid; j < NP; j += kThreads)
        s_inv[j] = j < pk ? VT(1) / (VT)__ldcg(&st->sigma[j]) : VT(0);
      __syncthreads();
    }
    for (int li = tid; li < (int)nr; li += kThreads) {
      const int64_t i = r0 + li;
      const VT* vr = V + i * p;
#pragma unroll 4
      for (int j = 0; j < NP; ++j) {
        const VT v = (j < pk) ? __ldcg(vr + j) : VT(0);
        if constexpr (KIND == tc::KIND_FP8) {
          const VT x = v * s_inv[j];
          __nv_fp8_storage_t h, l;
          if constexpr (kF32) {
            h = __nv_cvt_float_to_fp8(x, __NV_SATFINITE, __NV_E4M3);
            const float hv = __half2float(__half(__nv_cvt_fp8_to_halfraw(h, __NV_E4M3)));
            l = __nv_cvt_float_to_fp8(x - hv, __NV_SATFINITE, __NV_E4M3);
          } else {
            h = __nv_cvt_double_to_fp8(x, __NV_SATFINITE, __NV_E4M3);
            const double hv = (double)__half2float(__half(__nv_cvt_fp8_to_halfraw(h, __NV_E4M3)));
            l = __nv_cvt_double_to_fp8(x - hv, __NV_SATFINITE, __NV_E4M3);
          }
          uint8_t* o = reinterpret_cast<uint8_t*>(prm.lp_dq);
          o[(int64_t)j * ldk + i] = (uint8_t)h;
          o[(int64_t)(NP + j) * ldk + i] = (uint8_t)l;
        } else {
          lp_put<KIND, NP>(prm, j, i, v);
        }
      }
    }
    asm volatile("fence.proxy.async.global;" ::: "memory");
    if (!grid_barrier(prm, ss, s_err)) return false;
  }
  lp_pass<KIND, NP>(prm, L);
  if (!grid_barrier(prm, ss, s_err)) return false;
  // fixup: each owned row sums the partial tiles of the CTAs that covered it
  // (FP32 tiles; FP64 with the slices already summed for the sliced kind),
  // in CTA order.  The CTA range of each row tile of this CTA's rows is found
  // once, kRng row tiles at a time; a thread then takes a whole row and
  // reads its partial rows four columns at a time.
  const int G = gridDim.x;
  const int64_t U = prm.lp_units;
  const int kc = prm.lp_kc;
  using PartT = typename std::conditional<KIND == tc::KIND_SLICED, double, float>::type;
  const PartT* part = reinterpret_cast<const PartT*>(prm.lp_part);
  const int64_t per_tile = (KIND == tc::KIND_SLICED) ? (int64_t)tc::kSlices * kc : (int64_t)kc;
  constexpr int kRng = 8;
  __shared__ int s_rng[kRng][2];
  const int tr0 = (int)(r0 / tc::kBM);
  const int ntr = (nr > 0) ? (int)((r1 - 1) / tc::kBM) - tr0 + 1 : 0;
  const bool some_empty = U < G;  // with U >= G every CTA holds a unit
  for (int q0 = 0; q0 < ntr; q0 += kRng) {
    const int nq = min(kRng, ntr - q0);
    for (int q = tid; q < nq; q += kThreads) {
      const int64_t lo = (int64_t)(tr0 + q0 + q) * per_tile;
      const int64_t hi = lo + per_tile;
      int c0 = (int)((lo * G) / U);
      while (c0 > 0 && tc::unit_begin(U, G, c0) > lo) --c0;
      while (tc::unit_begin(U, G, c0 + 1) <= lo) ++c0;
      int c1 = c0;
      while (c1 + 1 < G && tc::unit_begin(U, G, c1 + 1) < hi) ++c1;
      s_rng[q][0] = c0;
      s_rng[q][1] = c1;
    }
    __syncthreads();
    const int64_t ra = max(r0, (int64_t)(tr0 + q0) * tc::kBM);
    const int nrow = (int)(min(r1, (int64_t)(tr0 + q0 + nq) * tc::kBM) - ra);
    for (int li = tid; li < nrow; li += kThreads) {
      const int64_t i = ra + li;
      const int tr = (int)(i / tc::kBM);
      const int rr = (int)(i - (int64_t)tr * tc::kBM);
      const int c0 = s_rng[tr - tr0 - q0][0], c1 = s_rng[tr - tr0 - q0][1];
      const VT rs = prm.lp_row_scale ? (VT)prm.lp_row_scale[i] : VT(1);
      for (int j0 = 0; j0 < pk; j0 += 4) {
        VT sv[4] = {VT(0), VT(0), VT(0), VT(0)};
        for (int cc = c0; cc <= c1; ++cc) {
          if (some_empty && tc::unit_begin(U, G, cc + 1) <= tc::unit_begin(U, G, cc)) continue;
          const PartT* pr = part + ((size_t)(cc + tr) * tc::kBM + rr) * NP + j0;
          if constexpr (NP >= 4) {
            if constexpr (KIND == tc::KIND_SLICED) {
              const double2 a = __ldcg(reinterpret_cast<const double2*>(pr));
              const double2 b = __ldcg(reinterpret_cast<const double2*>(pr) + 1);
              sv[0] += a.x; sv[1] += a.y; sv[2] += b.x; sv[3] += b.y;
            } else {
              const float4 a = __ldcg(reinterpret_cast<const float4*>(pr));
              sv[0] += (VT)a.x; sv[1] += (VT)a.y;
              sv[2] += (VT)a.z; sv[3] += (VT)a.w;
            }
          } else {
#pragma unroll
            for (int u = 0; u < 4; ++u)
              if (j0 + u < NP) sv[u] += (VT)__ldcg(pr + u);
          }
        }
        const int cnt = min(4, pk - j0);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int j = j0 + u;
          if (u < cnt) {
            if constexpr (KIND == tc::KIND_SLICED) {
              sv[u] *= rs * (double)__ldcg(&st->sigma[j]);
            } else {
              if (prm.lp_row_scale) sv[u] *= rs;
              if constexpr (KIND == tc::KIND_FP8) sv[u] *= (VT)__ldcg(&st->sigma[j]);
            }
          }
        }
        epi(i, j0, sv, cnt);
      }
    }
    __syncthreads();
  }
  return true;
}

template <int P, int POL>
__device__ bool lp_apass(const Params& prm, const double* V, int pk, double* Y, bool sub_b,
                         int64_t r0, int64_t r1, LpCtx& L, SyncShared* ss, int* s_err,
                         bool preconv = false, const unsigned long long* cmax = nullptr) {
  const int p = prm.p;
  return lp_apass_epi<P, POL>(prm, V, pk, r0, r1, L, ss, s_err, preconv,
                              [&](int64_t i, int j0, const double (&v)[4], int cnt) {
#pragma unroll
                                for (int u = 0; u < 4; ++u)
                                  if (u < cnt) Y[i * p + j0 + u] = sub_b ? v[u] - prm.b[i] : v[u];
                              },
                              cmax);
}

// --------------------------------------------------------------------------
// FP32 A-pass of the batched refinement's inner solves (policy POL_F32):
// Y = A32 V (- b 1^T) with A32 the FP32 copy of A (rows padded with zeros to
// a32_ld, a multiple of 4).  The operand columns are first written as FP32
// rows (own rows, then a barrier).  Each warp then takes whole rows: lane l
// multiplies the elements 4l + 128s of the row (16-byte loads) with the
// operand rows, and a butterfly over the lanes sums each column.  Products
// and sums are FP32 on the FP32 pipe: the inner solve needs only the
// accuracy of its FP32 operator, and the FP32 rate is 64 times the FP64 rate
// on GB300.  The operand rows are read through L1, which is coherent with
// this CTA's own writes: the policy runs in groups of one CTA only.
// --------------------------------------------------------------------------
template <int P>
__device__ bool apass_f32(const Params& prm, const double* V, int pk, double* Y, bool sub_b,
                          int64_t r0, int64_t r1, SyncShared* ss, int* s_err) {
  const int p = prm.p;
  const int64_t ld = prm.a32_ld;
  float* vt = prm.vt32;
  const int tid = threadIdx.x;
  const int64_t nr = r1 - r0;
  for (int64_t idx = tid; idx < nr * P; idx += kThreads) {
    const int c = (int)(idx / nr);
    const int64_t i = r0 + (idx - (int64_t)c * nr);
    vt[c * ld + i] = c < pk ? (float)ldcg(V + i * p + c) : 0.f;
  }
  if (!grid_barrier(prm, ss, s_err)) return false;
  const int lane = tid & 31, warp = tid >> 5;
  const int64_t w0 = r0 + (nr * warp) / kWarps;
  const int64_t w1 = r0 + (nr * (warp + 1)) / kWarps;
  for (int64_t row = w0; row < w1; ++row) {
    const float* Ar = prm.a32 + row * ld;
    float acc[P];
#pragma unroll
    for (int c = 0; c < P; ++c) acc[c] = 0.f;
    for (int64_t k = 4 * lane; k < ld; k += 128) {
      const float4 a = __ldcg(reinterpret_cast<const float4*>(Ar + k));
#pragma unroll
      for (int c = 0; c < P; ++c) {
        const float4 v = *reinterpret_cast<const float4*>(vt + c * ld + k);
        acc[c] = fmaf(a.x, v.x, acc[c]);
        acc[c] = fmaf(a.y, v.y, acc[c]);
        acc[c] = fmaf(a.z, v.z, acc[c]);
        acc[c] = fmaf(a.w, v.w, acc[c]);
      }
    }
    float mine = 0.f;
#pragma unroll
    for (int c = 0; c < P; ++c) {
#pragma unroll
      for (int m = 16; m >= 1; m >>= 1) acc[c] += __shfl_xor_sync(0xffffffffu, acc[c], m);
      if (lane == c) mine = acc[c];
    }
    if (lane < pk) {
      double y = (double)mine;
      if (sub_b) y -= prm.b[row];
      Y[row * p + lane] = y;
    }
  }
  __syncthreads();
  return true;
}

// --------------------------------------------------------------------------
// The persistent kernel.
// --------------------------------------------------------------------------
__device__ __forceinline__ double splitmix_uniform(unsigned long long seed,
                                                   unsigned long long c) {
  // SplitMix64 output number c+1 of the stream seeded with `seed`
  // (Steele, Lea, Flood 2014); top 53 bits -> [0, 1).
  unsigned long long z = seed + (c + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z = z ^ (z >> 31);
  return (double)(z >> 11) * 0x1.0p-53;
}

template <int P, bool VEC, int POL, bool VARIANTS = false>
__device__ __forceinline__ void solve_body(const Params& prm, double* smem, LpCtx* L) {
  // FP64 solves keep the oracle's arithmetic in the exchange steps; the inner
  // solves of the mixed-precision paths take the faster forms
  constexpr bool kExact = POL == POL_FP64 || POL == POL_SLICED;
  __shared__ SyncShared ss;
  __shared__ int s_int[4];
  __shared__ int s_err;
  SerialSmem& S = *reinterpret_cast<SerialSmem*>(smem);
  DevState* st = prm.st;
  const int G = grp_size(prm);
  const int cta = grp_rank(prm);
  const int tid = threadIdx.x;
  const int64_t n = prm.n;
  const int64_t r0 = ((int64_t)cta * n) / G;
  const int64_t r1 = ((int64_t)(cta + 1) * n) / G;
  const int p = prm.p;
  double* mypart = prm.part + (size_t)cta * kPartStride;

  // Exchange point: the group's sums of the reduction set SET (size from Q)
  // land in st->red, then the last-arriving CTA runs CALL and releases the
  // others.  Large sets are summed by all CTAs after an extra grid barrier.
#define CCG_SYNC_RED(SET, Q, CALL)                                           \
  {                                                                          \
    const int q_ = (Q);                                                      \
    const bool spread_ = G > 1 && red_count(SET, q_) > kRedLocalMax;         \
    if (spread_) {                                                           \
      if (!grid_barrier(prm, &ss, &s_err)) return;                           \
      reduce_entries<kExact>(prm, SET, q_, cta * kSubParts, G * kSubParts,     \
                             kSubParts);                                     \
    }                                                                        \
    const int f_ = grid_arrive(prm, &ss);                                    \
    if (f_ < 0) return;                                                      \
    if (f_ == 1) {                                                           \
      if (!cta_error(st, &s_err)) {                                          \
        if (!spread_) {                                                      \
          reduce_entries<kExact>(prm, SET, q_, 0, kWarps);                           \
          __syncthreads();                                                   \
        }                                                                    \
        CALL;                                                                \
      }                                                                      \
      grid_release(prm, &ss);                                                \
      if (cta_error(st, &s_err)) return;                                     \
    }                                                                        \
  }

  if (prm.mode == MODE_BARRIER_SELFTEST) {
    grid_barrier(prm, &ss, &s_err);
    return;
  }

  if constexpr (POL == POL_FP64) {
    if (prm.mode == MODE_BLOCK_PRODUCT) {
      const int q = prm.q;
      apass<P, VEC, VARIANTS>(prm, prm.V, q, 0, q, prm.Wout, q, false, r0, r1, smem);
      partial_grams<true>(prm.V, prm.Wout, prm.U, prm.U ? prm.V : nullptr, nullptr, q, q, r0, r1,
                    mypart, smem, kStageDoubles);
      CCG_SYNC_RED(RED_M_G, q, serial_block_product(prm, S));
      return;
    }
    if (prm.mode == MODE_REFINE) {
      // x += c delta ; r = A x - b (FP64) ; ||b||, ||r|| ; b_in = -r sqrt(n) / ||r||
      if (prm.ref_delta != nullptr)
        for (int64_t i = r0 + tid; i < r1; i += kThreads)
          prm.ref_x[i] = fma(prm.ref_coef, prm.ref_delta[i], prm.ref_x[i]);
      if (!grid_barrier(prm, &ss, &s_err)) return;
      apass<1, VEC, VARIANTS>(prm, prm.ref_x, 1, 0, 1, prm.ref_r, 1, true, r0, r1, smem);
      partial_sumsq(prm.ref_r, 1, r0, r1, mypart, kSlotScalar);
      __syncthreads();
      partial_sumsq(prm.b, 1, r0, r1, mypart, kSlotVec);
      CCG_SYNC_RED(RED_B_R, 1, serial_refine(prm));
      const double rn = ldcg(&st->rnorm);
      const double scale = rn > 0.0 ? sqrt((double)n) / rn : 0.0;
      for (int64_t i = r0 + tid; i < r1; i += kThreads) prm.ref_bin[i] = -ldcg(prm.ref_r + i) * scale;
      return;
    }
  } else {
    if constexpr (POL != POL_F32) {
      if (prm.mode == MODE_BLOCK_PRODUCT) {
        // W = A_lp V on the tensor cores (same code as the inner solves' A-pass)
        if (lp_apass<P, POL>(prm, prm.V, prm.q, prm.Wout, false, r0, r1, *L, &ss, &s_err) &&
            tid == 0 && cta == 0)
          st->result = ST_OK;
        return;
      }
      if constexpr (POL != POL_SLICED) {
        if (prm.mode == MODE_CHEB) {
          // Preconditioner of the FP64 solve: Z = q(A_lp) R, the Chebyshev
          // iteration for A_lp Z = R from Z = 0 on [lo, hi], cheb_steps
          // products with the quantised A (Saad, Iterative Methods for Sparse
          // Linear Systems, Sec. 12.3: Chebyshev acceleration).  The same
          // polynomial for every column; no inner products, so no reductions.
          if (tid == 0) s_int[1] = ldcg(&st->pk);
          __syncthreads();
          const int pk = s_int[1];
          const double th = 0.5 * (prm.cheb_hi + prm.cheb_lo);
          const double de = 0.5 * (prm.cheb_hi - prm.cheb_lo);
          const double sg = th / de;
          double rho = 1.0 / sg;
          double* Z = prm.Z;
          const int64_t cnt = (r1 - r0) * pk;
          if constexpr (POL == POL_FP8) {
            // FP8 operator: the recurrence runs in FP32 (d, S and Z as FP32
            // blocks in the scratch area), and so do the operand split and
            // the fixup; Z is widened to FP64 once, at the end.  The
            // preconditioner needs only the accuracy of the quantised
            // operator (E4M3, about 2^-4 relative with the row scales), and
            // the FP32 rate is 64 times the FP64 rate on GB300.  The column
            // maxima of each new d come from the update itself, as FP32 bit
            // patterns (two buffers: one feeds the next pass while the other
            // fills).
            float* df = reinterpret_cast<float*>(prm.cheb_d);
            float* sf = reinterpret_cast<float*>(prm.cheb_s);
            float* zf = reinterpret_cast<float*>(prm.cheb_w);
            __shared__ unsigned long long s_cf[2][P];
            for (int j = tid; j < 2 * P; j += kThreads) (&s_cf[0][0])[j] = 0ull;
            __syncthreads();
            const float inv_th = (float)(1.0 / th);
            for (int64_t idx = tid; idx < cnt; idx += kThreads) {
              const int64_t o = (r0 + idx / pk) * p + idx % pk;
              const float r = (float)ldcg(prm.V + o);
              const float v = r * inv_th;
              df[o] = v;
              zf[o] = v;
              sf[o] = r;
              atomicMax(&s_cf[0][idx % pk], (unsigned long long)__float_as_uint(fabsf(v)));
            }
            __syncthreads();
            // each step: W = A_lp d ; S -= W ; d = c1 d + c2 S ; Z += d, done
            // on the fixup's entries as they are summed, four columns at a time
            const bool vec4 = (p & 3) == 0;
            int cmb = 0;
            for (int k = 1; k < prm.cheb_steps; ++k) {
              const double rn = 1.0 / (2.0 * sg - rho);
              const float c1 = (float)(rn * rho), c2 = (float)(2.0 * rn / de);
              unsigned long long* cm_next = s_cf[cmb ^ 1];
              for (int j = tid; j < P; j += kThreads) cm_next[j] = 0ull;
              __syncthreads();
              const bool ok = lp_apass_epi<P, POL>(
                  prm, static_cast<const float*>(df), pk, r0, r1, *L, &ss, &s_err, false,
                  [&](int64_t i, int j0, const float (&w)[4], int cn) {
                    const int64_t o = i * p + j0;
                    float sv[4], dv[4], zv[4];
                    if (vec4 && cn == 4) {
                      const float4 s4 = *reinterpret_cast<const float4*>(sf + o);
                      const float4 d4 = *reinterpret_cast<const float4*>(df + o);
                      const float4 z4 = *reinterpret_cast<const float4*>(zf + o);
                      sv[0] = s4.x; sv[1] = s4.y; sv[2] = s4.z; sv[3] = s4.w;
                      dv[0] = d4.x; dv[1] = d4.y; dv[2] = d4.z; dv[3] = d4.w;
                      zv[0] = z4.x; zv[1] = z4.y; zv[2] = z4.z; zv[3] = z4.w;
                    } else {
#pragma unroll
                      for (int u = 0; u < 4; ++u)
                        if (u < cn) {
                          sv[u] = sf[o + u];
                          dv[u] = df[o + u];
                          zv[u] = zf[o + u];
                        }
                    }
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                      if (u < cn) {
                        sv[u] -= w[u];
                        dv[u] = c1 * dv[u] + c2 * sv[u];
                        zv[u] += dv[u];
                        atomicMax(&cm_next[j0 + u],
                                  (unsigned long long)__float_as_uint(fabsf(dv[u])));
                      }
                    }
                    if (vec4 && cn == 4) {
                      *reinterpret_cast<float4*>(sf + o) = make_float4(sv[0], sv[1], sv[2], sv[3]);
                      *reinterpret_cast<float4*>(df + o) = make_float4(dv[0], dv[1], dv[2], dv[3]);
                      *reinterpret_cast<float4*>(zf + o) = make_float4(zv[0], zv[1], zv[2], zv[3]);
                    } else {
#pragma unroll
                      for (int u = 0; u < 4; ++u)
                        if (u < cn) {
                          sf[o + u] = sv[u];
                          df[o + u] = dv[u];
                          zf[o + u] = zv[u];
                        }
                    }
                  },
                  s_cf[cmb]);
              if (!ok) return;
              rho = rn;
              cmb ^= 1;
            }
            for (int64_t idx = tid; idx < cnt; idx += kThreads) {
              const int64_t o = (r0 + idx / pk) * p + idx % pk;
              Z[o] = (double)zf[o];
            }
            return;
          } else {
          double* d = prm.cheb_d;
          double* sr = prm.cheb_s;
          __syncthreads();
          for (int64_t idx = tid; idx < cnt; idx += kThreads) {
            const int64_t o = (r0 + idx / pk) * p + idx % pk;
            const double r = ldcg(prm.V + o);
            const double v = r / th;
            d[o] = v;
            Z[o] = v;
            sr[o] = r;
          }
          __syncthreads();
          // each step: W = A_lp d ; S -= W ; d = c1 d + c2 S ; Z += d, the update
          // done on the fixup's entries as they are summed, four columns at a
          // time; BF16 / TF32 also write the next step's operand rows there (no
          // separate conversion)
          constexpr bool kConvInFixup = POL == POL_BF16 || POL == POL_TF32X3;
          const bool vec2 = (p & 1) == 0;
          bool conv = false;
          for (int k = 1; k < prm.cheb_steps; ++k) {
            const double rn = 1.0 / (2.0 * sg - rho);
            const double c1 = rn * rho, c2 = 2.0 * rn / de;
            const bool conv_next = kConvInFixup && k + 1 < prm.cheb_steps;
            const bool ok = lp_apass_epi<P, POL>(
                prm, d, pk, r0, r1, *L, &ss, &s_err, conv,
                [&](int64_t i, int j0, const double (&w)[4], int cn) {
                  const int64_t o = i * p + j0;
                  double sv[4], dv[4], zv[4];
                  if (vec2 && cn == 4) {
                    const double2 s01 = *reinterpret_cast<const double2*>(sr + o);
                    const double2 s23 = *reinterpret_cast<const double2*>(sr + o + 2);
                    const double2 d01 = *reinterpret_cast<const double2*>(d + o);
                    const double2 d23 = *reinterpret_cast<const double2*>(d + o + 2);
                    const double2 z01 = *reinterpret_cast<const double2*>(Z + o);
                    const double2 z23 = *reinterpret_cast<const double2*>(Z + o + 2);
                    sv[0] = s01.x; sv[1] = s01.y; sv[2] = s23.x; sv[3] = s23.y;
                    dv[0] = d01.x; dv[1] = d01.y; dv[2] = d23.x; dv[3] = d23.y;
                    zv[0] = z01.x; zv[1] = z01.y; zv[2] = z23.x; zv[3] = z23.y;
                  } else {
#pragma unroll
                    for (int u = 0; u < 4; ++u)
                      if (u < cn) {
                        sv[u] = sr[o + u];
                        dv[u] = d[o + u];
                        zv[u] = Z[o + u];
                      }
                  }
#pragma unroll
                  for (int u = 0; u < 4; ++u) {
                    if (u < cn) {
                      sv[u] -= w[u];
                      dv[u] = c1 * dv[u] + c2 * sv[u];
                      zv[u] += dv[u];
                      if (conv_next)
                        lp_put<LpCfg<POL>::KIND, LpNP<P, POL>::value>(prm, j0 + u, i, dv[u]);
                    }
                  }
                  if (vec2 && cn == 4) {
                    *reinterpret_cast<double2*>(sr + o) = make_double2(sv[0], sv[1]);
                    *reinterpret_cast<double2*>(sr + o + 2) = make_double2(sv[2], sv[3]);
                    *reinterpret_cast<double2*>(d + o) = make_double2(dv[0], dv[1]);
                    *reinterpret_cast<double2*>(d + o + 2) = make_double2(dv[2], dv[3]);
                    *reinterpret_cast<double2*>(Z + o) = make_double2(zv[0], zv[1]);
                    *reinterpret_cast<double2*>(Z + o + 2) = make_double2(zv[2], zv[3]);
                  } else {
#pragma unroll
                    for (int u = 0; u < 4; ++u)
                      if (u < cn) {
                        sr[o + u] = sv[u];
                        d[o + u] = dv[u];
                        Z[o + u] = zv[u];
                      }
                  }
                });
            if (!ok) return;
            rho = rn;
            if (conv_next) {
              // the operand rows of every CTA are complete before the next pass
              asm volatile("fence.proxy.async.global;" ::: "memory");
              if (!grid_barrier(prm, &ss, &s_err)) return;
            }
            conv = conv_next;
          }
          return;
          }
        }
      }
    }
    // inner solves only, except the sliced FP64 policy: a full FP64 solve
    if (prm.mode != MODE_SOLVE || (!prm.skip_true_check && POL != POL_SLICED)) {
      if (tid == 0 && cta == 0) set_error(st, ST_ERR_INVALID, 14);
      return;
    }
  }

  // Preconditioned FP64 solve: a serial step that leaves the solve waiting
  // for Z = q(A_lp) R sets st->pc_stage; every CTA then records the direction
  // buffer and leaves, and the next launch (resume = 1) continues.
  const bool pc = kExact && prm.precond;
#define CCG_PC_YIELD(CUR)                                                    \
  if (pc) {                                                                  \
    if (tid == 0) s_int[3] = ldcg(&st->pc_stage);                            \
    __syncthreads();                                                         \
    if (s_int[3] != PC_NONE) {                                               \
      if (tid == 0 && cta == 0) st->cur = (CUR);                             \
      return;                                                                \
    }                                                                        \
  }

  if (!prm.resume) {
  // ---- initial block X_0 and ||b|| ----
  for (int64_t idx = r0 * p + tid; idx < r1 * p; idx += kThreads) {
    const int64_t i = idx / p;
    const int j = (int)(idx - i * p);
    double v;
    if (prm.X0 != nullptr) {
      v = prm.X0[idx];
    } else {
      const double base = prm.x0 ? prm.x0[i] : 0.0;
      if (j == 0) {
        v = base;
      } else {
        const double u = splitmix_uniform(prm.seed, (unsigned long long)j * (unsigned long long)n +
                                                        (unsigned long long)i);
        v = __dadd_rn(base, __dmul_rn(prm.spread, __dsub_rn(2.0 * u, 1.0)));
      }
    }
    prm.X[idx] = v;
  }
  partial_sumsq(prm.b, 1, r0, r1, mypart);
  CCG_SYNC_RED(RED_SCALAR, 1, serial_bnorm(prm, S));

  if (tid == 0) s_int[0] = ldcg(&st->ctrl);
  __syncthreads();
  if (s_int[0] != CTRL_FINISH) {
    // R_0 = A X_0 - b 1^T ; D_0 = R_0
    if constexpr (POL == POL_FP64) {
      apass<P, VEC, VARIANTS>(prm, prm.X, p, 0, p, prm.R, p, true, r0, r1, smem);
    } else if constexpr (POL == POL_F32) {
      if (!apass_f32<P>(prm, prm.X, p, prm.R, true, r0, r1, &ss, &s_err)) return;
    } else {
      if (!lp_apass<P, POL>(prm, prm.X, p, prm.R, true, r0, r1, *L, &ss, &s_err)) return;
    }
    for (int64_t idx = r0 * p + tid; idx < r1 * p; idx += kThreads) prm.D0[idx] = ldcg(prm.R + idx);
    partial_grams<POL == POL_FP64 || POL == POL_SLICED>(nullptr, nullptr, nullptr, nullptr, prm.R, p, p, r0, r1, mypart, smem, kStageDoubles);
    CCG_SYNC_RED(RED_S, p, (serial_norms(prm, S, false), serial_pc_request(prm, PC_SET_D)));
    CCG_PC_YIELD(0);
  }
  }

  int cur = 0;
  // a resumed launch starts with the step its predecessor left waiting for Z
  int pc_stage = PC_NONE;
  if (prm.resume) {
    if (tid == 0) {
      s_int[0] = ldcg(&st->cur);
      s_int[1] = ldcg(&st->pc_stage);
    }
    __syncthreads();
    cur = s_int[0];
    pc_stage = s_int[1];
  }
  // BF16 / TF32 inner solves: the D-update writes D_{k+1} in the MMA type too,
  // and the next tensor-core A-pass skips its conversion and barrier
  constexpr bool kFuseConv = POL == POL_BF16 || POL == POL_TF32X3;
  bool conv_ready = false;
  // sliced FP64 policy: the D-update gathers the column maxima of D_{k+1}
  // over this CTA's rows, so the next A-pass skips its scan of D
  __shared__ unsigned long long s_dmax[P];
  bool dmax_ready = false;
  for (;;) {
    if (tid == 0) {
      s_int[0] = ldcg(&st->ctrl);
      s_int[1] = ldcg(&st->pk);
    }
    __syncthreads();
    const int ctrl = s_int[0];
    int pk = s_int[1];
    double* D = cur ? prm.D1 : prm.D0;
    double* Dn = cur ? prm.D0 : prm.D1;

    if (pc && pc_stage != PC_NONE && ctrl == CTRL_LOOP) {
      const int stage = pc_stage;
      pc_stage = PC_NONE;
      if (stage == PC_SET_D) {
        // D_k = Z_k (after the initial block or a residual replacement); the
        // serial step of the next exchange clears st->pc_stage
        for (int64_t idx = tid; idx < (r1 - r0) * pk; idx += kThreads) {
          const int64_t o = (r0 + idx / pk) * p + idx % pk;
          D[o] = ldcg(prm.Z + o);
        }
        if (!grid_barrier(prm, &ss, &s_err)) return;
      } else {
        // H = Z_{k+1}' A D_k ; beta_k^T = -M^{-1} H^T ; D_{k+1} = Z_{k+1} + D_k beta_k^T
        partial_grams<true>(prm.Z, prm.W, nullptr, nullptr, prm.R, p, pk, r0, r1, mypart, smem,
                            kStageDoubles);
        CCG_SYNC_RED(RED_H_S, pk, serial_beta_pc<P>(prm, S));
        double* Ts = smem;
        for (int e = tid; e < pk * pk; e += kThreads) {
          const int b = e / pk, a = e - b * pk;
          Ts[b * kLd + a] = ldcg(&st->betaT[b * kMaxP + a]);
        }
        __syncthreads();
        const int64_t cnt = (r1 - r0) * pk;
        for (int64_t idx = tid; idx < cnt; idx += kThreads) {
          const int64_t i = r0 + idx / pk;
          const int a = (int)(idx % pk);
          double acc = 0.0;
#pragma unroll 8
          for (int b = 0; b < pk; ++b) acc = fma(ldcg(D + i * p + b), Ts[b * kLd + a], acc);
          Dn[i * p + a] = ldcg(prm.Z + i * p + a) + acc;
        }
        if (!grid_barrier(prm, &ss, &s_err)) return;
        cur ^= 1;
      }
      continue;
    }

    if (ctrl == CTRL_FINISH) {
      const int zero = ldcg(&st->zero_rhs);
      const int jb = ldcg(&st->jbest);
      for (int64_t i = r0 + tid; i < r1; i += kThreads)
        prm.x_out[i] = zero ? 0.0 : ldcg(prm.X + i * p + jb);
      if (prm.X_out != nullptr) {
        for (int64_t idx = r0 * p + tid; idx < r1 * p; idx += kThreads) {
          const int64_t i = idx / p;
          const int c = (int)(idx - i * p);
          if (zero) prm.X_out[idx] = 0.0;
          else if (c < pk) prm.X_out[i * p + ldcg(&st->agent[c])] = ldcg(prm.X + idx);
        }
      }
      return;
    }

    if constexpr (POL != POL_FP64 && POL != POL_SLICED) {
      if (ctrl == CTRL_CHECK || ctrl == CTRL_REPLACE) {  // never reached by inner solves
        if (tid == 0) set_error(st, ST_ERR_INVALID, 15);
        return;
      }
    }

    if (ctrl == CTRL_CHECK) {
      // true residual of the best agent: W[:, 0] = A X e_jb - b
      const int jb = ldcg(&st->jbest);
      if constexpr (POL == POL_FP64 || POL == POL_SLICED) {
        // the FP64 true residual always runs on the FP64 pipe
        apass<1, VEC, VARIANTS>(prm, prm.X, p, jb, 1, prm.W, p, true, r0, r1, smem);
        partial_sumsq(prm.W, p, r0, r1, mypart);
        CCG_SYNC_RED(RED_SCALAR, 1, serial_check(prm));
      }
      continue;
    }

    if (ctrl == CTRL_REPLACE) {
      if constexpr (POL == POL_FP64) {
        apass<P, VEC, VARIANTS>(prm, prm.X, p, 0, pk, prm.R, p, true, r0, r1, smem);
      } else if constexpr (POL == POL_SLICED) {
        if (!lp_apass<P, POL>(prm, prm.X, pk, prm.R, true, r0, r1, *L, &ss, &s_err)) return;
      }
      for (int64_t idx = r0 * p + tid; idx < r1 * p; idx += kThreads) {
        const int c = (int)(idx % p);
        if (c < pk) D[idx] = ldcg(prm.R + idx);
      }
      partial_grams<POL == POL_FP64 || POL == POL_SLICED>(nullptr, nullptr, nullptr, nullptr, prm.R, p, pk, r0, r1, mypart, smem, kStageDoubles);
      CCG_SYNC_RED(RED_S, pk, (serial_norms(prm, S, true), serial_pc_request(prm, PC_SET_D)));
      CCG_PC_YIELD(cur);
      continue;
    }

    // ---- one cCG iteration ----
    if constexpr (POL == POL_FP64) {
      apass<P, VEC, VARIANTS>(prm, D, p, 0, pk, prm.W, p, false, r0, r1, smem);
    } else if constexpr (POL == POL_F32) {
      if (!apass_f32<P>(prm, D, pk, prm.W, false, r0, r1, &ss, &s_err)) return;
    } else {
      if (!lp_apass<P, POL>(prm, D, pk, prm.W, false, r0, r1, *L, &ss, &s_err, conv_ready,
                            dmax_ready ? s_dmax : nullptr))
        return;
      dmax_ready = false;
    }
    partial_grams<POL == POL_FP64 || POL == POL_SLICED>(D, prm.W, prm.R, D, nullptr, p, pk, r0, r1, mypart, smem, kStageDoubles);
    CCG_SYNC_RED(RED_M_G, pk, (serial_alpha<P, !kExact>(prm, S), serial_pc_clear(prm)));

    if (tid == 0) {
      s_int[2] = ldcg(&st->changed);
      s_int[1] = ldcg(&st->pk);
      s_int[3] = ldcg(&st->prev_pk);
    }
    __syncthreads();
    if (s_int[2]) {
      // restrict X, R, D, W to the kept agents (own rows, in place)
      const int m = s_int[1];
      const int ppk = s_int[3];
      int* keep = reinterpret_cast<int*>(smem);
      int* oldag = keep + kMaxP;
      if (tid < ppk) {
        keep[tid] = tid < m ? ldcg(&st->keep[tid]) : 0;
        oldag[tid] = ldcg(&st->old_agent[tid]);
      }
      __syncthreads();
      for (int64_t i = r0 + tid; i < r1; i += kThreads) {
        double* rows[4] = {prm.X + i * p, prm.R + i * p, D + i * p, prm.W + i * p};
        if (prm.X_out != nullptr) {
          int t = 0;
          for (int c = 0; c < ppk; ++c) {
            if (t < m && keep[t] == c) { ++t; continue; }
            prm.X_out[i * p + oldag[c]] = rows[0][c];
          }
        }
        for (int r = 0; r < 4; ++r)
          for (int c = 0; c < m; ++c) rows[r][c] = rows[r][keep[c]];
      }
      __syncthreads();
    }
    pk = s_int[1];

    // X += D alpha^T ; R += W alpha^T (or, explicit residual, R = A X - b 1^T
    // after a grid barrier: every CTA's rows of X are needed)
    {
      double* Ts = smem;
      for (int e = tid; e < pk * pk; e += kThreads) {
        const int b = e / pk, a = e - b * pk;
        Ts[b * kLd + a] = ldcg(&st->alphaT[b * kMaxP + a]);
      }
      __syncthreads();
      const bool rec = !prm.explicit_residual;
      const int64_t cnt = (r1 - r0) * pk;
      for (int64_t idx = tid; idx < cnt; idx += kThreads) {
        const int64_t i = r0 + idx / pk;
        const int a = (int)(idx % pk);
        double dx = 0.0, dr = 0.0;
#pragma unroll 8
        for (int b = 0; b < pk; ++b) {
          const double t = Ts[b * kLd + a];
          dx = fma(ldcg(D + i * p + b), t, dx);
          if (rec) dr = fma(ldcg(prm.W + i * p + b), t, dr);
        }
        prm.X[i * p + a] += dx;
        if (rec) prm.R[i * p + a] += dr;
      }
      __syncthreads();
      if constexpr (POL == POL_FP64) {
        if (!rec) {
          if (!grid_barrier(prm, &ss, &s_err)) return;
          apass<P, VEC, VARIANTS>(prm, prm.X, p, 0, pk, prm.R, p, true, r0, r1, smem);
        }
      }
    }
    if (pc) {
      // residual norms and the stop test now; beta_k once Z_{k+1} is there
      partial_grams<true>(nullptr, nullptr, nullptr, nullptr, prm.R, p, pk, r0, r1, mypart, smem,
                          kStageDoubles);
      CCG_SYNC_RED(RED_S, pk, (serial_kstop(prm, S), serial_pc_request(prm, PC_BETA)));
      CCG_PC_YIELD(cur);
      continue;
    }
    partial_grams<POL == POL_FP64 || POL == POL_SLICED>(prm.R, prm.W, nullptr, nullptr, prm.R, p, pk, r0, r1, mypart, smem, kStageDoubles);
    CCG_SYNC_RED(RED_H_S, pk, serial_beta<P>(prm, S));

    if (tid == 0) s_int[0] = ldcg(&st->ctrl);
    __syncthreads();
    if (s_int[0] == CTRL_LOOP) {
      // D_{k+1} = R_{k+1} + D_k beta^T
      double* Ts = smem;
      for (int e = tid; e < pk * pk; e += kThreads) {
        const int b = e / pk, a = e - b * pk;
        Ts[b * kLd + a] = ldcg(&st->betaT[b * kMaxP + a]);
      }
      __syncthreads();
      constexpr bool kMaxD = POL == POL_SLICED;
      if constexpr (kMaxD) {
        for (int j = tid; j < P; j += kThreads) s_dmax[j] = 0ull;
        __syncthreads();
      }
      const int64_t cnt = (r1 - r0) * pk;
      for (int64_t idx = tid; idx < cnt; idx += kThreads) {
        const int64_t i = r0 + idx / pk;
        const int a = (int)(idx % pk);
        double acc = 0.0;
#pragma unroll 8
        for (int b = 0; b < pk; ++b) acc = fma(ldcg(D + i * p + b), Ts[b * kLd + a], acc);
        const double v = ldcg(prm.R + i * p + a) + acc;
        Dn[i * p + a] = v;
        if constexpr (kFuseConv) lp_put<LpCfg<POL>::KIND, LpNP<P, POL>::value>(prm, a, i, v);
        if constexpr (kMaxD)
          atomicMax(&s_dmax[a], (unsigned long long)__double_as_longlong(fabs(v)));
      }
      if constexpr (kFuseConv) {
        // operand rows of the inactive columns stay zero
        constexpr int NP = LpNP<P, POL>::value;
        const int64_t nz = (r1 - r0) * (NP - pk);
        for (int64_t idx = tid; idx < nz; idx += kThreads) {
          const int j = pk + (int)(idx / (r1 - r0));
          lp_put<LpCfg<POL>::KIND, NP>(prm, j, r0 + idx % (r1 - r0), 0.0);
        }
        asm volatile("fence.proxy.async.global;" ::: "memory");
      }
      if constexpr (kMaxD) {
        // no grid barrier: the next A-pass starts with the grid-wide
        // reduction of the column maxima, its slicing reads this CTA's rows
        // only, and a grid barrier follows the slicing
        __syncthreads();
        dmax_ready = true;
      } else {
        if (!grid_barrier(prm, &ss, &s_err)) return;
      }
      conv_ready = kFuseConv;
      cur ^= 1;
    }
  }
#undef CCG_PC_YIELD
#undef CCG_SYNC_RED
}


template <int P, bool VEC, int POL>
__global__ void __launch_bounds__(kThreads, 1) fp64_kernel(const __grid_constant__ Params prm) {
  extern __shared__ __align__(1024) uint8_t dyn_smem[];
  if constexpr (POL == POL_FP64) {
    solve_body<P, VEC, POL>(prm, reinterpret_cast<double*>(dyn_smem), nullptr);
  } else {
    constexpr int KIND = LpCfg<POL>::KIND;
    constexpr int NP = LpNP<P, POL>::value;
    using Lay = LpLayout<KIND, NP>;
    using S = tc::Shape<KIND, NP>;
    uint8_t* base = reinterpret_cast<uint8_t*>(
        (reinterpret_cast<uintptr_t>(dyn_smem) + 1023) & ~uintptr_t(1023));
    LpCtx L;
    L.ring = base;
    L.bars = reinterpret_cast<uint64_t*>(base + S::kRingBytes);
    L.sh = reinterpret_cast<LpShared*>(L.bars + Lay::kBars);
    double* uni = reinterpret_cast<double*>(
        (reinterpret_cast<uintptr_t>(L.sh + 1) + 15) & ~uintptr_t(15));
    const int warp = threadIdx.x >> 5;
    constexpr int ST = S::kStagesK;
    uint64_t* drain = L.bars + 3 * ST + 4;
    if (threadIdx.x == 0) {
      for (int s = 0; s < ST; ++s) {
        tc::mbar_init(tc::smem_u32(&L.bars[s]), 1);           // full: TMA bytes
        tc::mbar_init(tc::smem_u32(&L.bars[ST + s]), 1);      // empty: MMA commit
        tc::mbar_init(tc::smem_u32(&L.bars[2 * ST + s]), 2);  // split: two warps
      }
      for (int s = 0; s < tc::kStages; ++s) L.sh->issued[s] = -1;
      for (int b = 0; b < 2; ++b) {
        tc::mbar_init(tc::smem_u32(&L.bars[3 * ST + b]), 1);
        tc::mbar_init(tc::smem_u32(&L.bars[3 * ST + 2 + b]), 4);
      }
      tc::mbar_init(tc::smem_u32(drain), 1);
      L.sh->p_stage = 0;
      L.sh->p_phase = 0;
      L.sh->m_stage = 0;
      L.sh->m_phase = 0;
      L.sh->m_seg = 0;
      L.sh->m_any = 0;
      for (int q = 0; q < 4; ++q) L.sh->e_seg[q] = 0;
      for (int q = 0; q < 2; ++q) {
        L.sh->s_stage[q] = 0;
        L.sh->s_phase[q] = 0;
      }
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) {
      asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                       tc::smem_u32(&L.sh->tmem)),
                   "r"(S::kTmemCols)
                   : "memory");
      asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();

    solve_body<P, VEC, POL>(prm, uni, &L);

    // teardown: this CTA's copies and MMAs complete before TMEM is freed
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int s = 0; s < ST; ++s)
        if (L.sh->issued[s] >= 0)
          mbar_wait_drain(tc::smem_u32(&L.bars[s]), (uint32_t)L.sh->issued[s], prm.timeout_ns);
    }
    if (threadIdx.x == 32 && L.sh->m_any) {
      tc::mma_commit(tc::smem_u32(drain));
      mbar_wait_drain(tc::smem_u32(drain), 0u, prm.timeout_ns);
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    if (warp == 1) {
      asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(L.sh->tmem),
                   "r"(S::kTmemCols)
                   : "memory");
    }
  }
}

// Batched solver: each CTA repeatedly takes the next system from the queue
// (largest first, as ordered by the host) and solves it alone -- the solver
// body with a group of one CTA, whose barriers are CTA barriers.
// Out-of-line copies of the solve body for the batched kernels: the batched
// refinement kernel runs two policies, and separate calls keep each one's
// register allocation its own.
template <int P, bool VEC, int POL>
__device__ __noinline__ void solve_call(const Params& prm, double* smem) {
  solve_body<P, VEC, POL, true>(prm, smem, nullptr);
}

// Fresh solver state for one system of a batch (thread 0).
__device__ void reset_state(DevState* st, int p) {
  st->bar_count = 0;
  st->bar_gen = 0;
  st->error = 0;
  st->result = 0;
  st->ctrl = 0;
  st->k = 0;
  st->pk = p;
  st->prev_pk = p;
  st->changed = 0;
  st->jbest = 0;
  st->replacements = 0;
  st->drops = 0;
  st->k_replaced = -1;
  st->zero_rhs = 0;
  st->relres_true = 0.0;
  for (int j = 0; j < kMaxP; ++j) st->agent[j] = j;
}

// Per-system parameters of a batched solve (thread 0; q in shared memory).
__device__ void batch_params(const Params& prm, Params& q, long long i, size_t slot) {
  const int64_t* d = prm.batch_desc + 4 * i;  // n, A offset, vector offset, index
  q = prm;
  q.n = d[0];
  q.lda = d[0] + (d[0] & 1);
  q.A = prm.A + d[1];
  q.b = prm.b + d[2];
  q.x_out = prm.x_out + d[2];
  double* w = prm.X + slot * (size_t)prm.batch_slot_stride;
  const size_t blk = (size_t)prm.batch_slot_stride / 5;
  q.X = w;
  q.R = w + blk;
  q.D0 = w + 2 * blk;
  q.D1 = w + 3 * blk;
  q.W = w + 4 * blk;
  q.part = prm.part + slot * kPartStride;
  q.st = prm.st + slot;
  q.expected_ctas = 1u;
  q.group_ctas = 1;
  q.group_rank = 0;
  // A-pass variant of the system's size bucket: [2^(b+5), 2^(b+6)), b in 0..7
  int b = 31 - __clz((unsigned)(d[0] > 0 ? d[0] : 1)) - 5;
  b = b < 0 ? 0 : (b > 7 ? 7 : b);
  q.apass_variant = prm.batch_variant[b];
}

// Batched solver: each CTA takes systems from a queue (largest first) and
// solves them one at a time as a group of one CTA (grid barriers become CTA
// barriers).
template <int P>
__global__ void __launch_bounds__(kThreads, 1) batch_kernel(const __grid_constant__ Params prm) {
  extern __shared__ __align__(1024) uint8_t dyn_smem[];
  __shared__ Params q;
  __shared__ long long s_sys;
  const int tid = threadIdx.x;
  const size_t slot = blockIdx.x;
  for (;;) {
    if (tid == 0) s_sys = (long long)atomicAdd(prm.batch_next, 1u);
    __syncthreads();
    const long long i = s_sys;
    if (i >= prm.batch_count) break;
    if (tid == 0) {
      batch_params(prm, q, i, slot);
      reset_state(q.st, prm.p);
      __threadfence();
    }
    __syncthreads();
    solve_body<P, false, POL_FP64, true>(q, reinterpret_cast<double*>(dyn_smem), nullptr);
    __syncthreads();
    if (tid == 0) {
      const DevState* st = q.st;
      const int64_t idx = prm.batch_desc[4 * i + 3];
      const int err = *(volatile const int*)&st->error;
      prm.batch_status[idx] = err != 0 ? err : *(volatile const int*)&st->result;
      prm.batch_iters[idx] = *(volatile const int*)&st->k;
      prm.batch_relres[idx] = *(volatile const double*)&st->relres_true;
    }
    __syncthreads();
  }
}

// Batched mixed-precision solver: per system, an FP32 copy of A, then FP64
// iterative refinement (x += d; r = b - A x in FP64) around inner cCG solves
// on the FP32 copy (A-pass on the FP32 pipe), all inside one launch.  The
// refinement ends when the true relative residual reaches tol, when two
// steps in a row fail to reduce it, after batch_max_outer steps, or when the
// inner solve breaks down; the best x is returned.
template <int P>
__global__ void __launch_bounds__(kThreads, 1) batch_ir_kernel(const __grid_constant__ Params prm) {
  extern __shared__ __align__(1024) uint8_t dyn_smem[];
  __shared__ Params q;
  __shared__ long long s_sys;
  double* smem = reinterpret_cast<double*>(dyn_smem);
  const int tid = threadIdx.x;
  const size_t slot = blockIdx.x;
  for (;;) {
    if (tid == 0) s_sys = (long long)atomicAdd(prm.batch_next, 1u);
    __syncthreads();
    const long long i = s_sys;
    if (i >= prm.batch_count) break;
    if (tid == 0) {
      batch_params(prm, q, i, slot);
      double* v = prm.batch_vec + slot * (size_t)prm.batch_vec_stride;
      const int64_t n = q.n;
      q.ref_x = q.x_out;
      q.ref_r = v;
      q.ref_bin = v + n;
      q.ref_delta = nullptr;
      q.ref_coef = 0.0;
      q.a32_ld = (n + 3) & ~int64_t(3);
      float* f = prm.batch_f32 + slot * (size_t)prm.batch_f32_stride;
      q.a32 = f;
      q.vt32 = f + n * q.a32_ld;
    }
    __syncthreads();
    const int64_t n = q.n;
    const int64_t ld = q.a32_ld;
    double* xs = q.x_out;
    double* delta = q.ref_bin + n;
    double* xbest = delta + n;
    const double* bsys = q.b;
    {
      // FP32 copy of A (zero padding to ld), zero operand padding, x = 0
      float* a32 = const_cast<float*>(q.a32);
      for (int64_t idx = tid; idx < n * ld; idx += kThreads) {
        const int64_t r = idx / ld, c = idx - r * ld;
        a32[idx] = c < n ? (float)q.A[r * q.lda + c] : 0.f;
      }
      for (int64_t idx = tid; idx < (int64_t)P * (ld - n); idx += kThreads) {
        const int64_t c = idx / (ld - n), k = n + (idx - c * (ld - n));
        q.vt32[c * ld + k] = 0.f;
      }
      for (int64_t r = tid; r < n; r += kThreads) xs[r] = 0.0;
    }
    // r = b - A x, norms
    if (tid == 0) {
      reset_state(q.st, 1);
      q.mode = MODE_REFINE;
      q.p = 1;
      __threadfence();
    }
    __syncthreads();
    solve_call<P, false, POL_FP64>(q, smem);
    __syncthreads();
    const DevState* st = q.st;
    int err = ldcg(&st->error);
    double rnorm = ldcg(&st->rnorm);
    double relres = ldcg(&st->relres_true);
    const double bnorm = ldcg(&st->bnorm);
    double best = relres;
    for (int64_t r = tid; r < n; r += kThreads) xbest[r] = xs[r];
    int status = (err != 0) ? err : ((bnorm == 0.0 || relres <= prm.tol) ? ST_OK : ST_NOT_CONVERGED);
    int total = 0, outer = 0, stall = 0;
    while (status == ST_NOT_CONVERGED && outer < prm.batch_max_outer && total < prm.maxit) {
      ++outer;
      __syncthreads();
      if (tid == 0) {
        // inner solve A32 d = b_in (unit-RMS right-hand side), recurrence stop
        reset_state(q.st, prm.p);
        q.mode = MODE_SOLVE;
        q.p = prm.p;
        q.b = q.ref_bin;
        q.x_out = delta;
        q.skip_true_check = 1;
        q.replacement = 0;
        q.tol = fmax(prm.batch_inner_tol, 0.5 * prm.tol / relres);
        q.maxit = prm.maxit - total;
        __threadfence();
      }
      __syncthreads();
      solve_call<P, false, POL_F32>(q, smem);
      __syncthreads();
      err = ldcg(&st->error);
      if (err == ST_ERR_NOT_SPD || err == ST_ERR_NUMERICAL) break;  // inner breakdown
      if (err != 0) {
        status = err;
        break;
      }
      total += ldcg(&st->k);
      // x += d ||r|| / sqrt(n) ; r = b - A x (FP64)
      __syncthreads();
      if (tid == 0) {
        reset_state(q.st, 1);
        q.mode = MODE_REFINE;
        q.p = 1;
        q.b = bsys;
        q.x_out = xs;
        q.ref_delta = delta;
        q.ref_coef = rnorm / sqrt((double)n);
        __threadfence();
      }
      __syncthreads();
      solve_call<P, false, POL_FP64>(q, smem);
      __syncthreads();
      err = ldcg(&st->error);
      if (err != 0) {
        status = err;
        break;
      }
      rnorm = ldcg(&st->rnorm);
      relres = ldcg(&st->relres_true);
      if (relres < best) {
        best = relres;
        stall = 0;
        for (int64_t r = tid; r < n; r += kThreads) xbest[r] = xs[r];
      } else if (++stall >= 2) {
        break;
      }
      if (best <= prm.tol) status = ST_OK;
    }
    __syncthreads();
    for (int64_t r = tid; r < n; r += kThreads) xs[r] = xbest[r];
    if (tid == 0) {
      const int64_t idx = prm.batch_desc[4 * i + 3];
      prm.batch_status[idx] = (status == ST_NOT_CONVERGED && best <= prm.tol) ? ST_OK : status;
      prm.batch_iters[idx] = total;
      prm.batch_relres[idx] = best;
      if (prm.batch_outer) prm.batch_outer[idx] = outer;
    }
    __syncthreads();
  }
}

// --------------------------------------------------------------------------
// Serving kernel: continuous batching of solve requests.  The grid is split
// into slots of serve_group CTAs.  The first CTA of a slot takes the next
// request from a ring in host memory that the host appends to while the
// kernel runs, and hands its position to the other CTAs of the slot; the
// slot solves it (the solver body with a group of serve_group CTAs, the
// slot's state and workspace, A, b and x where the request points), writes
// the result into the ring entry and takes the next request.  Requests of
// all slots advance concurrently in this one launch; a request posted while
// others run starts as soon as a slot frees up.  The kernel ends once the
// host asks it to stop, or after serve_idle_ns with nothing to claim and no
// slot busy; every wait is bounded.
// --------------------------------------------------------------------------
__device__ __forceinline__ int ld_acquire_sys_i32(const int* p) {
  int v;
  asm volatile("ld.acquire.sys.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ long long ld_acquire_sys_i64(const int64_t* p) {
  long long v;
  asm volatile("ld.acquire.sys.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_sys_i64(int64_t* p, long long v) {
  asm volatile("st.release.sys.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Leader of a slot: the ring position of the next request, or -1 (leave).
__device__ int serve_claim(const Params& prm) {
  ServeCtl* ctl = prm.serve_ctl;
  const unsigned long long t0 = globaltimer_ns();
  for (;;) {
    if (*(volatile int*)&ctl->closing != 0 || *(volatile int*)&ctl->error != 0) return -1;
    const unsigned h = ld_acquire_u32(&ctl->head);
    const int t = ld_acquire_sys_i32(prm.serve_tail);
    if ((int)h < t) {
      if (atomicCAS(&ctl->head, h, h + 1u) == h) {
        atomicAdd(&ctl->busy, 1);
        return (int)h;
      }
      continue;
    }
    const bool stop = ld_acquire_sys_i32(prm.serve_stop) != 0;
    const unsigned long long waited = globaltimer_ns() - t0;
    const bool idle = waited > (unsigned long long)prm.serve_idle_ns;
    if ((stop || idle) && *(volatile int*)&ctl->busy == 0) {
      atomicExch(&ctl->closing, 1);
      return -1;
    }
    // other slots are busy, but this one has waited timeout_ns for work: it
    // leaves (the kernel ends once the others do, and the host launches it
    // again for new requests)
    if (waited > (unsigned long long)prm.timeout_ns) return -1;
    __nanosleep(500);
  }
}

template <int P>
__global__ void __launch_bounds__(kThreads, 1) serve_kernel(const __grid_constant__ Params prm) {
  extern __shared__ __align__(1024) uint8_t dyn_smem[];
  __shared__ Params q;
  __shared__ int s_ticket;
  const int tid = threadIdx.x;
  const int C = prm.serve_group;
  const int slot = (int)blockIdx.x / C;
  const int rank = (int)blockIdx.x - slot * C;
  SlotSync* sy = prm.serve_sync + slot;
  ServeCtl* ctl = prm.serve_ctl;
  DevState* st = prm.st + slot;
  // a follower waits at most as long as its leader may wait for work, plus
  // the time to check the ring entry
  const long long wait_ns = 2 * prm.timeout_ns + prm.serve_idle_ns;
  unsigned gen = 0;
  for (;;) {
    // ---- the leader claims; the slot learns the ticket ----
    if (tid == 0) {
      int ticket = -1;
      if (rank == 0) {
        ticket = serve_claim(prm);
        if (ticket >= 0) {
          const ServeDesc* d = prm.serve_desc + ticket % prm.serve_capacity;
          // the host writes the entry before it moves the tail past it
          const unsigned long long t0 = globaltimer_ns();
          while (ld_acquire_sys_i64(&d->seq) != (long long)ticket + 1) {
            if (globaltimer_ns() - t0 > (unsigned long long)prm.timeout_ns) {
              atomicExch(&ctl->error, ST_ERR_TIMEOUT);
              atomicSub(&ctl->busy, 1);
              ticket = -1;
              break;
            }
          }
        }
        if (ticket >= 0) {
          const ServeDesc* d = prm.serve_desc + ticket % prm.serve_capacity;
          reset_state(st, *(volatile const int*)&d->p);
          ServeOut* o = prm.serve_out + ticket % prm.serve_capacity;
          o->slot = slot;
          o->t_start_ns = (long long)globaltimer_ns();
          __threadfence_system();
          st_release_sys_i64(&o->claimed, (long long)ticket + 1);
        }
        sy->ticket = ticket;
        __threadfence();
        st_release_u32(&sy->gen, gen + 1u);
      } else {
        const unsigned long long t0 = globaltimer_ns();
        while (ld_acquire_u32(&sy->gen) == gen) {
          if (globaltimer_ns() - t0 > (unsigned long long)wait_ns) {
            atomicExch(&ctl->error, ST_ERR_TIMEOUT);
            break;
          }
          __nanosleep(200);
        }
        ticket = (ld_acquire_u32(&sy->gen) == gen) ? -1 : ldcg(&sy->ticket);
      }
      s_ticket = ticket;
    }
    __syncthreads();
    ++gen;
    const int ticket = s_ticket;
    if (ticket < 0) return;

    // ---- the request's parameters: the slot's state and workspace ----
    if (tid == 0) {
      // the ring entry through volatile loads: the host reuses entries
      const volatile ServeDesc* d = prm.serve_desc + ticket % prm.serve_capacity;
      q = prm;
      q.n = d->n;
      q.lda = d->lda;
      q.A = d->A;
      q.b = d->b;
      q.x_out = d->x;
      q.tol = d->tol;
      q.maxit = d->maxit;
      q.p = d->p;
      q.x0 = nullptr;
      q.X0 = nullptr;
      q.X_out = nullptr;
      double* w = prm.X + (size_t)slot * (size_t)prm.serve_ws_stride;
      const size_t blk = (size_t)prm.serve_ws_stride / 5;
      q.X = w;
      q.R = w + blk;
      q.D0 = w + 2 * blk;
      q.D1 = w + 3 * blk;
      q.W = w + 4 * blk;
      q.part = prm.part + (size_t)slot * C * kPartStride;
      q.st = st;
      q.expected_ctas = (unsigned)C;
      q.group_ctas = C;
      q.group_rank = rank;
      q.mode = MODE_SOLVE;
    }
    __syncthreads();
    // the leader's reset of the state is visible: it was fenced before the
    // ticket went out, and the other CTAs read it after the ticket
    solve_body<P, true, POL_FP64, false>(q, reinterpret_cast<double*>(dyn_smem), nullptr);
    __syncthreads();

    // ---- the slot reports the result and frees up ----
    if (tid == 0) {
      __threadfence();
      atom_add_acqrel_u32(&sy->count, 1u);
      if (rank == 0) {
        const unsigned long long t0 = globaltimer_ns();
        bool ok = true;
        while (ld_acquire_u32(&sy->count) != (unsigned)C) {
          if (globaltimer_ns() - t0 > (unsigned long long)prm.timeout_ns) {
            atomicExch(&ctl->error, ST_ERR_TIMEOUT);
            ok = false;
            break;
          }
        }
        sy->count = 0u;
        ServeOut* o = prm.serve_out + ticket % prm.serve_capacity;
        const int err = *(volatile const int*)&st->error;
        o->status = !ok ? ST_ERR_TIMEOUT : (err != 0 ? err : *(volatile const int*)&st->result);
        o->iterations = *(volatile const int*)&st->k;
        o->relres_true = *(volatile const double*)&st->relres_true;
        o->t_end_ns = (long long)globaltimer_ns();
        __threadfence_system();
        st_release_sys_i64(&o->done, (long long)ticket + 1);
        atomicSub(&ctl->busy, 1);
      }
    }
    __syncthreads();
  }
}

template <int P>
constexpr size_t vs_bytes() {
  return 2 * sizeof(double) * (size_t)P * Tile<P>::VSTR;
}

// Dynamic shared memory of fp64_kernel<P, *, POL>.
template <int P, int POL>
constexpr size_t solver_smem_bytes() {
  size_t b = vs_bytes<P>() > sizeof(SerialSmem) ? vs_bytes<P>() : sizeof(SerialSmem);
  if (b < vs_bytes<1>()) b = vs_bytes<1>();  // CHECK / REFINE use the P = 1 tile
  b = (b + 15) & ~size_t(15);
  if constexpr (POL == POL_FP64) {
    return b;
  } else {
    return LpLayout<LpCfg<POL>::KIND, LpNP<P, POL>::value>::kBytes + b;
  }
}

template <int P, bool VEC, int POL>
void* kernel_ptr() {
  // dynamic + static shared memory within the 227 KB a CTA may hold
  static_assert(solver_smem_bytes<P, POL>() + 2048 <= 232448, "shared memory budget");
  return reinterpret_cast<void*>(&fp64_kernel<P, VEC, POL>);
}

}  // namespace
}  // namespace ccg
