// ccg_fp64.cu -- persistent FP64 solver kernel for the cooperative conjugate
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
//   sync #1  last-arriving CTA: fixed-order sum of the partials, scaled
//            Cholesky of M with the rank test of Algorithm 3, alpha_k
//   update   X += D alpha^T, R += W alpha^T (recurrence, proof of Thm. 2);
//            partials of H = R_{k+1}'W and ||R_{k+1} e_j||^2  (Table 1, rows 5-7)
//   sync #2  last-arriving CTA: beta_k, stop test min_j ||R e_j|| <= tol ||b||
//   D-update D_{k+1} = R_{k+1} + D_k beta^T                  (Table 1, row 9)
//   barrier
//
// The p x p Grams and the norms are inner products that the method treats as
// exact (Sec. 4 works in exact arithmetic); they decide the matrix stepsizes
// and the stop test, so they are accumulated with error-free transformations
// (Dot2 of Ogita, Rump and Oishi 2005: exact products by FMA, TwoSum for the
// running sum) per CTA and again across CTAs.  All cross-CTA sums run in a
// fixed order (CTA 0, 1, ...), so a solve is bitwise reproducible for a fixed
// grid.  Every wait on another CTA gives up
// after Params::timeout_ns and sets CCG_ERR_TIMEOUT; all CTAs then return.
#include <cstdint>
#include <cuda_runtime.h>

#include "ccg_internal.h"

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

// Compensated accumulation (Dot2).  The intrinsics keep the compiler from
// contracting the error-free transformations into FMAs.
struct DSum {
  double hi;
  double lo;
};
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

__device__ int grid_arrive(const Params& prm, SyncShared* ss) {
  __syncthreads();
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
      while (ld_acquire_u32(&st->bar_gen) == gen) {
        if (*(volatile int*)&st->error != 0) { flag = -1; break; }
        if (globaltimer_ns() - t0 > (unsigned long long)prm.timeout_ns) {
          set_error(st, ST_ERR_TIMEOUT, 100);
          flag = -1;
          break;
        }
        __nanosleep(64);
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

// Plain barrier; false = leave the kernel.
__device__ bool grid_barrier(const Params& prm, SyncShared* ss, int* s_err) {
  const int f = grid_arrive(prm, ss);
  if (f < 0) return false;
  if (f == 1) grid_release(prm, ss);
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

// Y[row, c] = sum_k A[row, k] V[k, coff + c] (- b[row]) for the rows
// [r0, r1) and c < pk.  Vs: shared scratch of 2 * P * VSTR doubles.
template <int P, bool VEC>
__device__ void apass(const Params& prm, const double* __restrict__ V, int ldv,
                      int coff, int pk, double* __restrict__ Y, int ldy,
                      bool sub_b, int64_t r0, int64_t r1, double* Vs) {
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
// Each entry is one thread's compensated sum over i in row order (hi at
// [slot], lo at [kPartHalf + slot]).
__device__ void partial_grams(const double* U0, const double* V0, const double* U1,
                              const double* V1, const double* S, int ld, int pk,
                              int64_t r0, int64_t r1, double* out) {
  const int sq = pk * pk;
  const int total = 2 * sq + pk;
  for (int e = threadIdx.x; e < total; e += kThreads) {
    const double* U;
    const double* Vv;
    int a, c, slot;
    if (e < sq) {
      U = U0; Vv = V0; a = e / pk; c = e - a * pk; slot = kSlotGram0 + a * kMaxP + c;
    } else if (e < 2 * sq) {
      const int f = e - sq;
      U = U1; Vv = V1; a = f / pk; c = f - a * pk; slot = kSlotGram1 + a * kMaxP + c;
    } else {
      U = S; Vv = S; a = c = e - 2 * sq; slot = kSlotVec + a;
    }
    if (U == nullptr) continue;
    DSum t{0.0, 0.0};
    for (int64_t i = r0; i < r1; ++i) dsum_fma(t, ldcg(U + i * ld + a), ldcg(Vv + i * ld + c));
    out[slot] = t.hi;
    out[kPartHalf + slot] = t.lo;
  }
}

// Per-CTA compensated sum of squares of x[i * ld] over the rows [r0, r1)
// by warp 0, into the scalar slot.
__device__ void partial_sumsq(const double* x, int ld, int64_t r0, int64_t r1, double* out) {
  if (threadIdx.x < 32) {
    DSum t{0.0, 0.0};
    for (int64_t i = r0 + threadIdx.x; i < r1; i += 32) {
      const double v = ldcg(x + i * ld);
      dsum_fma(t, v, v);
    }
    t = dsum_warp(t);
    if (threadIdx.x == 0) {
      out[kSlotScalar] = t.hi;
      out[kPartHalf + kSlotScalar] = t.lo;
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
  int keep[kMaxP];
  int flag[4];
};

// Compensated sum of a slot entry over the CTAs, in CTA order.
__device__ __forceinline__ double sum_parts(const Params& prm, int off) {
  DSum t{0.0, 0.0};
  const int G = gridDim.x;
  for (int g = 0; g < G; ++g) {
    const double* q = prm.part + (size_t)g * kPartStride;
    dsum_add(t, ldcg(q + off), ldcg(q + kPartHalf + off));
  }
  return __dadd_rn(t.hi, t.lo);
}

// Y <- L^{-T} L^{-1} Y for m right-hand sides (thread per column), L lower.
__device__ void chol_solve_cols(const double* l, double* y, int m) {
  const int c = threadIdx.x;
  if (c < m) {
    for (int a = 0; a < m; ++a) {
      double v = y[a * kLd + c];
      for (int u = 0; u < a; ++u) v -= l[a * kLd + u] * y[u * kLd + c];
      y[a * kLd + c] = v / l[a * kLd + a];
    }
    for (int a = m - 1; a >= 0; --a) {
      double v = y[a * kLd + c];
      for (int u = a + 1; u < m; ++u) v -= l[u * kLd + a] * y[u * kLd + c];
      y[a * kLd + c] = v / l[a * kLd + a];
    }
  }
  __syncthreads();
}

__device__ __forceinline__ bool finite(double v) { return isfinite(v); }

// Stop test on the residual norms s2 (squared), shared by the init, beta and
// replacement steps: sets s, jbest, relres_recur and the next ctrl.
__device__ void stop_test(const Params& prm, SerialSmem& S, int pk, int where) {
  DevState* st = prm.st;
  if (threadIdx.x == 0) {
    bool bad = false;
    int jmin = 0;
    for (int j = 0; j < pk; ++j) {
      const double s = sqrt(S.s2[j]);
      st->s[j] = s;
      if (!finite(s)) bad = true;
      if (j > 0 && s < sqrt(S.s2[jmin])) jmin = j;
    }
    if (bad) {
      set_error(st, ST_ERR_NUMERICAL, where);
    } else {
      const double smin = sqrt(S.s2[jmin]);
      const double bn = ldcg(&st->bnorm);
      const bool stop = smin <= prm.tol * bn;
      st->jbest = jmin;
      st->relres_recur = smin / bn;
      st->ctrl = (stop || ldcg(&st->k) >= prm.maxit) ? CTRL_CHECK : CTRL_LOOP;
    }
  }
  __syncthreads();
}

// alpha step: M, G -> rank test, factor, alpha_k^T (Algorithm 2 / 3).
__device__ void serial_alpha(const Params& prm, SerialSmem& S) {
  DevState* st = prm.st;
  const int tid = threadIdx.x;
  const int pk = ldcg(&st->pk);
  const int sq = pk * pk;
  if (tid < 4) S.flag[tid] = 0;
  for (int e = tid; e < 2 * sq; e += kThreads) {
    const int f = e < sq ? e : e - sq;
    const int a = f / pk, c = f - a * pk;
    const int off = (e < sq ? kSlotGram0 : kSlotGram1) + a * kMaxP + c;
    (e < sq ? S.m : S.g)[a * kLd + c] = sum_parts(prm, off);
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
    S.sc[tid] = mjj > 0.0 ? 1.0 / sqrt(mjj) : 0.0;
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
  // right-looking Cholesky, columns in agent order; a column whose pivot is
  // below rank_tol is skipped (agent dropped, Algorithm 3)
  const double neg_lim = -sqrt(prm.rank_tol);
  int m = 0;
  for (int j = 0; j < pk; ++j) {
    const double d = S.l[j * kLd + j];
    const bool zero_dir = S.m[j * kLd + j] == 0.0;
    int decision = 0;  // 0 keep, 1 drop, 2 not SPD, 3 NaN
    if (zero_dir) decision = 1;
    else if (!(d == d)) decision = 3;
    else if (d < neg_lim) decision = 2;
    else if (d < prm.rank_tol) decision = 1;
    if (decision >= 2) {
      if (tid == 0) set_error(st, decision == 2 ? ST_ERR_NOT_SPD : ST_ERR_NUMERICAL, 2);
      __syncthreads();
      return;
    }
    if (decision == 1) continue;
    const double ljj = sqrt(d);
    __syncthreads();
    if (tid == 0) { S.l[j * kLd + j] = ljj; S.keep[m] = j; }
    for (int i = j + 1 + tid; i < pk; i += kThreads) S.l[i * kLd + j] /= ljj;
    __syncthreads();
    const int nt = pk - j - 1;
    for (int e = tid; e < nt * nt; e += kThreads) {
      const int ii = j + 1 + e / nt, ll = j + 1 + e % nt;
      if (ll <= ii) S.l[ii * kLd + ll] -= S.l[ii * kLd + j] * S.l[ll * kLd + j];
    }
    ++m;
    __syncthreads();
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
  chol_solve_cols(S.m, S.l, m);
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
__device__ void serial_beta(const Params& prm, SerialSmem& S) {
  DevState* st = prm.st;
  const int tid = threadIdx.x;
  const int pk = ldcg(&st->pk);
  const int sq = pk * pk;
  if (tid < 4) S.flag[tid] = 0;
  for (int e = tid; e < sq + pk; e += kThreads) {
    if (e < sq) {
      const int a = e / pk, c = e - a * pk;
      S.g[a * kLd + c] = sum_parts(prm, kSlotGram0 + a * kMaxP + c);
    } else {
      S.s2[e - sq] = sum_parts(prm, kSlotVec + (e - sq));
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
  chol_solve_cols(S.m, S.l, pk);
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

__device__ void serial_bnorm(const Params& prm, SerialSmem& S) {
  DevState* st = prm.st;
  if (threadIdx.x == 0) {
    const double b2 = sum_parts(prm, kSlotScalar);
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
  for (int e = threadIdx.x; e < pk; e += kThreads) S.s2[e] = sum_parts(prm, kSlotVec + e);
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
    const double tr = sqrt(sum_parts(prm, kSlotScalar)) / ldcg(&st->bnorm);
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
    const int off = (e < sq ? kSlotGram0 : kSlotGram1) + a * kMaxP + c;
    (e < sq ? S.m : S.g)[a * kLd + c] = sum_parts(prm, off);
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

template <int P, bool VEC>
__global__ void __launch_bounds__(kThreads, 1) fp64_kernel(const __grid_constant__ Params prm) {
  extern __shared__ __align__(16) double smem[];
  __shared__ SyncShared ss;
  __shared__ int s_int[4];
  __shared__ int s_err;
  SerialSmem& S = *reinterpret_cast<SerialSmem*>(smem);
  DevState* st = prm.st;
  const int G = gridDim.x;
  const int cta = blockIdx.x;
  const int tid = threadIdx.x;
  const int64_t n = prm.n;
  const int64_t r0 = ((int64_t)cta * n) / G;
  const int64_t r1 = ((int64_t)(cta + 1) * n) / G;
  const int p = prm.p;
  double* mypart = prm.part + (size_t)cta * kPartStride;

#define CCG_SYNC_SERIAL(CALL)              \
  {                                        \
    const int f_ = grid_arrive(prm, &ss);  \
    if (f_ < 0) return;                    \
    if (f_ == 1) {                         \
      if (!cta_error(st, &s_err)) {        \
        CALL;                              \
      }                                    \
      grid_release(prm, &ss);              \
    }                                      \
    if (cta_error(st, &s_err)) return;     \
  }

  if (prm.mode == MODE_BARRIER_SELFTEST) {
    grid_barrier(prm, &ss, &s_err);
    return;
  }

  if (prm.mode == MODE_BLOCK_PRODUCT) {
    const int q = prm.q;
    apass<P, VEC>(prm, prm.V, q, 0, q, prm.Wout, q, false, r0, r1, smem);
    partial_grams(prm.V, prm.Wout, prm.U, prm.U ? prm.V : nullptr, nullptr, q, q, r0, r1,
                  mypart);
    CCG_SYNC_SERIAL(serial_block_product(prm, S));
    return;
  }

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
  CCG_SYNC_SERIAL(serial_bnorm(prm, S));

  if (tid == 0) s_int[0] = ldcg(&st->ctrl);
  __syncthreads();
  if (s_int[0] != CTRL_FINISH) {
    // R_0 = A X_0 - b 1^T ; D_0 = R_0
    apass<P, VEC>(prm, prm.X, p, 0, p, prm.R, p, true, r0, r1, smem);
    for (int64_t idx = r0 * p + tid; idx < r1 * p; idx += kThreads) prm.D0[idx] = ldcg(prm.R + idx);
    partial_grams(nullptr, nullptr, nullptr, nullptr, prm.R, p, p, r0, r1, mypart);
    CCG_SYNC_SERIAL(serial_norms(prm, S, false));
  }

  int cur = 0;
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

    if (ctrl == CTRL_CHECK) {
      // true residual of the best agent: W[:, 0] = A X e_jb - b
      const int jb = ldcg(&st->jbest);
      apass<1, VEC>(prm, prm.X, p, jb, 1, prm.W, p, true, r0, r1, smem);
      partial_sumsq(prm.W, p, r0, r1, mypart);
      CCG_SYNC_SERIAL(serial_check(prm));
      continue;
    }

    if (ctrl == CTRL_REPLACE) {
      apass<P, VEC>(prm, prm.X, p, 0, pk, prm.R, p, true, r0, r1, smem);
      for (int64_t idx = r0 * p + tid; idx < r1 * p; idx += kThreads) {
        const int c = (int)(idx % p);
        if (c < pk) D[idx] = ldcg(prm.R + idx);
      }
      partial_grams(nullptr, nullptr, nullptr, nullptr, prm.R, p, pk, r0, r1, mypart);
      CCG_SYNC_SERIAL(serial_norms(prm, S, true));
      continue;
    }

    // ---- one cCG iteration ----
    apass<P, VEC>(prm, D, p, 0, pk, prm.W, p, false, r0, r1, smem);
    partial_grams(D, prm.W, prm.R, D, nullptr, p, pk, r0, r1, mypart);
    CCG_SYNC_SERIAL(serial_alpha(prm, S));

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

    // X += D alpha^T ; R += W alpha^T
    {
      double* Ts = smem;
      for (int e = tid; e < pk * pk; e += kThreads) {
        const int b = e / pk, a = e - b * pk;
        Ts[b * kLd + a] = ldcg(&st->alphaT[b * kMaxP + a]);
      }
      __syncthreads();
      const int64_t cnt = (r1 - r0) * pk;
      for (int64_t idx = tid; idx < cnt; idx += kThreads) {
        const int64_t i = r0 + idx / pk;
        const int a = (int)(idx % pk);
        double dx = 0.0, dr = 0.0;
        for (int b = 0; b < pk; ++b) {
          const double t = Ts[b * kLd + a];
          dx = fma(ldcg(D + i * p + b), t, dx);
          dr = fma(ldcg(prm.W + i * p + b), t, dr);
        }
        prm.X[i * p + a] += dx;
        prm.R[i * p + a] += dr;
      }
      __syncthreads();
    }
    partial_grams(prm.R, prm.W, nullptr, nullptr, prm.R, p, pk, r0, r1, mypart);
    CCG_SYNC_SERIAL(serial_beta(prm, S));

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
      const int64_t cnt = (r1 - r0) * pk;
      for (int64_t idx = tid; idx < cnt; idx += kThreads) {
        const int64_t i = r0 + idx / pk;
        const int a = (int)(idx % pk);
        double acc = 0.0;
        for (int b = 0; b < pk; ++b) acc = fma(ldcg(D + i * p + b), Ts[b * kLd + a], acc);
        Dn[i * p + a] = ldcg(prm.R + i * p + a) + acc;
      }
      if (!grid_barrier(prm, &ss, &s_err)) return;
      cur ^= 1;
    }
  }
#undef CCG_SYNC_SERIAL
}

template <int P, bool VEC>
void* kernel_ptr() {
  return reinterpret_cast<void*>(&fp64_kernel<P, VEC>);
}

void* select_kernel(int P, bool vec) {
  switch (P) {
    case 1: return vec ? kernel_ptr<1, true>() : kernel_ptr<1, false>();
    case 2: return vec ? kernel_ptr<2, true>() : kernel_ptr<2, false>();
    case 4: return vec ? kernel_ptr<4, true>() : kernel_ptr<4, false>();
    case 8: return vec ? kernel_ptr<8, true>() : kernel_ptr<8, false>();
    case 16: return vec ? kernel_ptr<16, true>() : kernel_ptr<16, false>();
    case 32: return vec ? kernel_ptr<32, true>() : kernel_ptr<32, false>();
    default: return nullptr;
  }
}

template <int P>
constexpr size_t vs_bytes() {
  return 2 * sizeof(double) * (size_t)P * Tile<P>::VSTR;
}

}  // namespace

int p_bucket(int p) {
  int P = 1;
  while (P < p) P <<= 1;
  return P;
}

size_t fp64_smem_bytes(int P) {
  size_t vs = 0;
  switch (P) {
    case 1: vs = vs_bytes<1>(); break;
    case 2: vs = vs_bytes<2>(); break;
    case 4: vs = vs_bytes<4>(); break;
    case 8: vs = vs_bytes<8>(); break;
    case 16: vs = vs_bytes<16>(); break;
    default: vs = vs_bytes<32>(); break;
  }
  const size_t ser = sizeof(SerialSmem);
  size_t b = vs > ser ? vs : ser;
  if (b < vs_bytes<1>()) b = vs_bytes<1>();  // CHECK phase uses the P = 1 tile
  return (b + 15) & ~size_t(15);
}

int fp64_ctas_per_sm(int P, bool vec) {
  void* fn = select_kernel(P, vec);
  if (!fn) return 0;
  const size_t smem = fp64_smem_bytes(P);
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return 0;
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, kThreads, smem) != cudaSuccess) return 0;
  return nb;
}

cudaError_t launch_fp64(const Params& prm, int P, bool vec, int ctas, cudaStream_t stream) {
  void* fn = select_kernel(P, vec);
  if (!fn) return cudaErrorInvalidValue;
  const size_t smem = fp64_smem_bytes(P);
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  Params local = prm;
  void* args[] = {&local};
  return cudaLaunchCooperativeKernel(fn, dim3(ctas), dim3(kThreads), args, smem, stream);
}

}  // namespace ccg
