// ccg_batch.cu -- C ABI of the batched solver (include/ccg.h:
// ccg_solve_batched, ccg_batch_tuning): argument checks, the largest-first
// queue of system descriptors, workspace (plus the FP32 copies and refinement
// vectors of the mixed-precision variant), the A-pass autotuner, one launch,
// and the per-system results.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <vector>

#include "ccg.h"
#include "ccg_handle.h"
#include "ccg_internal.h"

using namespace ccg_host;

namespace {

// Size bucket of a system (the kernel's rule): [2^(b+5), 2^(b+6)), b in 0..7.
int size_bucket(int64_t n) {
  int b = 0;
  while (b < 7 && n >= (int64_t(64) << b)) ++b;
  return b;
}

int p_index(int P) {
  int i = 0;
  while ((1 << i) < P) ++i;
  return i;  // 0..5 for P = 1..32
}

struct BatchOut {
  int* status = nullptr;      // host arrays of `count` entries (nullable)
  int* iterations = nullptr;
  double* relres = nullptr;
  int worst = CCG_OK;
  long long total_iters = 0;
  int max_outer = 0;
  float ms = 0.f;
  int ctas = 0;
};

// One launch of the batched kernel over the systems of `desc` (4 int64 per
// system: n, A offset, vector offset, result index).  Results land at the
// result indices (count_all entries on the host).
int run_batch(ccg_handle* h, const std::vector<int64_t>& desc, int64_t count_all, int p,
              double tol, int maxit, const double* A, const double* b, double* x, bool ir,
              const int* variant, BatchOut* out) {
  const int64_t count = (int64_t)desc.size() / 4;
  int64_t nmax = 0;
  for (int64_t k = 0; k < count; ++k) nmax = std::max(nmax, desc[4 * k]);
  const int P = ccg::p_bucket(p);
  const int per_sm = ccg::batch_ctas_per_sm(P, ir);
  if (per_sm < 1) return CCG_ERR_CUDA;
  int G = h->num_sms * per_sm;
  if (h->cfg.max_ctas > 0) G = std::min(G, h->cfg.max_ctas);
  G = (int)std::max<int64_t>(1, std::min<int64_t>(G, count));
  const int64_t slot = 5 * nmax * p;
  // refinement slots: r, b_in, delta, x_best; FP32 A copy and operand rows
  const int64_t ld32 = (nmax + 3) & ~int64_t(3);
  const int64_t vslot = ir ? 4 * nmax : 0;
  const int64_t fslot = ir ? (nmax + P) * ld32 : 0;
  int rc = ensure(&h->ws, &h->ws_bytes,
                  Carve::need({(size_t)G * slot * sizeof(double),
                               (size_t)G * ccg::kPartStride * sizeof(double),
                               (size_t)G * sizeof(ccg::DevState), desc.size() * sizeof(int64_t),
                               sizeof(unsigned), (size_t)count_all * sizeof(int),
                               (size_t)count_all * sizeof(int), (size_t)count_all * sizeof(double),
                               (size_t)count_all * sizeof(int), (size_t)G * vslot * sizeof(double),
                               (size_t)G * fslot * sizeof(float)}));
  if (rc != CCG_OK) return rc;
  Carve wc(h->ws);
  double* X = wc.take<double>((size_t)G * slot);
  double* part = wc.take<double>((size_t)G * ccg::kPartStride);
  ccg::DevState* st = wc.take<ccg::DevState>(G);
  int64_t* ddesc = wc.take<int64_t>(desc.size());
  unsigned* next = wc.take<unsigned>(1);
  int* dstatus = wc.take<int>(count_all);
  int* diters = wc.take<int>(count_all);
  double* drelres = wc.take<double>(count_all);
  int* douter = wc.take<int>(count_all);
  double* vbuf = wc.take<double>((size_t)G * vslot);
  float* fbuf = wc.take<float>((size_t)G * fslot);

  cudaStream_t s = h->stream;
  cudaError_t e = cudaMemcpyAsync(ddesc, desc.data(), desc.size() * sizeof(int64_t),
                                  cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(next, 0, sizeof(unsigned), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(douter, 0, (size_t)count_all * sizeof(int), s);
  if (e != cudaSuccess) return map_cuda(e);

  ccg::Params prm{};
  prm.A = A;
  prm.b = b;
  prm.x0 = nullptr;
  prm.X0 = nullptr;
  prm.spread = h->cfg.x0_spread;
  prm.seed = h->cfg.seed;
  prm.X = X;
  prm.part = part;
  prm.st = st;
  prm.x_out = x;
  prm.p = p;
  prm.maxit = maxit;
  prm.tol = tol;
  prm.rank_tol = h->cfg.rank_tol;
  prm.replacement = h->cfg.residual_replacement ? 1 : 0;
  prm.mode = ccg::MODE_SOLVE;
  prm.timeout_ns = (long long)(h->cfg.barrier_timeout_ms * 1e6);
  prm.expected_ctas = 1u;
  prm.group_ctas = 1;
  prm.batch_count = count;
  prm.batch_desc = ddesc;
  prm.batch_slot_stride = slot;
  prm.batch_next = next;
  prm.batch_status = dstatus;
  prm.batch_iters = diters;
  prm.batch_relres = drelres;
  for (int k = 0; k < 8; ++k) prm.batch_variant[k] = variant ? variant[k] : 0;
  if (ir) {
    prm.batch_vec = vbuf;
    prm.batch_vec_stride = vslot;
    prm.batch_f32 = fbuf;
    prm.batch_f32_stride = fslot;
    prm.batch_inner_tol = h->cfg.inner_tol > 0.0 ? h->cfg.inner_tol : 1e-5;
    prm.batch_max_outer = h->cfg.max_outer > 0 ? h->cfg.max_outer : 30;
    prm.batch_outer = douter;
  }

  e = cudaEventRecord(h->ev0, s);
  if (e == cudaSuccess) e = ccg::launch_batch(prm, P, G, s, ir);
  if (e == cudaSuccess) e = cudaEventRecord(h->ev1, s);
  std::vector<int> hs(count_all), hi(count_all), ho(count_all, 0);
  std::vector<double> hr(count_all);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(hs.data(), dstatus, count_all * sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(hi.data(), diters, count_all * sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(hr.data(), drelres, count_all * sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess && ir)
    e = cudaMemcpyAsync(ho.data(), douter, count_all * sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return map_cuda(e);
  out->worst = CCG_OK;
  out->total_iters = 0;
  out->max_outer = 0;
  for (int64_t k = 0; k < count; ++k) {
    const int64_t i = desc[4 * k + 3];
    if (out->status) out->status[i] = hs[i];
    if (out->iterations) out->iterations[i] = hi[i];
    if (out->relres) out->relres[i] = hr[i];
    if (out->worst == CCG_OK && hs[i] != CCG_OK) out->worst = hs[i];
    out->total_iters += hi[i];
    out->max_outer = std::max(out->max_outer, ho[i]);
  }
  cudaEventElapsedTime(&out->ms, h->ev0, h->ev1);
  out->ctas = G;
  return CCG_OK;
}

// A-pass variants worth trying for bucket P (apass in ccg_solver.cuh).
std::vector<int> candidates(int P) {
  if (P <= 2) return {0, 2};
  if (P <= 8) return {0, 1, 2};
  return {0};
}

// Per size bucket present in the batch: time each A-pass variant on up to two
// systems per CTA of that bucket, a fixed number of iterations each (x goes
// to a scratch buffer), and keep the fastest.  Buckets absent from the batch
// keep variant 0 and are tuned when a later batch brings them.
int autotune(ccg_handle* h, const std::vector<int64_t>& desc, int64_t count_all, int p,
             const double* A, const double* b, int64_t vtotal, bool ir) {
  const int P = ccg::p_bucket(p);
  const int pi = p_index(P);
  const std::vector<int> cand = candidates(P);
  int* table = h->batch_variant[ir ? 1 : 0][pi];
  bool* known = h->batch_known[ir ? 1 : 0][pi];
  std::vector<std::vector<int64_t>> by(8);
  for (size_t k = 0; k + 3 < desc.size(); k += 4) {
    const int bk = size_bucket(desc[k]);
    if (known[bk]) continue;
    if ((int64_t)by[bk].size() < 4 * 2 * h->num_sms)
      by[bk].insert(by[bk].end(), desc.begin() + k, desc.begin() + k + 4);
  }
  double* xs = nullptr;
  bool any = false;
  for (int bk = 0; bk < 8; ++bk) any = any || !by[bk].empty();
  if (!any) return CCG_OK;
  if (cand.size() == 1) {
    for (int bk = 0; bk < 8; ++bk)
      if (!by[bk].empty()) known[bk] = true;
    return CCG_OK;
  }
  cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&xs), (size_t)vtotal * sizeof(double),
                                  h->stream);
  if (e != cudaSuccess) return map_cuda(e);
  int rc = CCG_OK;
  for (int bk = 0; bk < 8 && rc == CCG_OK; ++bk) {
    if (by[bk].empty()) continue;
    float best_ms = 0.f;
    int best = 0;
    for (int v : cand) {
      int trial[8];
      std::memcpy(trial, table, sizeof(trial));
      trial[bk] = v;
      BatchOut o;
      float ms = 0.f;
      for (int rep = 0; rep < 2 && rc == CCG_OK; ++rep) {  // second run: warm caches
        rc = run_batch(h, by[bk], count_all, p, 1e-300, 6, A, b, xs, ir, trial, &o);
        ms = o.ms;
      }
      if (rc != CCG_OK) break;
      if (v == cand.front() || ms < best_ms) {
        best_ms = ms;
        best = v;
      }
    }
    if (rc == CCG_OK) {
      table[bk] = best;
      known[bk] = true;
    }
  }
  cudaFreeAsync(xs, h->stream);
  return rc;
}

}  // namespace

extern "C" int ccg_solve_batched(ccg_handle* h, int64_t count, const int64_t* n,
                                 const double* A, const double* b, int p, double tol, int maxit,
                                 double* x_out, int* status, int* iterations, double* relres,
                                 ccg_result* summary) {
  if (summary) {
    std::memset(summary, 0, sizeof(*summary));
    summary->agent = -1;
  }
  auto fail = [&](int st) {
    if (summary) summary->status = st;
    return st;
  };
  if (!h || count < 0 || p < 1 || p > ccg::kMaxP || !(tol > 0.0) || !std::isfinite(tol) ||
      maxit < 0)
    return fail(CCG_ERR_INVALID);
  if (count == 0) return fail(CCG_OK);
  if (!n || !A || !b || !x_out) return fail(CCG_ERR_INVALID);
  DeviceGuard guard(h->device);
  if (!is_device_ptr(A) || !is_device_ptr(b) || !is_device_ptr(x_out) || !aligned(A, 16) ||
      !aligned(b, 8) || !aligned(x_out, 8))
    return fail(CCG_ERR_INVALID);
  std::vector<int64_t> aoff(count), voff(count);
  int64_t ao = 0, vo = 0;
  for (int64_t i = 0; i < count; ++i) {
    if (n[i] < 1 || n[i] < p) return fail(CCG_ERR_INVALID);
    aoff[i] = ao;
    voff[i] = vo;
    ao += n[i] * (n[i] + (n[i] & 1));
    vo += n[i];
  }
  const bool ir = h->cfg.precision == CCG_FP32_IR;
  if (!ir && h->cfg.precision != CCG_FP64) return fail(CCG_ERR_INVALID);
  // queue: largest systems first (longest-processing-time order)
  std::vector<int64_t> order(count);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int64_t a, int64_t c) { return n[a] > n[c]; });
  std::vector<int64_t> desc(4 * count);
  for (int64_t k = 0; k < count; ++k) {
    const int64_t i = order[k];
    desc[4 * k + 0] = n[i];
    desc[4 * k + 1] = aoff[i];
    desc[4 * k + 2] = voff[i];
    desc[4 * k + 3] = i;
  }
  if (h->cfg.batch_autotune) {
    const int rc = autotune(h, desc, count, p, A, b, vo, ir);
    if (rc != CCG_OK) return fail(rc);
  }
  BatchOut o;
  o.status = status;
  o.iterations = iterations;
  o.relres = relres;
  const int P = ccg::p_bucket(p);
  const int rc = run_batch(h, desc, count, p, tol, maxit, A, b, x_out, ir,
                           h->batch_variant[ir ? 1 : 0][p_index(P)], &o);
  if (rc != CCG_OK) return fail(rc);
  if (summary) {
    summary->status = o.worst;
    summary->iterations = (int)std::min<long long>(o.total_iters, 2147483647LL);
    summary->device_ms = o.ms;
    summary->ctas = o.ctas;
    summary->outer_steps = o.max_outer;
  }
  return o.worst;
}

extern "C" int ccg_batch_tuning(ccg_handle* h, int p, int precision, int* variant, int set) {
  if (!h || !variant || p < 1 || p > ccg::kMaxP ||
      (precision != CCG_FP64 && precision != CCG_FP32_IR))
    return CCG_ERR_INVALID;
  const int P = ccg::p_bucket(p);
  const int ir = precision == CCG_FP32_IR ? 1 : 0;
  int* table = h->batch_variant[ir][p_index(P)];
  bool* known = h->batch_known[ir][p_index(P)];
  if (set) {
    const std::vector<int> cand = candidates(P);
    for (int k = 0; k < 8; ++k)
      if (std::find(cand.begin(), cand.end(), variant[k]) == cand.end()) return CCG_ERR_INVALID;
    for (int k = 0; k < 8; ++k) {
      table[k] = variant[k];
      known[k] = true;
    }
  } else {
    for (int k = 0; k < 8; ++k) variant[k] = known[k] ? table[k] : -1;
  }
  return CCG_OK;
}
