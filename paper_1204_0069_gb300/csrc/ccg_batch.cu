// ccg_batch.cu -- C ABI of the batched solver (include/ccg.h:
// ccg_solve_batched): argument checks, the largest-first queue of system
// descriptors, workspace (plus the FP32 copies and refinement vectors of the
// mixed-precision variant), one launch, and the per-system results.
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
  int64_t nmax = 0;
  std::vector<int64_t> aoff(count), voff(count);
  int64_t ao = 0, vo = 0;
  for (int64_t i = 0; i < count; ++i) {
    if (n[i] < 1 || n[i] < p) return fail(CCG_ERR_INVALID);
    aoff[i] = ao;
    voff[i] = vo;
    ao += n[i] * (n[i] + (n[i] & 1));
    vo += n[i];
    nmax = std::max(nmax, n[i]);
  }
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

  const bool ir = h->cfg.precision == CCG_FP32_IR;
  if (!ir && h->cfg.precision != CCG_FP64) return fail(CCG_ERR_INVALID);
  const int P = ccg::p_bucket(p);
  const int per_sm = ccg::batch_ctas_per_sm(P, ir);
  if (per_sm < 1) return fail(CCG_ERR_CUDA);
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
                               sizeof(unsigned), (size_t)count * sizeof(int),
                               (size_t)count * sizeof(int), (size_t)count * sizeof(double),
                               (size_t)count * sizeof(int), (size_t)G * vslot * sizeof(double),
                               (size_t)G * fslot * sizeof(float)}));
  if (rc != CCG_OK) return fail(rc);
  Carve wc(h->ws);
  double* X = wc.take<double>((size_t)G * slot);
  double* part = wc.take<double>((size_t)G * ccg::kPartStride);
  ccg::DevState* st = wc.take<ccg::DevState>(G);
  int64_t* ddesc = wc.take<int64_t>(desc.size());
  unsigned* next = wc.take<unsigned>(1);
  int* dstatus = wc.take<int>(count);
  int* diters = wc.take<int>(count);
  double* drelres = wc.take<double>(count);
  int* douter = wc.take<int>(count);
  double* vbuf = wc.take<double>((size_t)G * vslot);
  float* fbuf = wc.take<float>((size_t)G * fslot);

  cudaStream_t s = h->stream;
  cudaError_t e = cudaMemcpyAsync(ddesc, desc.data(), desc.size() * sizeof(int64_t),
                                  cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(next, 0, sizeof(unsigned), s);
  if (e != cudaSuccess) return fail(map_cuda(e));

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
  prm.x_out = x_out;
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
  std::vector<int> hs(count), hi(count), ho(count, 0);
  std::vector<double> hr(count);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(hs.data(), dstatus, count * sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(hi.data(), diters, count * sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(hr.data(), drelres, count * sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess && ir)
    e = cudaMemcpyAsync(ho.data(), douter, count * sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return fail(map_cuda(e));
  int worst = CCG_OK;
  long long total = 0;
  int max_outer = 0;
  for (int64_t i = 0; i < count; ++i) {
    if (status) status[i] = hs[i];
    if (iterations) iterations[i] = hi[i];
    if (relres) relres[i] = hr[i];
    if (worst == CCG_OK && hs[i] != CCG_OK) worst = hs[i];
    total += hi[i];
    max_outer = std::max(max_outer, ho[i]);
  }
  if (summary) {
    summary->status = worst;
    summary->iterations = (int)std::min<long long>(total, 2147483647LL);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, h->ev0, h->ev1);
    summary->device_ms = ms;
    summary->ctas = G;
    summary->outer_steps = max_outer;
  }
  return worst;
}
