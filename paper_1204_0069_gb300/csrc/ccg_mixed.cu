// ccg_mixed.cu -- mixed-precision solve (include/ccg.h: ccg_solve_mixed).
//
// CCG_MIXED_PRECOND goes to the preconditioned FP64 solve (ccg_capi.cu);
// CCG_MIXED_REFINE is FP64 iterative refinement around inner cCG solves on a
// quantised A; CCG_MIXED_AUTO with BF16 / FP8 probes with refinement and
// hands over to the preconditioned solve when it contracts too slowly.
// Refinement:
//   x = x0;  r = b - A x (FP64, MODE_REFINE)
//   repeat:  solve A_lp d = r_s with p agents to a loose relative tolerance,
//            where r_s = r sqrt(n) / ||r|| (unit-RMS right-hand side, so the
//            agents' random starts have the scale of the solution);
//            x += d ||r|| / sqrt(n);  r = b - A x (FP64)
// The inner solves are the persistent solver kernel with its A-pass on the
// tensor cores (policy BF16 / FP8); their Grams, p x p solves and vectors stay
// in FP64.  The refinement step is the FP64 kernel in MODE_REFINE (update,
// residual with the FP64 A, norms, scaled right-hand side in one launch).
// Host code: argument checks, buffers, launches and the outer loop only.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>

#include "ccg.h"
#include "ccg_handle.h"
#include "ccg_internal.h"
#include "ccg_lowp.h"

using namespace ccg_host;
using ccg::DevState;
using ccg::Params;

namespace {

void init_state(DevState* s, int p) {
  std::memset(s, 0, sizeof(DevState));
  s->pk = p;
  s->prev_pk = p;
  s->k_replaced = -1;
  for (int j = 0; j < ccg::kMaxP; ++j) s->agent[j] = j;
}

int grid_size(const ccg_handle_s* h, int64_t n) {
  int64_t g = std::min<int64_t>(h->num_sms, (n + ccg::kWarps - 1) / ccg::kWarps);
  if (h->cfg.max_ctas > 0) g = std::min<int64_t>(g, h->cfg.max_ctas);
  return (int)std::max<int64_t>(1, g);
}

// Launch one persistent kernel with a fresh state and read the state back.
cudaError_t run(ccg_handle_s* h, const Params& prm, int P, bool vec, int G, int pol, int p) {
  init_state(h->h_state, p);
  cudaStream_t s = h->stream;
  cudaError_t e = cudaMemcpyAsync(prm.st, h->h_state, sizeof(DevState), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = ccg::launch_fp64(prm, P, vec, G, s, pol);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h->h_state, prm.st, sizeof(DevState), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return e;
}

}  // namespace

extern "C" int ccg_solve_mixed(ccg_handle* h, const ccg_lowp_matrix* m, int64_t n,
                               const double* A, int64_t lda, const double* b, const double* x0,
                               int p, double tol, int maxit, double* x_out, ccg_result* res) {
  if (res) {
    std::memset(res, 0, sizeof(*res));
    res->agent = -1;
  }
  auto fail = [&](int st) {
    if (res) res->status = st;
    return st;
  };
  // CCG_MIXED_AUTO with BF16 / FP8: refinement first, as a probe (short
  // inner solves, at least a tenfold gain per step); if it cannot contract
  // (the quantised A too coarse for the conditioning), the preconditioned
  // FP64 solve continues from its best x
  const bool probe = h && m && h->cfg.mixed_method == CCG_MIXED_AUTO &&
                     m->format != CCG_LOWP_FP32;
  if (h && m && h->cfg.mixed_method == CCG_MIXED_PRECOND)
    return ccg_solve_precond(h, m, n, A, lda, b, x0, p, tol, maxit, x_out, res);
  if (!h || !m || n < 1 || m->n != n || m->device != h->device || p < 1 || p > ccg::kMaxP ||
      p > n || lda < n || !(tol > 0.0) || !std::isfinite(tol) || maxit < 0 || !A || !b || !x_out)
    return fail(CCG_ERR_INVALID);
  for (const void* ptr : {(const void*)A, (const void*)b, (const void*)x0, (const void*)x_out})
    if (ptr && !aligned(ptr, 8)) return fail(CCG_ERR_INVALID);
  DeviceGuard guard(h->device);
  cudaStream_t s = h->stream;

  const bool fp8 = m->format == CCG_LOWP_FP8_E4M3;
  const bool f32 = m->format == CCG_LOWP_FP32;
  const int pol = fp8 ? ccg::POL_FP8 : f32 ? ccg::POL_TF32X3 : ccg::POL_BF16;
  const int kind = fp8 ? ccg::lp::KIND_FP8 : f32 ? ccg::lp::KIND_TF32X3 : ccg::lp::KIND_BF16;
  const int P = ccg::p_bucket(p);
  const int NP = P <= 16 ? 16 : 32;
  const int NB = (fp8 || f32) ? 2 * NP : NP;
  const int64_t ldk = ccg::lp::ld_elems(n);
  const size_t esz = fp8 ? 1 : f32 ? 4 : 2;
  const int G = grid_size(h, n);
  const int64_t T = (n + 127) / 128;
  const size_t np = (size_t)n * p;

  // host buffers are staged (A with an even leading dimension)
  const bool a_dev = is_device_ptr(A), b_dev = is_device_ptr(b);
  const bool x0_dev = x0 ? is_device_ptr(x0) : true, xo_dev = is_device_ptr(x_out);
  const int64_t lda_dev = a_dev ? lda : (n + (n & 1));
  int rc = ensure(&h->stage, &h->stage_bytes,
                  Carve::need({a_dev ? 0 : (size_t)n * lda_dev * sizeof(double),
                               b_dev ? 0 : n * sizeof(double), x0_dev ? 0 : n * sizeof(double),
                               xo_dev ? 0 : n * sizeof(double)}));
  if (rc != CCG_OK) return fail(rc);
  rc = ensure(&h->ws, &h->ws_bytes,
              Carve::need({5 * np * sizeof(double), (size_t)G * ccg::kPartStride * sizeof(double),
                           sizeof(DevState), (size_t)NB * ldk * esz,
                           (size_t)(G + T) * 128 * NP * sizeof(float), 5 * n * sizeof(double)}));
  if (rc != CCG_OK) return fail(rc);
  Carve sc(h->stage);
  const double* dA = A;
  const double* db = b;
  const double* dx0 = x0;
  double* dxo = x_out;
  cudaError_t e = cudaSuccess;
  if (!a_dev) {
    double* t = sc.take<double>((size_t)n * lda_dev);
    e = cudaMemcpy2DAsync(t, lda_dev * sizeof(double), A, lda * sizeof(double),
                          n * sizeof(double), n, cudaMemcpyHostToDevice, s);
    dA = t;
  }
  if (e == cudaSuccess && !b_dev) {
    double* t = sc.take<double>(n);
    e = cudaMemcpyAsync(t, b, n * sizeof(double), cudaMemcpyHostToDevice, s);
    db = t;
  }
  if (e == cudaSuccess && !x0_dev) {
    double* t = sc.take<double>(n);
    e = cudaMemcpyAsync(t, x0, n * sizeof(double), cudaMemcpyHostToDevice, s);
    dx0 = t;
  }
  if (!xo_dev) dxo = sc.take<double>(n);
  if (e != cudaSuccess) return fail(map_cuda(e));
  const int64_t ldA = a_dev ? lda : lda_dev;
  const bool vec = (ldA % 2 == 0) && aligned(dA, 16);

  Carve wc(h->ws);
  double* X = wc.take<double>(np);
  double* R = wc.take<double>(np);
  double* D0 = wc.take<double>(np);
  double* D1 = wc.take<double>(np);
  double* W = wc.take<double>(np);
  double* part = wc.take<double>((size_t)G * ccg::kPartStride);
  DevState* st = wc.take<DevState>(1);
  void* dq = wc.take<char>((size_t)NB * ldk * esz);
  float* lpart = wc.take<float>((size_t)(G + T) * 128 * NP);
  double* x = wc.take<double>(n);
  double* xbest = wc.take<double>(n);
  double* r = wc.take<double>(n);
  double* bin = wc.take<double>(n);
  double* d = wc.take<double>(n);

  // refinement launches: FP64 kernel, one column
  Params ref{};
  ref.n = n;
  ref.lda = ldA;
  ref.A = dA;
  ref.b = db;
  ref.part = part;
  ref.st = st;
  ref.p = 1;
  ref.mode = ccg::MODE_REFINE;
  ref.timeout_ns = (long long)(h->cfg.barrier_timeout_ms * 1e6);
  ref.expected_ctas = (unsigned)G;
  ref.ref_x = x;
  ref.ref_r = r;
  ref.ref_bin = bin;
  if (ccg::fp64_ctas_per_sm(1, vec) < 1 || ccg::fp64_ctas_per_sm(P, true, pol) < 1)
    return fail(CCG_ERR_CUDA);

  // inner solves: persistent kernel, tensor-core A-pass
  Params in{};
  in.n = n;
  in.lda = ldA;
  in.A = dA;
  in.b = bin;
  in.x0 = nullptr;
  in.spread = h->cfg.x0_spread;
  in.seed = h->cfg.seed;
  in.X = X;
  in.R = R;
  in.D0 = D0;
  in.D1 = D1;
  in.W = W;
  in.part = part;
  in.st = st;
  in.x_out = d;
  in.p = p;
  in.rank_tol = h->cfg.rank_tol;
  in.replacement = 0;
  in.mode = ccg::MODE_SOLVE;
  in.timeout_ns = ref.timeout_ns;
  in.expected_ctas = (unsigned)G;
  in.skip_true_check = 1;
  in.lp_kelems = (int)(128 / esz);
  in.lp_kc = (int)((n + in.lp_kelems - 1) / in.lp_kelems);
  in.lp_units = T * in.lp_kc;
  in.lp_row_scale = m->row_scale;
  in.lp_dq = dq;
  in.lp_ldk = ldk;
  in.lp_part = lpart;
  if (!ccg::lp::make_tensor_map(&in.lp_tmA, m->q, kind, n, n, m->ldq, 128) ||
      !ccg::lp::make_tensor_map(&in.lp_tmB, dq, kind, NB, n, ldk, NB))
    return fail(CCG_ERR_CUDA);

  const double tin_default = fp8 ? 1e-1 : f32 ? 1e-3 : 1e-2;
  const double tin = h->cfg.inner_tol > 0.0 ? h->cfg.inner_tol : tin_default;
  const int max_outer = h->cfg.max_outer > 0 ? h->cfg.max_outer : 60;

  e = cudaEventRecord(h->ev0, s);
  if (e == cudaSuccess) {
    if (dx0) e = cudaMemcpyAsync(x, dx0, n * sizeof(double), cudaMemcpyDeviceToDevice, s);
    else e = cudaMemsetAsync(x, 0, n * sizeof(double), s);
  }
  if (e == cudaSuccess) e = run(h, ref, 1, vec, G, ccg::POL_FP64, 1);
  if (e != cudaSuccess) return fail(map_cuda(e));
  if (h->h_state->error != 0) return fail(h->h_state->error);
  double bnorm = h->h_state->bnorm;
  double rnorm = h->h_state->rnorm;
  double relres = h->h_state->relres_true;
  double best = relres;
  e = cudaMemcpyAsync(xbest, x, n * sizeof(double), cudaMemcpyDeviceToDevice, s);
  if (e != cudaSuccess) return fail(map_cuda(e));

  int status = CCG_NOT_CONVERGED;
  int total = 0, outer = 0, stall = 0, drops = 0, last_agent = 0, last_pf = p;
  constexpr int kProbeInner = 200;  // inner iterations per probing step
  double last_recur = 0.0;
  if (bnorm == 0.0 || relres <= tol) status = CCG_OK;
  while (status != CCG_OK && outer < max_outer && total < maxit) {
    ++outer;
    // inner tolerance: loose, but not tighter than the outer target needs
    in.tol = std::max(tin, 0.5 * tol / relres);
    in.maxit = probe ? std::min(kProbeInner, maxit - total) : maxit - total;
    e = run(h, in, P, true, G, pol, p);
    if (e != cudaSuccess) return fail(map_cuda(e));
    const DevState& is = *h->h_state;
    if (is.error == CCG_ERR_NOT_SPD || is.error == CCG_ERR_NUMERICAL) {
      // the quantised system broke down (e.g. A_lp not positive definite):
      // refinement ends with the best x so far
      break;
    }
    if (is.error != 0) return fail(is.error);
    total += is.k;
    drops += is.drops;
    last_agent = is.agent[is.jbest];
    last_pf = is.pk;
    last_recur = is.relres_recur;
    // x += d ||r|| / sqrt(n) ; r = b - A x
    ref.ref_delta = d;
    ref.ref_coef = rnorm / std::sqrt((double)n);
    e = run(h, ref, 1, vec, G, ccg::POL_FP64, 1);
    if (e != cudaSuccess) return fail(map_cuda(e));
    if (h->h_state->error != 0) return fail(h->h_state->error);
    rnorm = h->h_state->rnorm;
    const double prev = relres;
    relres = h->h_state->relres_true;
    if (probe && !(relres <= 0.1 * prev)) {
      if (relres < best) {
        best = relres;
        e = cudaMemcpyAsync(xbest, x, n * sizeof(double), cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) return fail(map_cuda(e));
      }
      break;  // refinement contracts too slowly: hand over to the preconditioned solve
    }
    if (relres < best) {
      best = relres;
      stall = 0;
      e = cudaMemcpyAsync(xbest, x, n * sizeof(double), cudaMemcpyDeviceToDevice, s);
      if (e != cudaSuccess) return fail(map_cuda(e));
    } else if (++stall >= 2) {
      break;  // refinement no longer contracts
    }
    if (best <= tol) status = CCG_OK;
  }
  e = cudaMemcpyAsync(dxo, xbest, n * sizeof(double), cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess) e = cudaEventRecord(h->ev1, s);
  if (e == cudaSuccess && !xo_dev)
    e = cudaMemcpyAsync(x_out, dxo, n * sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return fail(map_cuda(e));
  if (res) {
    res->status = status;
    res->iterations = total;
    res->agent = last_agent;
    res->p_final = last_pf;
    res->replacements = 0;
    res->drops = drops;
    res->relres_true = best;
    res->relres_recur = last_recur;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, h->ev0, h->ev1);
    res->device_ms = ms;
    res->ctas = G;
    res->outer_steps = outer;
  }
  if (probe && status != CCG_OK && total < maxit) {
    // continue from the refinement's best x with the preconditioned solve;
    // the counts of both parts add up
    ccg_result r2;
    const int st2 = ccg_solve_precond(h, m, n, A, lda, b, x_out, p, tol, maxit - total, x_out,
                                      &r2);
    if (res) {
      const ccg_result r1 = *res;
      *res = r2;
      res->iterations += r1.iterations;
      res->outer_steps += r1.outer_steps;
      res->drops += r1.drops;
      res->device_ms += r1.device_ms;
    }
    return st2;
  }
  return status;
}
