// ccg_capi.cu -- C ABI (include/ccg.h): argument checks, handle and workspace
// management, host/device buffer staging, and the cooperative launch of the
// persistent solver kernel.  No compute happens here: every arithmetic step
// of the solve runs in the persistent solver kernels of ccg_solver.cuh
// (instantiated in ccg_fp64.cu and its sibling files).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstddef>
#include <cstdint>
#include <cstring>
#include <new>

#include "ccg.h"
#include "ccg_handle.h"
#include "ccg_internal.h"
#include "ccg_lowp.h"

using ccg::DevState;
using ccg::Params;

namespace {

using namespace ccg_host;

int grid_size(const ccg_handle_s* h, int64_t n) {
  int64_t g = std::min<int64_t>(h->num_sms, (n + ccg::kWarps - 1) / ccg::kWarps);
  if (h->cfg.max_ctas > 0) g = std::min<int64_t>(g, h->cfg.max_ctas);
  return (int)std::max<int64_t>(1, g);
}

// Stream-ordered buffers of one sliced FP64 solve (freed after the launch is
// queued: the pool reuses them only after it completes).
void release_aligned_copy(ccg_handle_s* h) {
  if (h->aligned_copy) cudaFreeAsync(h->aligned_copy, h->stream);
  h->aligned_copy = nullptr;
}
void release_sliced(ccg_handle_s* h, ccg_lowp_matrix_s* m) {
  if (m) lowp_destroy_async(h, m);
  if (h->sliced_dq) cudaFreeAsync(h->sliced_dq, h->stream);
  if (h->sliced_part) cudaFreeAsync(h->sliced_part, h->stream);
  h->sliced_dq = nullptr;
  h->sliced_part = nullptr;
  release_aligned_copy(h);
}

void init_state(DevState* s, int p) {
  std::memset(s, 0, sizeof(DevState));
  s->pk = p;
  s->prev_pk = p;
  s->k_replaced = -1;
  for (int j = 0; j < ccg::kMaxP; ++j) s->agent[j] = j;
}

// Staged view of a caller buffer: device pointer to use and, for host
// buffers, where the device copy lives.
struct Buf {
  const void* user = nullptr;
  void* dev = nullptr;
  bool host = false;
  size_t bytes = 0;
};

// Policy and tensor-core kind of a quantised preconditioner matrix.
int pre_policy(int format) {
  return format == CCG_LOWP_FP8_E4M3 ? ccg::POL_FP8
         : format == CCG_LOWP_FP32   ? ccg::POL_TF32X3
                                     : ccg::POL_BF16;
}
int pre_kind(int format) {
  return format == CCG_LOWP_FP8_E4M3 ? ccg::lp::KIND_FP8
         : format == CCG_LOWP_FP32   ? ccg::lp::KIND_TF32X3
                                     : ccg::lp::KIND_BF16;
}

// One FP64 solve.  With `pre` (a quantised copy of A) the solve is the
// preconditioned form (CCG_MIXED_PRECOND): the persistent kernel yields
// whenever it needs Z = q(A_lp) R, the Chebyshev launch writes Z, and the
// solve resumes; its block products are formed from FP8 slices for p <= 16.
int solve_impl(ccg_handle_s* h, int64_t n, const double* A, int64_t lda, const double* b,
               const double* x0, const double* X0, int p, double tol, int maxit, double* x_out,
               double* X_out, ccg_result* res, const ccg_lowp_matrix_s* pre = nullptr) {
  if (res) {
    std::memset(res, 0, sizeof(*res));
    res->agent = -1;
  }
  auto fail = [&](int st) {
    if (res) res->status = st;
    return st;
  };
  if (!h || n < 1 || p < 1 || p > ccg::kMaxP || p > n || lda < n || !(tol > 0.0) ||
      (!pre && h->cfg.precision == CCG_FP64_SLICED && p > 16) ||
      (pre && (pre->n != n || pre->device != h->device)) ||
      !std::isfinite(tol) || maxit < 0 || !A || !b || !x_out)
    return fail(CCG_ERR_INVALID);
  DeviceGuard guard(h->device);

  const bool a_dev = is_device_ptr(A);
  const bool b_dev = is_device_ptr(b);
  const bool x0_dev = x0 ? is_device_ptr(x0) : true;
  const bool X0_dev = X0 ? is_device_ptr(X0) : true;
  const bool xo_dev = is_device_ptr(x_out);
  const bool Xo_dev = X_out ? is_device_ptr(X_out) : true;
  for (const void* ptr : {(const void*)A, (const void*)b, (const void*)x0, (const void*)X0,
                          (const void*)x_out, (const void*)X_out})
    if (ptr && !aligned(ptr, 8)) return fail(CCG_ERR_INVALID);

  const size_t np = (size_t)n * (size_t)p;
  // host A is staged with an even leading dimension (vectorised A stream)
  const int64_t lda_dev = a_dev ? lda : (n + (n & 1));
  const size_t a_bytes = a_dev ? 0 : (size_t)n * (size_t)lda_dev * sizeof(double);
  const size_t stage_need = Carve::need({a_bytes, b_dev ? 0 : n * sizeof(double),
                                         x0_dev ? 0 : n * sizeof(double),
                                         X0_dev ? 0 : np * sizeof(double),
                                         xo_dev ? 0 : n * sizeof(double),
                                         Xo_dev ? 0 : np * sizeof(double)});
  int rc = ensure(&h->stage, &h->stage_bytes, stage_need);
  if (rc != CCG_OK) return fail(rc);

  const int G = grid_size(h, n);
  // preconditioner buffers: Z and the Chebyshev scratch blocks, the operand
  // rows and partial tiles of the quantised product, the eigenvalue bound
  const int P0 = ccg::p_bucket(p);
  const int pre_NP = P0 <= 16 ? 16 : 32;
  const int pre_kd = pre ? pre_kind(pre->format) : 0;
  const size_t pre_esz = pre_kd == ccg::lp::KIND_BF16 ? 2 : pre_kd == ccg::lp::KIND_TF32X3 ? 4 : 1;
  const int pre_NB = pre_kd == ccg::lp::KIND_BF16 ? pre_NP : 2 * pre_NP;
  const int64_t ldk0 = ccg::lp::ld_elems(n);
  const int64_t T0 = (n + 127) / 128;
  const size_t ws_need =
      Carve::need({5 * np * sizeof(double), (size_t)G * ccg::kPartStride * sizeof(double),
                   sizeof(DevState), pre ? 4 * np * sizeof(double) : 0,
                   pre ? (size_t)pre_NB * ldk0 * pre_esz : 0,
                   pre ? (size_t)(G + T0) * 128 * pre_NP * sizeof(float) : 0,
                   pre ? sizeof(unsigned long long) : 0});
  rc = ensure(&h->ws, &h->ws_bytes, ws_need);
  if (rc != CCG_OK) return fail(rc);

  cudaStream_t s = h->stream;
  Carve sc(h->stage);
  const double* dA = A;
  const double* db = b;
  const double* dx0 = x0;
  const double* dX0 = X0;
  double* dxo = x_out;
  double* dXo = X_out;
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
  if (e == cudaSuccess && !X0_dev) {
    double* t = sc.take<double>(np);
    e = cudaMemcpyAsync(t, X0, np * sizeof(double), cudaMemcpyHostToDevice, s);
    dX0 = t;
  }
  if (!xo_dev) dxo = sc.take<double>(n);
  if (!Xo_dev) dXo = sc.take<double>(np);
  if (e != cudaSuccess) return fail(map_cuda(e));

  Carve wc(h->ws);
  Params prm{};
  prm.n = n;
  prm.lda = a_dev ? lda : lda_dev;
  prm.A = dA;
  prm.b = db;
  prm.x0 = X0 ? nullptr : dx0;
  prm.X0 = X0 ? dX0 : nullptr;
  prm.spread = h->cfg.x0_spread;
  prm.seed = h->cfg.seed;
  prm.X = wc.take<double>(np);
  prm.R = wc.take<double>(np);
  prm.D0 = wc.take<double>(np);
  prm.D1 = wc.take<double>(np);
  prm.W = wc.take<double>(np);
  prm.part = wc.take<double>((size_t)G * ccg::kPartStride);
  prm.st = wc.take<DevState>(1);
  prm.x_out = dxo;
  prm.X_out = dXo;
  prm.p = p;
  prm.maxit = maxit;
  prm.tol = tol;
  prm.rank_tol = h->cfg.rank_tol;
  prm.replacement = h->cfg.residual_replacement ? 1 : 0;
  prm.explicit_residual = h->cfg.explicit_residual ? 1 : 0;
  prm.mode = ccg::MODE_SOLVE;
  prm.timeout_ns = (long long)(h->cfg.barrier_timeout_ms * 1e6);
  prm.expected_ctas = (unsigned)G;

  const int P = ccg::p_bucket(p);
  bool vec = (prm.lda % 2 == 0) && aligned(dA, 16);
  const bool sliced = pre ? p <= 16 : h->cfg.precision == CCG_FP64_SLICED;
  const int pol = sliced ? ccg::POL_SLICED : ccg::POL_FP64;
  ccg_lowp_matrix_s* m = nullptr;
  if (sliced) {
    // FP64 cCG whose block products come from the FP8 slices of A on the
    // tensor cores; the kernel's true-residual pass streams the FP64 A with
    // 16-byte loads, so an unaligned A is copied with an even ld first
    if (!vec) {
      const int64_t ld2 = n + (n & 1);
      double* t = nullptr;
      e = cudaMallocAsync(reinterpret_cast<void**>(&t), (size_t)n * ld2 * sizeof(double), s);
      if (e == cudaSuccess)
        e = cudaMemcpy2DAsync(t, ld2 * sizeof(double), dA, prm.lda * sizeof(double),
                              n * sizeof(double), n, cudaMemcpyDeviceToDevice, s);
      if (e != cudaSuccess) {
        if (t) cudaFreeAsync(t, s);
        return fail(map_cuda(e));
      }
      h->aligned_copy = t;
      prm.A = t;
      prm.lda = ld2;
      vec = true;
    }
    const int rc2 = lowp_create_async(h, CCG_LOWP_FP64_SLICED, n, prm.A, prm.lda, &m);
    if (rc2 != CCG_OK) {
      release_aligned_copy(h);
      return fail(rc2);
    }
    const int NP = P;
    const int NB = (ccg::lp::kSlicesHost * NP + 15) / 16 * 16;
    const int64_t ldk = ccg::lp::ld_elems(n);
    const int64_t T = (n + 127) / 128;
    const size_t dq_bytes = (size_t)NB * ldk;
    const size_t part_bytes = (size_t)(G + T) * 128 * NP * sizeof(double);
    void* dq = nullptr;
    void* lpart = nullptr;
    e = cudaMallocAsync(&dq, dq_bytes, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(dq, 0, dq_bytes, s);
    if (e == cudaSuccess) e = cudaMallocAsync(&lpart, part_bytes, s);
    h->sliced_dq = dq;
    h->sliced_part = lpart;
    if (e != cudaSuccess) {
      release_sliced(h, m);
      return fail(map_cuda(e));
    }
    prm.lp_kelems = 128;
    prm.lp_kc = (int)((n + 127) / 128);
    prm.lp_tiles = T;
    prm.lp_units = (int64_t)ccg::lp::kSlicesHost * T * prm.lp_kc;
    prm.lp_row_scale = m->row_scale;
    prm.lp_dq = dq;
    prm.lp_ldk = ldk;
    prm.lp_part = reinterpret_cast<float*>(lpart);
    if (!ccg::lp::make_tensor_map(&prm.lp_tmA, m->q, ccg::lp::KIND_SLICED,
                                  ccg::lp::kSlicesHost * ccg::lp::slice_rows(n), n, m->ldq, 128) ||
        !ccg::lp::make_tensor_map(&prm.lp_tmB, dq, ccg::lp::KIND_SLICED, NB, n, ldk, NB)) {
      release_sliced(h, m);
      return fail(CCG_ERR_CUDA);
    }
  }
  if (ccg::fp64_ctas_per_sm(P, vec, pol) < 1) {
    release_sliced(h, m);
    return fail(CCG_ERR_CUDA);
  }

  // Chebyshev preconditioner launches on the quantised A (MODE_CHEB): same
  // grid, state and partial slots as the solve
  Params cp{};
  const int pre_pol = pre ? pre_policy(pre->format) : 0;
  if (pre) {
    cp = prm;
    cp.mode = ccg::MODE_CHEB;
    cp.V = prm.R;
    cp.Z = wc.take<double>(np);
    cp.cheb_d = wc.take<double>(np);
    cp.cheb_s = wc.take<double>(np);
    cp.cheb_w = wc.take<double>(np);
    void* pdq = wc.take<char>((size_t)pre_NB * ldk0 * pre_esz);
    float* ppart = wc.take<float>((size_t)(G + T0) * 128 * pre_NP);
    auto* bound = wc.take<unsigned long long>(1);
    cp.lp_kelems = (int)(128 / pre_esz);
    cp.lp_kc = (int)((n + cp.lp_kelems - 1) / cp.lp_kelems);
    cp.lp_tiles = T0;
    cp.lp_units = T0 * cp.lp_kc;
    cp.lp_row_scale = pre->row_scale;
    cp.lp_dq = pdq;
    cp.lp_ldk = ldk0;
    cp.lp_part = ppart;
    // measured best on the precision workload: 32 products for FP8, 48 for BF16
    cp.cheb_steps = h->cfg.cheb_degree > 0 ? h->cfg.cheb_degree
                    : pre->format == CCG_LOWP_BF16 ? 48
                                                   : 32;
    const double ratio = h->cfg.cheb_ratio > 0.0 ? h->cfg.cheb_ratio : 1e-4;
    prm.precond = 1;
    prm.Z = cp.Z;
    if (!ccg::lp::make_tensor_map(&cp.lp_tmA, pre->q, pre_kd, n, n, pre->ldq, 128) ||
        !ccg::lp::make_tensor_map(&cp.lp_tmB, pdq, pre_kd, pre_NB, n, ldk0, pre_NB) ||
        ccg::fp64_ctas_per_sm(P, true, pre_pol) < 1) {
      release_sliced(h, m);
      return fail(CCG_ERR_CUDA);
    }
    // operand rows beyond the active columns must read as zeros
    e = cudaMemsetAsync(pdq, 0, (size_t)pre_NB * ldk0 * pre_esz, s);
    if (e == cudaSuccess) e = ccg::lp::eig_bound(pre_kd, prm.A, prm.lda, n, bound, s);
    unsigned long long hb = 0;
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(&hb, bound, sizeof(hb), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
      release_sliced(h, m);
      return fail(map_cuda(e));
    }
    double hi;
    std::memcpy(&hi, &hb, sizeof(hi));
    if (!(hi > 0.0) || !std::isfinite(hi)) {
      release_sliced(h, m);
      return fail(CCG_ERR_NUMERICAL);
    }
    cp.cheb_hi = hi;
    cp.cheb_lo = ratio * hi;
  }

  init_state(h->h_state, p);
  int pc_apps = 0;
  e = cudaMemcpyAsync(prm.st, h->h_state, sizeof(DevState), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaEventRecord(h->ev0, s);
  if (e == cudaSuccess) e = ccg::launch_fp64(prm, P, vec, G, s, pol);
  if (pre) {
    // the solve yields for each preconditioner application: read the state's
    // leading words, run the Chebyshev launch, resume
    constexpr size_t kHeadBytes = offsetof(DevState, keep);
    Params rp = prm;
    rp.resume = 1;
    while (e == cudaSuccess) {
      e = cudaMemcpyAsync(h->h_state, prm.st, kHeadBytes, cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) break;
      const DevState& hs = *h->h_state;
      if (hs.error != 0 || hs.ctrl == ccg::CTRL_FINISH || hs.pc_stage == ccg::PC_NONE) break;
      e = ccg::launch_fp64(cp, P, true, G, s, pre_pol);
      if (e == cudaSuccess) e = ccg::launch_fp64(rp, P, vec, G, s, pol);
      ++pc_apps;
    }
  }
  if (e == cudaSuccess) e = cudaEventRecord(h->ev1, s);
  release_sliced(h, m);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h->h_state, prm.st, sizeof(DevState), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess && !xo_dev)
    e = cudaMemcpyAsync(x_out, dxo, n * sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess && X_out && !Xo_dev)
    e = cudaMemcpyAsync(X_out, dXo, np * sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return fail(map_cuda(e));

  const DevState& st = *h->h_state;
  int status = st.error != 0 ? st.error : st.result;
  if (res) {
    res->status = status;
    res->iterations = st.k;
    res->agent = (st.error == 0) ? st.agent[st.jbest] : -1;
    res->p_final = st.pk;
    res->replacements = st.replacements;
    res->drops = st.drops;
    res->relres_true = st.relres_true;
    res->relres_recur = st.relres_recur;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, h->ev0, h->ev1);
    res->device_ms = ms;
    res->ctas = G;
    res->outer_steps = pc_apps;
  }
  if (pre && status == CCG_OK && h->h_state->pc_stage != ccg::PC_NONE) status = CCG_ERR_CUDA;
  return status;
}

}  // namespace

// The preconditioned mixed-precision solve (CCG_MIXED_PRECOND) for
// ccg_solve_mixed: FP64 cCG on A with Chebyshev directions on lpA.
int ccg_solve_precond(ccg_handle* h, const ccg_lowp_matrix* m, int64_t n, const double* A,
                      int64_t lda, const double* b, const double* x0, int p, double tol,
                      int maxit, double* x_out, ccg_result* res) {
  if (!m || m->format == CCG_LOWP_FP64_SLICED) {
    if (res) {
      std::memset(res, 0, sizeof(*res));
      res->status = CCG_ERR_INVALID;
    }
    return CCG_ERR_INVALID;
  }
  return solve_impl(h, n, A, lda, b, x0, nullptr, p, tol, maxit, x_out, nullptr, res, m);
}

extern "C" {

void ccg_config_init(ccg_config* cfg) {
  if (!cfg) return;
  std::memset(cfg, 0, sizeof(*cfg));
  cfg->device = 0;
  cfg->stream = nullptr;
  cfg->precision = CCG_FP64;
  cfg->rank_tol = 1e-12;
  cfg->x0_spread = 1.0;
  cfg->seed = 0;
  cfg->residual_replacement = 1;
  cfg->barrier_timeout_ms = 10000.0;
  cfg->max_ctas = 0;
  cfg->inner_tol = 0.0;
  cfg->max_outer = 0;
  cfg->explicit_residual = 0;
  cfg->batch_autotune = 1;
  cfg->mixed_method = CCG_MIXED_AUTO;
  cfg->cheb_degree = 0;
  cfg->cheb_ratio = 0.0;
}

int ccg_create(ccg_handle** out, const ccg_config* cfg) {
  if (!out) return CCG_ERR_INVALID;
  *out = nullptr;
  ccg_config c;
  if (cfg) c = *cfg;
  else ccg_config_init(&c);
  if (!(c.rank_tol > 0.0) || !(c.barrier_timeout_ms > 0.0) ||
      (c.precision != CCG_FP64 && c.precision != CCG_FP32_IR && c.precision != CCG_BF16_IR &&
       c.precision != CCG_FP8_IR && c.precision != CCG_FP64_SLICED) ||
      c.max_ctas < 0 || c.inner_tol < 0.0 || c.max_outer < 0 ||
      (c.explicit_residual != 0 && c.explicit_residual != 1) ||
      (c.batch_autotune != 0 && c.batch_autotune != 1) ||
      (c.explicit_residual && c.precision != CCG_FP64) ||
      (c.mixed_method != CCG_MIXED_AUTO && c.mixed_method != CCG_MIXED_REFINE &&
       c.mixed_method != CCG_MIXED_PRECOND) ||
      c.cheb_degree < 0 || c.cheb_degree > 1024 || !(c.cheb_ratio >= 0.0 && c.cheb_ratio < 1.0))
    return CCG_ERR_INVALID;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess) {
    cudaGetLastError();
    return CCG_ERR_CUDA;
  }
  if (c.device < 0 || c.device >= ndev) return CCG_ERR_INVALID;
  ccg_handle_s* h = new (std::nothrow) ccg_handle_s();
  if (!h) return CCG_ERR_OOM;
  h->cfg = c;
  h->device = c.device;
  h->stream = static_cast<cudaStream_t>(c.stream);
  DeviceGuard guard(h->device);
  cudaError_t e = cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device);
  if (e == cudaSuccess) e = cudaMallocHost(reinterpret_cast<void**>(&h->h_state), sizeof(DevState));
  if (e == cudaSuccess) e = cudaEventCreate(&h->ev0);
  if (e == cudaSuccess) e = cudaEventCreate(&h->ev1);
  if (e != cudaSuccess) {
    ccg_destroy(h);
    return map_cuda(e);
  }
  *out = h;
  return CCG_OK;
}

int ccg_destroy(ccg_handle* h) {
  if (!h) return CCG_OK;
  {
    DeviceGuard guard(h->device);
    if (h->stream) cudaStreamSynchronize(h->stream);
    if (h->ws) cudaFree(h->ws);
    if (h->stage) cudaFree(h->stage);
    if (h->h_state) cudaFreeHost(h->h_state);
    if (h->ev0) cudaEventDestroy(h->ev0);
    if (h->ev1) cudaEventDestroy(h->ev1);
  }
  if (h->lp) ccg_lowp_destroy(h->lp);
  delete h;
  return CCG_OK;
}

int ccg_solve(ccg_handle* h, int64_t n, const double* A, int64_t lda, const double* b,
              const double* x0, int p, double tol, int maxit, double* x_out, ccg_result* res) {
  if (h && h->cfg.precision != CCG_FP64 && h->cfg.precision != CCG_FP64_SLICED) {
    // mixed precision: quantise A into a copy for this solve, refine in FP64
    const int fmt = h->cfg.precision == CCG_BF16_IR   ? CCG_LOWP_BF16
                    : h->cfg.precision == CCG_FP32_IR ? CCG_LOWP_FP32
                                                      : CCG_LOWP_FP8_E4M3;
    if (res) std::memset(res, 0, sizeof(*res));
    if (n < 1 || lda < n || !A || !aligned(A, 8)) {
      if (res) res->status = CCG_ERR_INVALID;
      return CCG_ERR_INVALID;
    }
    DeviceGuard guard(h->device);
    const double* dA = A;
    int64_t ldA = lda;
    if (!is_device_ptr(A)) {
      // host A: ccg_solve_mixed stages it; the quantiser needs a device copy too
      const int rc0 = ensure(&h->stage, &h->stage_bytes, (size_t)n * n * sizeof(double));
      if (rc0 != CCG_OK) return rc0;
      cudaError_t e = cudaMemcpy2DAsync(h->stage, n * sizeof(double), A, lda * sizeof(double),
                                        n * sizeof(double), n, cudaMemcpyHostToDevice, h->stream);
      if (e != cudaSuccess) return map_cuda(e);
      dA = reinterpret_cast<const double*>(h->stage);
      ldA = n;
    }
    ccg_lowp_matrix_s* m = nullptr;
    const int rc = lowp_create_async(h, fmt, n, dA, ldA, &m);
    if (rc != CCG_OK) {
      if (res) res->status = rc;
      return rc;
    }
    // (host A is staged again by the mixed-precision host loop; a device A is used in place)
    const int st = ccg_solve_mixed(h, m, n, A, lda, b, x0, p, tol, maxit, x_out, res);
    lowp_destroy_async(h, m);
    return st;
  }
  return solve_impl(h, n, A, lda, b, x0, nullptr, p, tol, maxit, x_out, nullptr, res);
}

int ccg_solve_block(ccg_handle* h, int64_t n, const double* A, int64_t lda, const double* b,
                    const double* X0, int p, double tol, int maxit, double* x_out,
                    double* X_out, ccg_result* res) {
  if (!X0) {
    if (res) {
      std::memset(res, 0, sizeof(*res));
      res->status = CCG_ERR_INVALID;
    }
    return CCG_ERR_INVALID;
  }
  return solve_impl(h, n, A, lda, b, nullptr, X0, p, tol, maxit, x_out, X_out, res);
}

int ccg_block_product(ccg_handle* h, int64_t n, const double* A, int64_t lda, const double* V,
                      const double* U, int q, double* W, double* M, double* G_out,
                      float* device_ms) {
  if (!h || n < 1 || q < 1 || q > ccg::kMaxP || lda < n || !A || !V || !W)
    return CCG_ERR_INVALID;
  for (const void* ptr : {(const void*)A, (const void*)V, (const void*)U, (const void*)W})
    if (ptr && !aligned(ptr, 8)) return CCG_ERR_INVALID;
  DeviceGuard guard(h->device);
  const bool a_dev = is_device_ptr(A), v_dev = is_device_ptr(V);
  const bool u_dev = U ? is_device_ptr(U) : true, w_dev = is_device_ptr(W);
  const size_t nq = (size_t)n * (size_t)q;
  const int64_t lda_dev = a_dev ? lda : (n + (n & 1));
  int rc = ensure(&h->stage, &h->stage_bytes,
                  Carve::need({a_dev ? 0 : (size_t)n * lda_dev * sizeof(double),
                               v_dev ? 0 : nq * sizeof(double), u_dev ? 0 : nq * sizeof(double),
                               w_dev ? 0 : nq * sizeof(double)}));
  if (rc != CCG_OK) return rc;
  const int G = grid_size(h, n);
  rc = ensure(&h->ws, &h->ws_bytes,
              Carve::need({(size_t)G * ccg::kPartStride * sizeof(double), sizeof(DevState)}));
  if (rc != CCG_OK) return rc;
  cudaStream_t s = h->stream;
  Carve sc(h->stage);
  const double* dA = A;
  const double* dV = V;
  const double* dU = U;
  double* dW = W;
  cudaError_t e = cudaSuccess;
  if (!a_dev) {
    double* t = sc.take<double>((size_t)n * lda_dev);
    e = cudaMemcpy2DAsync(t, lda_dev * sizeof(double), A, lda * sizeof(double),
                          n * sizeof(double), n, cudaMemcpyHostToDevice, s);
    dA = t;
  }
  if (e == cudaSuccess && !v_dev) {
    double* t = sc.take<double>(nq);
    e = cudaMemcpyAsync(t, V, nq * sizeof(double), cudaMemcpyHostToDevice, s);
    dV = t;
  }
  if (e == cudaSuccess && U && !u_dev) {
    double* t = sc.take<double>(nq);
    e = cudaMemcpyAsync(t, U, nq * sizeof(double), cudaMemcpyHostToDevice, s);
    dU = t;
  }
  if (!w_dev) dW = sc.take<double>(nq);
  if (e != cudaSuccess) return map_cuda(e);

  Carve wc(h->ws);
  Params prm{};
  prm.n = n;
  prm.lda = a_dev ? lda : lda_dev;
  prm.A = dA;
  prm.part = wc.take<double>((size_t)G * ccg::kPartStride);
  prm.st = wc.take<DevState>(1);
  prm.mode = ccg::MODE_BLOCK_PRODUCT;
  prm.timeout_ns = (long long)(h->cfg.barrier_timeout_ms * 1e6);
  prm.expected_ctas = (unsigned)G;
  prm.V = dV;
  prm.U = dU;
  prm.Wout = dW;
  prm.q = q;
  prm.p = q;
  const int P = ccg::p_bucket(q);
  const bool vec = (prm.lda % 2 == 0) && aligned(dA, 16);
  if (ccg::fp64_ctas_per_sm(P, vec) < 1) return CCG_ERR_CUDA;
  init_state(h->h_state, q);
  e = cudaMemcpyAsync(prm.st, h->h_state, sizeof(DevState), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaEventRecord(h->ev0, s);
  if (e == cudaSuccess) e = ccg::launch_fp64(prm, P, vec, G, s);
  if (e == cudaSuccess) e = cudaEventRecord(h->ev1, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h->h_state, prm.st, sizeof(DevState), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess && !w_dev)
    e = cudaMemcpyAsync(W, dW, nq * sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return map_cuda(e);
  const DevState& st = *h->h_state;
  if (st.error != 0) return st.error;
  for (int a = 0; a < q; ++a)
    for (int c = 0; c < q; ++c) {
      if (M) M[a * q + c] = st.gram_out[a * ccg::kMaxP + c];
      if (G_out && U) G_out[a * q + c] = st.gram_out[ccg::kSq + a * ccg::kMaxP + c];
    }
  if (device_ms) cudaEventElapsedTime(device_ms, h->ev0, h->ev1);
  return CCG_OK;
}

int ccg_selftest_barrier_timeout(ccg_handle* h, double timeout_ms) {
  if (!h || !(timeout_ms > 0.0) || timeout_ms > 60000.0) return CCG_ERR_INVALID;
  DeviceGuard guard(h->device);
  const int G = 2;
  int rc = ensure(&h->ws, &h->ws_bytes,
                  Carve::need({(size_t)G * ccg::kPartStride * sizeof(double), sizeof(DevState)}));
  if (rc != CCG_OK) return rc;
  Carve wc(h->ws);
  Params prm{};
  prm.n = 1;
  prm.lda = 1;
  prm.part = wc.take<double>((size_t)G * ccg::kPartStride);
  prm.st = wc.take<DevState>(1);
  prm.mode = ccg::MODE_BARRIER_SELFTEST;
  prm.timeout_ns = (long long)(timeout_ms * 1e6);
  prm.expected_ctas = (unsigned)G + 1u;  // one arrival more than the grid holds
  cudaStream_t s = h->stream;
  init_state(h->h_state, 1);
  cudaError_t e = cudaMemcpyAsync(prm.st, h->h_state, sizeof(DevState), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = ccg::launch_fp64(prm, 1, false, G, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h->h_state, prm.st, sizeof(DevState), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return map_cuda(e);
  return h->h_state->error;
}

const char* ccg_status_string(int status) {
  switch (status) {
    case CCG_OK: return "CCG_OK";
    case CCG_NOT_CONVERGED: return "CCG_NOT_CONVERGED";
    case CCG_ERR_INVALID: return "CCG_ERR_INVALID";
    case CCG_ERR_NOT_SPD: return "CCG_ERR_NOT_SPD";
    case CCG_ERR_NUMERICAL: return "CCG_ERR_NUMERICAL";
    case CCG_ERR_OOM: return "CCG_ERR_OOM";
    case CCG_ERR_TIMEOUT: return "CCG_ERR_TIMEOUT";
    case CCG_ERR_CUDA: return "CCG_ERR_CUDA";
    default: return "CCG_UNKNOWN_STATUS";
  }
}

const char* ccg_version(void) { return "ccg-gb300 0.1 (fp64 persistent)"; }

}  // extern "C"
