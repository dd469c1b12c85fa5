// ccg_capi_lowp.cu -- C ABI of the quantised matrices and of the tensor-core
// low-precision block product (include/ccg.h, "Mixed precision").  Argument
// checks, device buffers and launches only; the arithmetic is in ccg_lowp.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <new>

#include "ccg.h"
#include "ccg_handle.h"
#include "ccg_internal.h"
#include "ccg_lowp.h"

using namespace ccg_host;


namespace {

int lp_kind(int format) {
  return format == CCG_LOWP_BF16          ? ccg::lp::KIND_BF16
         : format == CCG_LOWP_FP32        ? ccg::lp::KIND_TF32X3
         : format == CCG_LOWP_FP64_SLICED ? ccg::lp::KIND_SLICED
                                          : ccg::lp::KIND_FP8;
}

size_t lp_esize(int format) {
  return format == CCG_LOWP_BF16 ? 2 : format == CCG_LOWP_FP32 ? 4 : 1;
}

// Bytes of the entries of a quantised n x n matrix (sliced: all slices,
// each padded to whole 128-row tiles).
size_t lp_qbytes(int format, int64_t n, int64_t ldq) {
  if (format == CCG_LOWP_FP64_SLICED)
    return (size_t)ccg::lp::kSlicesHost * (size_t)ccg::lp::slice_rows(n) * (size_t)ldq;
  return (size_t)n * (size_t)ldq * lp_esize(format);
}

// W = A_lp V through the persistent solver kernel's tensor-core A-pass (the
// code path of the solves), used for the FP32 (TF32x3) and the sliced FP64
// formats.
int block_product_persistent(ccg_handle* h, const ccg_lowp_matrix_s* m, const double* dV, int q,
                             double* dW, float* device_ms) {
  const int64_t n = m->n;
  const int P = ccg::p_bucket(q);
  const bool sliced = m->format == CCG_LOWP_FP64_SLICED;
  const int NP = sliced ? P : P <= 16 ? 16 : 32;
  const int NB = sliced ? (ccg::lp::kSlicesHost * NP + 15) / 16 * 16 : 2 * NP;
  const int64_t ldk = ccg::lp::ld_elems(n);
  const int64_t T = (n + 127) / 128;
  const int pol = sliced ? ccg::POL_SLICED : ccg::POL_TF32X3;
  const int kind = sliced ? ccg::lp::KIND_SLICED : ccg::lp::KIND_TF32X3;
  const size_t esz = sliced ? 1 : sizeof(float);
  const int64_t tiles = sliced ? ccg::lp::kSlicesHost * T : T;
  const size_t pesz = sliced ? sizeof(double) : sizeof(float);
  int64_t g = std::min<int64_t>(h->num_sms, (n + ccg::kWarps - 1) / ccg::kWarps);
  if (h->cfg.max_ctas > 0) g = std::min<int64_t>(g, h->cfg.max_ctas);
  const int G = (int)std::max<int64_t>(1, g);
  if (ccg::fp64_ctas_per_sm(P, true, pol) < 1) return CCG_ERR_CUDA;
  int rc = ensure(&h->ws, &h->ws_bytes,
                  Carve::need({(size_t)G * ccg::kPartStride * sizeof(double),
                               sizeof(ccg::DevState), (size_t)NB * ldk * esz,
                               (size_t)(G + T) * 128 * NP * pesz}));
  if (rc != CCG_OK) return rc;
  Carve wc(h->ws);
  ccg::Params prm{};
  prm.n = n;
  prm.lda = n;
  prm.part = wc.take<double>((size_t)G * ccg::kPartStride);
  prm.st = wc.take<ccg::DevState>(1);
  prm.lp_dq = wc.take<char>((size_t)NB * ldk * esz);
  prm.lp_part = reinterpret_cast<float*>(wc.take<char>((size_t)(G + T) * 128 * NP * pesz));
  prm.mode = ccg::MODE_BLOCK_PRODUCT;
  prm.timeout_ns = (long long)(h->cfg.barrier_timeout_ms * 1e6);
  prm.expected_ctas = (unsigned)G;
  prm.V = dV;
  prm.Wout = dW;
  prm.q = q;
  prm.p = q;
  prm.lp_kelems = sliced ? 128 : 32;
  prm.lp_kc = (int)((n + prm.lp_kelems - 1) / prm.lp_kelems);
  prm.lp_tiles = T;
  prm.lp_units = tiles * prm.lp_kc;
  prm.lp_ldk = ldk;
  prm.lp_row_scale = m->row_scale;
  const int64_t arows = sliced ? ccg::lp::kSlicesHost * ccg::lp::slice_rows(n) : n;
  if (!ccg::lp::make_tensor_map(&prm.lp_tmA, m->q, kind, arows, n, m->ldq, 128) ||
      !ccg::lp::make_tensor_map(&prm.lp_tmB, prm.lp_dq, kind, NB, n, ldk, NB))
    return CCG_ERR_CUDA;
  std::memset(h->h_state, 0, sizeof(ccg::DevState));
  h->h_state->pk = q;
  cudaStream_t s = h->stream;
  cudaError_t e = cudaMemsetAsync(prm.lp_dq, 0, (size_t)NB * ldk * esz, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(prm.st, h->h_state, sizeof(ccg::DevState), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaEventRecord(h->ev0, s);
  if (e == cudaSuccess) e = ccg::launch_fp64(prm, P, true, G, s, pol);
  if (e == cudaSuccess) e = cudaEventRecord(h->ev1, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h->h_state, prm.st, sizeof(ccg::DevState), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return map_cuda(e);
  if (device_ms) cudaEventElapsedTime(device_ms, h->ev0, h->ev1);
  return h->h_state->error != 0 ? h->h_state->error : CCG_OK;
}

}  // namespace

namespace ccg_host {

// Quantised copy of A for one solve, in stream-ordered memory of the
// handle's stream (returned to the pool without a device-wide sync).
int lowp_create_async(ccg_handle* h, int format, int64_t n, const double* A, int64_t lda,
                      ccg_lowp_matrix_s** out) {
  *out = nullptr;
  cudaStream_t s = h->stream;
  ccg_lowp_matrix_s* m = new (std::nothrow) ccg_lowp_matrix_s();
  if (!m) return CCG_ERR_OOM;
  m->format = format;
  m->device = h->device;
  m->n = n;
  m->ldq = ccg::lp::ld_elems(n);
  const size_t qbytes = lp_qbytes(format, n, m->ldq);
  cudaError_t e = cudaMallocAsync(&m->q, qbytes, s);
  if (e == cudaSuccess && (format == CCG_LOWP_FP8_E4M3 || format == CCG_LOWP_FP64_SLICED))
    e = cudaMallocAsync(reinterpret_cast<void**>(&m->row_scale), (size_t)n * sizeof(float), s);
  if (e == cudaSuccess) e = ccg::lp::quantize(lp_kind(format), A, lda, n, m->q, m->ldq, m->row_scale, s);
  if (e != cudaSuccess) {
    lowp_destroy_async(h, m);
    return map_cuda(e);
  }
  m->bytes = (int64_t)qbytes;
  *out = m;
  return CCG_OK;
}

void lowp_destroy_async(ccg_handle* h, ccg_lowp_matrix_s* m) {
  if (!m) return;
  if (m->q) cudaFreeAsync(m->q, h->stream);
  if (m->row_scale) cudaFreeAsync(m->row_scale, h->stream);
  delete m;
}

}  // namespace ccg_host

extern "C" {

int ccg_lowp_create(ccg_handle* h, int format, int64_t n, const double* A, int64_t lda,
                    ccg_lowp_matrix** out) {
  if (!out) return CCG_ERR_INVALID;
  *out = nullptr;
  if (!h || !A || n < 1 || lda < n ||
      (format != CCG_LOWP_BF16 && format != CCG_LOWP_FP8_E4M3 && format != CCG_LOWP_FP32 &&
       format != CCG_LOWP_FP64_SLICED) ||
      !aligned(A, 8))
    return CCG_ERR_INVALID;
  DeviceGuard guard(h->device);
  cudaStream_t s = h->stream;
  const double* dA = A;
  int64_t ldA = lda;
  if (!is_device_ptr(A)) {
    int rc = ensure(&h->stage, &h->stage_bytes, (size_t)n * n * sizeof(double));
    if (rc != CCG_OK) return rc;
    cudaError_t e = cudaMemcpy2DAsync(h->stage, n * sizeof(double), A, lda * sizeof(double),
                                      n * sizeof(double), n, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return map_cuda(e);
    dA = reinterpret_cast<const double*>(h->stage);
    ldA = n;
  }
  ccg_lowp_matrix_s* m = new (std::nothrow) ccg_lowp_matrix_s();
  if (!m) return CCG_ERR_OOM;
  m->format = format;
  m->device = h->device;
  m->n = n;
  m->ldq = ccg::lp::ld_elems(n);
  const size_t qbytes = lp_qbytes(format, n, m->ldq);
  cudaError_t e = cudaMalloc(&m->q, qbytes);
  if (e == cudaSuccess && (format == CCG_LOWP_FP8_E4M3 || format == CCG_LOWP_FP64_SLICED))
    e = cudaMalloc(reinterpret_cast<void**>(&m->row_scale), (size_t)n * sizeof(float));
  if (e == cudaSuccess)
    e = ccg::lp::quantize(lp_kind(format), dA, ldA, n, m->q, m->ldq, m->row_scale, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    ccg_lowp_destroy(m);
    return map_cuda(e);
  }
  m->bytes = (int64_t)qbytes + (m->row_scale ? n * (int64_t)sizeof(float) : 0);
  *out = m;
  return CCG_OK;
}

int64_t ccg_lowp_bytes(const ccg_lowp_matrix* m) { return m ? m->bytes : 0; }

int ccg_lowp_destroy(ccg_lowp_matrix* m) {
  if (!m) return CCG_OK;
  {
    DeviceGuard guard(m->device);
    if (m->q) cudaFree(m->q);
    if (m->row_scale) cudaFree(m->row_scale);
  }
  delete m;
  return CCG_OK;
}

int ccg_lowp_block_product(ccg_handle* h, const ccg_lowp_matrix* m, const double* V, int q,
                           double* W, float* device_ms) {
  if (!h || !m || !V || !W || q < 1 || q > ccg::kMaxP || !aligned(V, 8) || !aligned(W, 8))
    return CCG_ERR_INVALID;
  if (m->device != h->device) return CCG_ERR_INVALID;
  DeviceGuard guard(h->device);
  cudaStream_t s = h->stream;
  const int64_t n = m->n;
  const int kind = lp_kind(m->format);
  const int NP = q <= 16 ? 16 : 32;
  const int NB = kind == ccg::lp::KIND_FP8 ? 2 * NP : NP;
  const int64_t ldk = ccg::lp::ld_elems(n);
  const size_t esz = kind == ccg::lp::KIND_BF16 ? 2 : 1;
  const int G = h->num_sms;
  const size_t nq = (size_t)n * q;
  const bool v_dev = is_device_ptr(V), w_dev = is_device_ptr(W);
  int rc = ensure(&h->stage, &h->stage_bytes,
                  Carve::need({v_dev ? 0 : nq * sizeof(double), w_dev ? 0 : nq * sizeof(double)}));
  if (rc != CCG_OK) return rc;
  rc = ensure(&h->ws, &h->ws_bytes,
              Carve::need({(size_t)NB * ldk * esz, 32 * sizeof(unsigned), 32 * sizeof(float),
                           ccg::lp::part_floats(n, G, NP) * sizeof(float), sizeof(int)}));
  if (rc != CCG_OK) return rc;
  Carve sc(h->stage);
  const double* dV = V;
  double* dW = W;
  cudaError_t e = cudaSuccess;
  if (!v_dev) {
    double* t = sc.take<double>(nq);
    e = cudaMemcpyAsync(t, V, nq * sizeof(double), cudaMemcpyHostToDevice, s);
    dV = t;
  }
  if (!w_dev) dW = sc.take<double>(nq);
  if (e != cudaSuccess) return map_cuda(e);
  if (m->format == CCG_LOWP_FP32 || m->format == CCG_LOWP_FP64_SLICED) {
    if (m->format == CCG_LOWP_FP64_SLICED && q > 16) return CCG_ERR_INVALID;
    int rc2 = block_product_persistent(h, m, dV, q, dW, device_ms);
    if (rc2 == CCG_OK && !w_dev) {
      e = cudaMemcpyAsync(W, dW, nq * sizeof(double), cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) return map_cuda(e);
    }
    return rc2;
  }
  Carve wc(h->ws);
  void* Vt = wc.take<char>((size_t)NB * ldk * esz);
  unsigned* cmax = wc.take<unsigned>(32);
  float* cscale = wc.take<float>(32);
  float* part = wc.take<float>(ccg::lp::part_floats(n, G, NP));
  int* err = wc.take<int>(1);
  e = cudaMemsetAsync(err, 0, sizeof(int), s);
  if (e == cudaSuccess)
    e = ccg::lp::convert_operand(kind, dV, n, q, NP, Vt, ldk, cmax, cscale, s);
  ccg::lp::LpRun run{};
  run.n = n;
  run.ctas = G;
  run.part = part;
  run.error = err;
  run.timeout_ns = (long long)(h->cfg.barrier_timeout_ms * 1e6);
  run.row_scale = m->row_scale;
  run.col_scale = kind == ccg::lp::KIND_FP8 ? cscale : nullptr;
  if (e == cudaSuccess)
    e = ccg::lp::block_product(kind, NP, m->q, m->ldq, Vt, ldk, run, q, dW, s, h->ev0, h->ev1);
  int herr = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h->h_state->error, err, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess && !w_dev)
    e = cudaMemcpyAsync(W, dW, nq * sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return map_cuda(e);
  herr = h->h_state->error;
  if (device_ms) cudaEventElapsedTime(device_ms, h->ev0, h->ev1);
  return herr != 0 ? herr : CCG_OK;
}

}  // extern "C"
