// ccg_capi_lowp.cu -- C ABI of the quantised matrices and of the tensor-core
// low-precision block product (include/ccg.h, "Mixed precision").  Argument
// checks, device buffers and launches only; the arithmetic is in ccg_lowp.cu.
#include <cuda_runtime.h>

#include <cstring>
#include <new>

#include "ccg.h"
#include "ccg_handle.h"
#include "ccg_lowp.h"

using namespace ccg_host;


namespace {

int lp_kind(int format) { return format == CCG_LOWP_BF16 ? ccg::lp::KIND_BF16 : ccg::lp::KIND_FP8; }

}  // namespace

extern "C" {

int ccg_lowp_create(ccg_handle* h, int format, int64_t n, const double* A, int64_t lda,
                    ccg_lowp_matrix** out) {
  if (!out) return CCG_ERR_INVALID;
  *out = nullptr;
  if (!h || !A || n < 1 || lda < n || (format != CCG_LOWP_BF16 && format != CCG_LOWP_FP8_E4M3) ||
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
  const size_t esz = (format == CCG_LOWP_BF16) ? 2 : 1;
  const size_t qbytes = (size_t)n * (size_t)m->ldq * esz;
  cudaError_t e = cudaMalloc(&m->q, qbytes);
  if (e == cudaSuccess && format == CCG_LOWP_FP8_E4M3)
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
