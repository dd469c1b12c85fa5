// ccg_handle.h -- the solver handle and host-side helpers shared by the C-ABI
// translation units.  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <initializer_list>

#include "ccg.h"
#include "ccg_internal.h"

struct ccg_lowp_matrix_s {
  int format = 0;
  int device = 0;
  int64_t n = 0;
  int64_t ldq = 0;
  void* q = nullptr;          // n x ldq entries
  float* row_scale = nullptr; // FP8: n scales
  int64_t bytes = 0;
};

struct ccg_handle_s {
  ccg_config cfg;
  cudaStream_t stream = nullptr;
  int device = 0;
  int num_sms = 0;
  char* ws = nullptr;         // solver workspace
  size_t ws_bytes = 0;
  char* stage = nullptr;      // device copies of host inputs / outputs
  size_t stage_bytes = 0;
  ccg::DevState* h_state = nullptr;  // pinned host mirror of the device state
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  ccg_lowp_matrix_s* lp = nullptr;  // quantised copy made by ccg_solve (mixed precision)
  // batched solves: A-pass variant per (FP64 / FP32-IR, agent bucket, size
  // bucket), and whether the autotuner has settled it
  int batch_variant[2][6][8] = {};
  bool batch_known[2][6][8] = {};
  // stream-ordered buffers of a sliced FP64 solve (live during one call)
  void* sliced_dq = nullptr;
  void* sliced_part = nullptr;
  double* aligned_copy = nullptr;
};

namespace ccg_host {

// Restores the caller's current device on scope exit.
struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

inline int map_cuda(cudaError_t e) {
  if (e == cudaSuccess) return CCG_OK;
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    return CCG_ERR_OOM;
  }
  return CCG_ERR_CUDA;
}

inline bool is_device_ptr(const void* p) {
  if (p == nullptr) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

inline bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

inline size_t round_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

inline int ensure(char** buf, size_t* have, size_t need) {
  if (*have >= need) return CCG_OK;
  if (*buf) {
    cudaFree(*buf);
    *buf = nullptr;
    *have = 0;
  }
  const size_t sz = round_up(std::max<size_t>(need, 1), size_t(1) << 20);
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(buf), sz);
  if (e != cudaSuccess) {
    *buf = nullptr;
    return map_cuda(e);
  }
  *have = sz;
  return CCG_OK;
}

// Bump allocator over a contiguous region (256-byte aligned pieces).
struct Carve {
  char* base;
  size_t off = 0;
  explicit Carve(char* b) : base(b) {}
  template <class T>
  T* take(size_t count) {
    off = round_up(off, 256);
    T* p = reinterpret_cast<T*>(base + off);
    off += count * sizeof(T);
    return p;
  }
  static size_t need(std::initializer_list<size_t> bytes) {
    size_t o = 0;
    for (size_t b : bytes) o = round_up(o, 256) + b;
    return round_up(o, 256);
  }
};

// Stream-ordered quantised copy for one solve (ccg_capi_lowp.cu).
int lowp_create_async(ccg_handle* h, int format, int64_t n, const double* A, int64_t lda,
                      ccg_lowp_matrix_s** out);
void lowp_destroy_async(ccg_handle* h, ccg_lowp_matrix_s* m);

}  // namespace ccg_host

// Preconditioned mixed-precision solve (ccg_capi.cu), the CCG_MIXED_PRECOND
// method of ccg_solve_mixed.
int ccg_solve_precond(ccg_handle* h, const ccg_lowp_matrix* m, int64_t n, const double* A,
                      int64_t lda, const double* b, const double* x0, int p, double tol,
                      int maxit, double* x_out, ccg_result* res);
