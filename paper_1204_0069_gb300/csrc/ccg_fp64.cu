// ccg_fp64.cu -- instantiations of the persistent solver kernel with the FP64
// A-pass and 16-byte loads of A (ccg_solver.cuh), and the host-side launch
// helpers for every policy.  The other instantiations sit in files of their
// own so that the library compiles in parallel: ccg_fp64_scalar.cu (FP64
// A-pass with 8-byte loads), ccg_solver_lp.cu (tensor-core policies),
// ccg_batch_fp64_kernels.cu and ccg_batch_ir_kernels.cu (batched solver).
#include <cuda_runtime.h>

#include "ccg_internal.h"
#include "ccg_solver.cuh"

namespace ccg {

void* select_kernel_lp(int P, int pol);
size_t solver_smem_bytes_lp(int P, int pol);
void* select_kernel_fp64_scalar(int P);
void* select_batch_fp64(int P);
void* select_batch_ir(int P);

namespace {

void* select_kernel(int P, bool vec) {
  if (!vec) return select_kernel_fp64_scalar(P);
  switch (P) {
    case 1: return kernel_ptr<1, true, POL_FP64>();
    case 2: return kernel_ptr<2, true, POL_FP64>();
    case 4: return kernel_ptr<4, true, POL_FP64>();
    case 8: return kernel_ptr<8, true, POL_FP64>();
    case 16: return kernel_ptr<16, true, POL_FP64>();
    case 32: return kernel_ptr<32, true, POL_FP64>();
    default: return nullptr;
  }
}

void* select_any(int P, bool vec, int pol) {
  return pol == POL_FP64 ? select_kernel(P, vec) : select_kernel_lp(P, pol);
}

void* select_batch(int P, bool ir) { return ir ? select_batch_ir(P) : select_batch_fp64(P); }

}  // namespace

int batch_ctas_per_sm(int P, bool ir) {
  void* fn = select_batch(P, ir);
  if (!fn) return 0;
  const size_t smem = fp64_smem_bytes(P, POL_FP64);
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return 0;
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, kThreads, smem) != cudaSuccess) return 0;
  return nb;
}

cudaError_t launch_batch(const Params& prm, int P, int ctas, cudaStream_t stream, bool ir) {
  void* fn = select_batch(P, ir);
  if (!fn) return cudaErrorInvalidValue;
  const size_t smem = fp64_smem_bytes(P, POL_FP64);
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  Params local = prm;
  void* args[] = {&local};
  return cudaLaunchKernel(fn, dim3(ctas), dim3(kThreads), args, smem, stream);
}

int p_bucket(int p) {
  int P = 1;
  while (P < p) P <<= 1;
  return P;
}

size_t fp64_smem_bytes(int P, int pol) {
  if (pol != POL_FP64) return solver_smem_bytes_lp(P, pol);
  switch (P) {
    case 1: return solver_smem_bytes<1, POL_FP64>();
    case 2: return solver_smem_bytes<2, POL_FP64>();
    case 4: return solver_smem_bytes<4, POL_FP64>();
    case 8: return solver_smem_bytes<8, POL_FP64>();
    case 16: return solver_smem_bytes<16, POL_FP64>();
    default: return solver_smem_bytes<32, POL_FP64>();
  }
}

int fp64_ctas_per_sm(int P, bool vec, int pol) {
  void* fn = select_any(P, vec, pol);
  if (!fn) return 0;
  const size_t smem = fp64_smem_bytes(P, pol);
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return 0;
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, kThreads, smem) != cudaSuccess) return 0;
  return nb;
}

cudaError_t launch_fp64(const Params& prm, int P, bool vec, int ctas, cudaStream_t stream, int pol) {
  void* fn = select_any(P, vec, pol);
  if (!fn) return cudaErrorInvalidValue;
  const size_t smem = fp64_smem_bytes(P, pol);
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  Params local = prm;
  void* args[] = {&local};
  return cudaLaunchCooperativeKernel(fn, dim3(ctas), dim3(kThreads), args, smem, stream);
}

}  // namespace ccg
