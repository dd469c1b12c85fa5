// ccg_serve_kernels.cu -- instantiations and launch of the serving kernel
// (continuous batching over slots of CTAs, ccg_solver.cuh), compiled apart
// from the other kernels so that the library builds in parallel.  Two agent
// buckets: requests with p <= 8 run in the P = 8 kernel, the others in P = 32.
#include <cuda_runtime.h>

#include "ccg_internal.h"
#include "ccg_solver.cuh"

namespace ccg {

namespace {
void* select_serve(int P) {
  switch (P) {
    case 8: return reinterpret_cast<void*>(&serve_kernel<8>);
    case 32: return reinterpret_cast<void*>(&serve_kernel<32>);
    default: return nullptr;
  }
}
}  // namespace

int serve_ctas_per_sm(int P) {
  void* fn = select_serve(P);
  if (!fn) return 0;
  const size_t smem = fp64_smem_bytes(P, POL_FP64);
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return 0;
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, kThreads, smem) != cudaSuccess) return 0;
  return nb;
}

cudaError_t launch_serve(const Params& prm, int P, int ctas, cudaStream_t stream) {
  void* fn = select_serve(P);
  if (!fn) return cudaErrorInvalidValue;
  const size_t smem = fp64_smem_bytes(P, POL_FP64);
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  Params local = prm;
  void* args[] = {&local};
  // the slots' barriers need every CTA resident at once
  return cudaLaunchCooperativeKernel(fn, dim3(ctas), dim3(kThreads), args, smem, stream);
}

}  // namespace ccg
