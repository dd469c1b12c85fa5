// ccg_batch_fp64_kernels.cu -- instantiations of the batched FP64 solver
// kernel (one CTA per system at a time), compiled apart from the other
// kernels so that the library builds in parallel.
#include <cuda_runtime.h>

#include "ccg_internal.h"
#include "ccg_solver.cuh"

namespace ccg {

void* select_batch_fp64(int P) {
  switch (P) {
    case 1: return reinterpret_cast<void*>(&batch_kernel<1>);
    case 2: return reinterpret_cast<void*>(&batch_kernel<2>);
    case 4: return reinterpret_cast<void*>(&batch_kernel<4>);
    case 8: return reinterpret_cast<void*>(&batch_kernel<8>);
    case 16: return reinterpret_cast<void*>(&batch_kernel<16>);
    case 32: return reinterpret_cast<void*>(&batch_kernel<32>);
    default: return nullptr;
  }
}

}  // namespace ccg
