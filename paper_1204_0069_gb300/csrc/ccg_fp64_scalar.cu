// ccg_fp64_scalar.cu -- instantiations of the persistent solver kernel with the
// FP64 A-pass for matrices whose rows do not allow 16-byte loads (odd leading
// dimension or an A pointer not 16-byte aligned).  Kept apart from
// ccg_fp64.cu so that the two compile in parallel.
#include <cuda_runtime.h>

#include "ccg_internal.h"
#include "ccg_solver.cuh"

namespace ccg {

void* select_kernel_fp64_scalar(int P) {
  switch (P) {
    case 1: return kernel_ptr<1, false, POL_FP64>();
    case 2: return kernel_ptr<2, false, POL_FP64>();
    case 4: return kernel_ptr<4, false, POL_FP64>();
    case 8: return kernel_ptr<8, false, POL_FP64>();
    case 16: return kernel_ptr<16, false, POL_FP64>();
    case 32: return kernel_ptr<32, false, POL_FP64>();
    default: return nullptr;
  }
}

}  // namespace ccg
