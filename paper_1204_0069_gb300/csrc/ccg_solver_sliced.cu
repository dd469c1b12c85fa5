// ccg_solver_sliced.cu -- instantiations of the persistent solver kernel whose
// block product is the FP64 product formed exactly from FP8 slices on the
// tensor cores (policy POL_SLICED, at most 16 agents: the kSlices slices of
// every operand column share the MMA's N <= 256).
#include <cuda_runtime.h>

#include "ccg_internal.h"
#include "ccg_solver.cuh"

namespace ccg {

void* select_kernel_sliced(int P) {
  switch (P) {
    case 1: return kernel_ptr<1, true, POL_SLICED>();
    case 2: return kernel_ptr<2, true, POL_SLICED>();
    case 4: return kernel_ptr<4, true, POL_SLICED>();
    case 8: return kernel_ptr<8, true, POL_SLICED>();
    case 16: return kernel_ptr<16, true, POL_SLICED>();
    default: return nullptr;
  }
}

size_t solver_smem_bytes_sliced(int P) {
  switch (P) {
    case 1: return solver_smem_bytes<1, POL_SLICED>();
    case 2: return solver_smem_bytes<2, POL_SLICED>();
    case 4: return solver_smem_bytes<4, POL_SLICED>();
    case 8: return solver_smem_bytes<8, POL_SLICED>();
    default: return solver_smem_bytes<16, POL_SLICED>();
  }
}

}  // namespace ccg
