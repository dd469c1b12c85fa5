// ccg_solver_fp8.cu -- instantiations of the persistent solver kernel whose A-pass
// runs on the tensor cores with A stored in FP8 E4M3 with row scales (policy POL_FP8), used by the
// inner solves of the mixed-precision path.  One file per policy so that the
// library compiles in parallel.
#include <cuda_runtime.h>

#include "ccg_internal.h"
#include "ccg_solver.cuh"

namespace ccg {

void* select_kernel_fp8(int P) {
  switch (P) {
    case 1: return kernel_ptr<1, true, POL_FP8>();
    case 2: return kernel_ptr<2, true, POL_FP8>();
    case 4: return kernel_ptr<4, true, POL_FP8>();
    case 8: return kernel_ptr<8, true, POL_FP8>();
    case 16: return kernel_ptr<16, true, POL_FP8>();
    case 32: return kernel_ptr<32, true, POL_FP8>();
    default: return nullptr;
  }
}

size_t solver_smem_bytes_fp8(int P) {
  switch (P) {
    case 1: return solver_smem_bytes<1, POL_FP8>();
    case 2: return solver_smem_bytes<2, POL_FP8>();
    case 4: return solver_smem_bytes<4, POL_FP8>();
    case 8: return solver_smem_bytes<8, POL_FP8>();
    case 16: return solver_smem_bytes<16, POL_FP8>();
    default: return solver_smem_bytes<32, POL_FP8>();
  }
}

}  // namespace ccg
