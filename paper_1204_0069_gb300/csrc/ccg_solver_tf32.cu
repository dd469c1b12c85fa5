// ccg_solver_tf32.cu -- instantiations of the persistent solver kernel whose A-pass
// runs on the tensor cores with A stored in FP32 (products of TF32 halves) (policy POL_TF32X3), used by the
// inner solves of the mixed-precision path.  One file per policy so that the
// library compiles in parallel.
#include <cuda_runtime.h>

#include "ccg_internal.h"
#include "ccg_solver.cuh"

namespace ccg {

void* select_kernel_tf32(int P) {
  switch (P) {
    case 1: return kernel_ptr<1, true, POL_TF32X3>();
    case 2: return kernel_ptr<2, true, POL_TF32X3>();
    case 4: return kernel_ptr<4, true, POL_TF32X3>();
    case 8: return kernel_ptr<8, true, POL_TF32X3>();
    case 16: return kernel_ptr<16, true, POL_TF32X3>();
    case 32: return kernel_ptr<32, true, POL_TF32X3>();
    default: return nullptr;
  }
}

size_t solver_smem_bytes_tf32(int P) {
  switch (P) {
    case 1: return solver_smem_bytes<1, POL_TF32X3>();
    case 2: return solver_smem_bytes<2, POL_TF32X3>();
    case 4: return solver_smem_bytes<4, POL_TF32X3>();
    case 8: return solver_smem_bytes<8, POL_TF32X3>();
    case 16: return solver_smem_bytes<16, POL_TF32X3>();
    default: return solver_smem_bytes<32, POL_TF32X3>();
  }
}

}  // namespace ccg
