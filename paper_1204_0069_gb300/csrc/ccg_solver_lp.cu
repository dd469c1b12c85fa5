// ccg_solver_lp.cu -- instantiations of the persistent solver kernel whose
// A-pass runs on the tensor cores (BF16 or FP8 E4M3 A), used by the inner
// solves of the mixed-precision path.
#include <cuda_runtime.h>

#include "ccg_internal.h"
#include "ccg_solver.cuh"

namespace ccg {

void* select_kernel_lp(int P, int pol) {
  const bool fp8 = pol == POL_FP8;
  switch (P) {
    case 1: return fp8 ? kernel_ptr<1, true, POL_FP8>() : kernel_ptr<1, true, POL_BF16>();
    case 2: return fp8 ? kernel_ptr<2, true, POL_FP8>() : kernel_ptr<2, true, POL_BF16>();
    case 4: return fp8 ? kernel_ptr<4, true, POL_FP8>() : kernel_ptr<4, true, POL_BF16>();
    case 8: return fp8 ? kernel_ptr<8, true, POL_FP8>() : kernel_ptr<8, true, POL_BF16>();
    case 16: return fp8 ? kernel_ptr<16, true, POL_FP8>() : kernel_ptr<16, true, POL_BF16>();
    case 32: return fp8 ? kernel_ptr<32, true, POL_FP8>() : kernel_ptr<32, true, POL_BF16>();
    default: return nullptr;
  }
}

size_t solver_smem_bytes_lp(int P, int pol) {
  const bool fp8 = pol == POL_FP8;
  switch (P) {
    case 1: return fp8 ? solver_smem_bytes<1, POL_FP8>() : solver_smem_bytes<1, POL_BF16>();
    case 2: return fp8 ? solver_smem_bytes<2, POL_FP8>() : solver_smem_bytes<2, POL_BF16>();
    case 4: return fp8 ? solver_smem_bytes<4, POL_FP8>() : solver_smem_bytes<4, POL_BF16>();
    case 8: return fp8 ? solver_smem_bytes<8, POL_FP8>() : solver_smem_bytes<8, POL_BF16>();
    case 16: return fp8 ? solver_smem_bytes<16, POL_FP8>() : solver_smem_bytes<16, POL_BF16>();
    default: return fp8 ? solver_smem_bytes<32, POL_FP8>() : solver_smem_bytes<32, POL_BF16>();
  }
}

}  // namespace ccg
