// ccg_solver_lp.cu -- instantiations of the persistent solver kernel whose
// A-pass runs on the tensor cores (BF16 or FP8 E4M3 A), used by the inner
// solves of the mixed-precision path.
#include <cuda_runtime.h>

#include "ccg_internal.h"
#include "ccg_solver.cuh"

namespace ccg {

// Sliced FP64 policy: ccg_solver_sliced.cu (compiled in parallel).
void* select_kernel_sliced(int P);
size_t solver_smem_bytes_sliced(int P);

namespace {

template <int POL>
void* select_pol(int P) {
  switch (P) {
    case 1: return kernel_ptr<1, true, POL>();
    case 2: return kernel_ptr<2, true, POL>();
    case 4: return kernel_ptr<4, true, POL>();
    case 8: return kernel_ptr<8, true, POL>();
    case 16: return kernel_ptr<16, true, POL>();
    case 32: return kernel_ptr<32, true, POL>();
    default: return nullptr;
  }
}

template <int POL>
size_t smem_pol(int P) {
  switch (P) {
    case 1: return solver_smem_bytes<1, POL>();
    case 2: return solver_smem_bytes<2, POL>();
    case 4: return solver_smem_bytes<4, POL>();
    case 8: return solver_smem_bytes<8, POL>();
    case 16: return solver_smem_bytes<16, POL>();
    default: return solver_smem_bytes<32, POL>();
  }
}

}  // namespace

void* select_kernel_lp(int P, int pol) {
  switch (pol) {
    case POL_BF16: return select_pol<POL_BF16>(P);
    case POL_FP8: return select_pol<POL_FP8>(P);
    case POL_TF32X3: return select_pol<POL_TF32X3>(P);
    case POL_SLICED: return select_kernel_sliced(P);
    default: return nullptr;
  }
}

size_t solver_smem_bytes_lp(int P, int pol) {
  switch (pol) {
    case POL_BF16: return smem_pol<POL_BF16>(P);
    case POL_FP8: return smem_pol<POL_FP8>(P);
    case POL_SLICED: return solver_smem_bytes_sliced(P);
    default: return smem_pol<POL_TF32X3>(P);
  }
}

}  // namespace ccg
