// ccg_solver_lp.cu -- instantiations of the persistent solver kernel whose
// A-pass runs on the tensor cores with A stored in BF16 (policy POL_BF16),
// and the dispatch over all tensor-core policies.  The other policies sit in
// files of their own so that the library compiles in parallel:
// ccg_solver_fp8.cu (FP8 E4M3 with row scales), ccg_solver_tf32.cu (FP32 as
// TF32 halves), ccg_solver_sliced.cu (FP64 as exact FP8 slices).
#include <cuda_runtime.h>

#include "ccg_internal.h"
#include "ccg_solver.cuh"

namespace ccg {

void* select_kernel_fp8(int P);
size_t solver_smem_bytes_fp8(int P);
void* select_kernel_tf32(int P);
size_t solver_smem_bytes_tf32(int P);
void* select_kernel_sliced(int P);
size_t solver_smem_bytes_sliced(int P);

namespace {

void* select_bf16(int P) {
  switch (P) {
    case 1: return kernel_ptr<1, true, POL_BF16>();
    case 2: return kernel_ptr<2, true, POL_BF16>();
    case 4: return kernel_ptr<4, true, POL_BF16>();
    case 8: return kernel_ptr<8, true, POL_BF16>();
    case 16: return kernel_ptr<16, true, POL_BF16>();
    case 32: return kernel_ptr<32, true, POL_BF16>();
    default: return nullptr;
  }
}

size_t smem_bf16(int P) {
  switch (P) {
    case 1: return solver_smem_bytes<1, POL_BF16>();
    case 2: return solver_smem_bytes<2, POL_BF16>();
    case 4: return solver_smem_bytes<4, POL_BF16>();
    case 8: return solver_smem_bytes<8, POL_BF16>();
    case 16: return solver_smem_bytes<16, POL_BF16>();
    default: return solver_smem_bytes<32, POL_BF16>();
  }
}

}  // namespace

void* select_kernel_lp(int P, int pol) {
  switch (pol) {
    case POL_BF16: return select_bf16(P);
    case POL_FP8: return select_kernel_fp8(P);
    case POL_TF32X3: return select_kernel_tf32(P);
    case POL_SLICED: return select_kernel_sliced(P);
    default: return nullptr;
  }
}

size_t solver_smem_bytes_lp(int P, int pol) {
  switch (pol) {
    case POL_BF16: return smem_bf16(P);
    case POL_FP8: return solver_smem_bytes_fp8(P);
    case POL_SLICED: return solver_smem_bytes_sliced(P);
    default: return solver_smem_bytes_tf32(P);
  }
}

}  // namespace ccg
