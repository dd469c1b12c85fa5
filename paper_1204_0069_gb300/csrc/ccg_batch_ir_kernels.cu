// ccg_batch_ir_kernels.cu -- instantiations of the batched solver kernel with
// FP32 inner solves inside FP64 refinement, compiled apart from the other
// kernels so that the library builds in parallel.
#include <cuda_runtime.h>

#include "ccg_internal.h"
#include "ccg_solver.cuh"

namespace ccg {

void* select_batch_ir(int P) {
  switch (P) {
    case 1: return reinterpret_cast<void*>(&batch_ir_kernel<1>);
    case 2: return reinterpret_cast<void*>(&batch_ir_kernel<2>);
    case 4: return reinterpret_cast<void*>(&batch_ir_kernel<4>);
    case 8: return reinterpret_cast<void*>(&batch_ir_kernel<8>);
    case 16: return reinterpret_cast<void*>(&batch_ir_kernel<16>);
    case 32: return reinterpret_cast<void*>(&batch_ir_kernel<32>);
    default: return nullptr;
  }
}

}  // namespace ccg
