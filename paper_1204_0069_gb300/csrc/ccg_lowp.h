// ccg_lowp.h -- internal interface of the tensor-core low-precision block
// product (ccg_lowp.cu).  Not part of the public ABI.
#pragma once

#include <cstdint>
#include <cuda.h>
#include <cuda_runtime.h>

namespace ccg {
namespace lp {

enum Kind : int { KIND_BF16 = 0, KIND_FP8 = 1, KIND_TF32X3 = 2, KIND_SLICED = 3 };
// Slices of the sliced FP64 format (equal to the device-side kSlices).
constexpr int kSlicesHost = 14;

// Launch description of one stream-K block product.
struct LpRun {
  int64_t n;               // rows = columns of A
  int64_t units;           // row tiles x k-chunks
  int kc;                  // k-chunks per row tile
  int k_elems;             // K elements per chunk (128 bytes)
  int ctas;                // grid size
  int pad;
  float* part;             // partial tiles, part_floats(n, ctas, NP) floats
  int* error;              // device error flag (0 = ok, -5 = wait timed out)
  long long timeout_ns;    // mbarrier wait limit
  const float* row_scale;  // FP8: per-row scale of A (else NULL)
  const float* col_scale;  // FP8: per-column scale of D (else NULL)
};

// Leading dimension (elements) of a quantised operand row: n rounded up to 128.
int64_t ld_elems(int64_t n);
// Floats of partial-tile storage for a launch on `ctas` CTAs with N = NP.
size_t part_floats(int64_t n, int ctas, int NP);
// A (FP64) -> Q: BF16, FP8 E4M3 with per-row scales (row_scale, n floats), or FP32.
// KIND_SLICED: kSlices FP8 slices stacked slice-major, each slice_rows() rows
// of ldq bytes, with one power-of-two scale per row (row_scale).
cudaError_t quantize(int kind, const double* A, int64_t lda, int64_t n, void* Q, int64_t ldq,
                     float* row_scale, cudaStream_t s);
// Upper bound on the eigenvalues of the copy of A quantised to `kind`
// (Gershgorin on the FP64 A with the format's rounding), as the bits of a
// double in *out (device memory).
cudaError_t eig_bound(int kind, const double* A, int64_t lda, int64_t n,
                      unsigned long long* out, cudaStream_t s);
// Rows of one slice of the sliced FP64 format (n rounded up to 128).
int64_t slice_rows(int64_t n);
// V (FP64, n x q row-major) -> Vt: NP (BF16) or 2 NP (FP8 hi, lo) rows of ldk
// elements, K contiguous; FP8 also writes the column scales (cmax: 32 uints).
cudaError_t convert_operand(int kind, const double* V, int64_t n, int q, int NP, void* Vt,
                            int64_t ldk, unsigned int* cmax, float* col_scale, cudaStream_t s);
// 2-D TMA tensor map over a rows x cols operand (K contiguous, ld elements),
// box of box_rows x 128 bytes, 128-byte swizzle.
bool make_tensor_map(CUtensorMap* m, const void* base, int kind, int64_t rows, int64_t cols,
                     int64_t ld, int box_rows);
// W (FP64, n x q) = A_lp V_lp; events (optional) bracket the two kernels.
cudaError_t block_product(int kind, int NP, const void* Q, int64_t ldq, const void* Vt,
                          int64_t ldk, LpRun run, int q, double* W, cudaStream_t s,
                          cudaEvent_t ev0, cudaEvent_t ev1);

}  // namespace lp
}  // namespace ccg
