// Host build of the solver's long accumulator (paper_1204_0069_gb300/csrc/
// ccg_xacc.h) for the CPU tests: the same source the kernels compile, with the
// portable carry chains in place of the inline PTX.
#include "ccg_xacc.h"

extern "C" int xacc_dot(const double* x, const double* y, long n, int fixed_anchor,
                        double* out) {
  ccg::XAcc a;
  ccg::xacc_init(a);
  if (fixed_anchor) {
    int K = 2;
    for (long i = 0; i < n; ++i) K = ccg::xacc_max(K, ccg::xacc_expsum(x[i], y[i]));
    a.K = K;
    for (long i = 0; i < n; ++i) ccg::xacc_fma_k(a, x[i], y[i]);
  } else {
    for (long i = 0; i < n; ++i) ccg::xacc_fma(a, x[i], y[i]);
  }
  const ccg::DSum d = ccg::xacc_value(a);
  out[0] = d.hi;
  out[1] = d.lo;
  return 0;
}
