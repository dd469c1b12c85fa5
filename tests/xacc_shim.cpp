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

// The value of the accumulator written with a conversion and ldexp per part
// (the textbook route: (double) of a 53-bit integer is exact, ldexp scales
// exactly unless the result is subnormal), to pin the bit-field assembly of
// xacc_value against.
extern "C" int xacc_dot_ldexp(const double* x, const double* y, long n, double* out) {
  ccg::XAcc a;
  ccg::xacc_init(a);
  for (long i = 0; i < n; ++i) ccg::xacc_fma(a, x[i], y[i]);
  if (a.bad) {
    out[0] = NAN;
    out[1] = 0.0;
    return 0;
  }
  const bool neg = (long long)a.w2 < 0;
  ccg::XAcc mag = a;
  if (neg) {
    mag.w0 = ~a.w0;
    mag.w1 = ~a.w1;
    mag.w2 = ~a.w2;
    ccg::xacc_add3(mag, 1ull, 0ull, 0ull);
  }
  const unsigned long long m[3] = {mag.w0, mag.w1, mag.w2};
  int b;
  if (m[2]) b = 191 - ccg::xacc_clz(m[2]);
  else if (m[1]) b = 127 - ccg::xacc_clz(m[1]);
  else if (m[0]) b = 63 - ccg::xacc_clz(m[0]);
  else {
    out[0] = out[1] = 0.0;
    return 0;
  }
  const double hi = std::ldexp((double)ccg::xacc_bits53(m, b - 52), b - 52 + a.K - 2203);
  const double lo = std::ldexp((double)ccg::xacc_bits53(m, b - 105), b - 105 + a.K - 2203);
  out[0] = neg ? -hi : hi;
  out[1] = neg ? -lo : lo;
  return 0;
}
