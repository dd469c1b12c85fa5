// ccg_xacc.h -- exact accumulation of FP64 products in integer arithmetic (a
// long accumulator in the sense of Kulisch, restricted to a window), used by
// the solver kernels for the per-lane sums of the p x p Grams and residue
// norms (Table 1, rows 2-3 and 5-7).  On GB300 the FP64 pipe retires about two
// operations per SM and clock, so a compensated product-sum (Dot2: about ten
// FP64 operations per term) is slow there, while integer operations run at
// 64 times that rate.
//
// The sum of x_i y_i is held as a signed 192-bit integer w (two's complement,
// three 64-bit words) times 2^(K - 2203), where K is the largest biased
// exponent sum e(x_i) + e(y_i) of the terms (subnormals count as exponent 1).
// The product P of the two 53-bit significands (< 2^106) enters as
// (P 2^53) >> (K - e): the largest products occupy bits below 159 (2^32 terms
// of headroom), and a product 2^-150 or more below the largest loses the bits
// that fall beneath the window.  An Inf or NaN operand makes the value NaN.
// The value is returned as the unevaluated pair hi + lo of its top 106 bits.
//
// Everything here compiles for the device (inline PTX carry chains) and for
// the host (the same arithmetic in portable C++), so the host build can be
// checked against exact rational sums without a GPU.
#pragma once

#include <cmath>
#include <cstdint>
#include <cstring>

#if defined(__CUDACC__)
#define CCG_XHD __host__ __device__ __forceinline__
#else
#define CCG_XHD inline
#endif

namespace ccg {

// An unevaluated sum hi + lo (also the running state of Dot2).
struct DSum {
  double hi;
  double lo;
};

struct XAcc {
  unsigned long long w0, w1, w2;  // w2 carries the sign (two's complement)
  int K;
  int bad;
};

CCG_XHD unsigned long long xacc_bits(double x) {
#if defined(__CUDA_ARCH__)
  return (unsigned long long)__double_as_longlong(x);
#else
  unsigned long long u;
  std::memcpy(&u, &x, sizeof u);
  return u;
#endif
}
CCG_XHD unsigned long long xacc_mulhi(unsigned long long a, unsigned long long b) {
#if defined(__CUDA_ARCH__)
  return __umul64hi(a, b);
#else
  return (unsigned long long)(((unsigned __int128)a * b) >> 64);
#endif
}
CCG_XHD int xacc_clz(unsigned long long v) {  // v != 0
#if defined(__CUDA_ARCH__)
  return __clzll((long long)v);
#else
  return __builtin_clzll(v);
#endif
}
CCG_XHD int xacc_max(int a, int b) { return a > b ? a : b; }
CCG_XHD int xacc_min(int a, int b) { return a < b ? a : b; }
// (w2:w1:w0) += (r2:r1:r0) modulo 2^192
CCG_XHD void xacc_add3(XAcc& a, unsigned long long r0, unsigned long long r1,
                       unsigned long long r2) {
#if defined(__CUDA_ARCH__)
  asm("add.cc.u64 %0, %0, %3;\n\taddc.cc.u64 %1, %1, %4;\n\taddc.u64 %2, %2, %5;"
      : "+l"(a.w0), "+l"(a.w1), "+l"(a.w2) : "l"(r0), "l"(r1), "l"(r2));
#else
  const unsigned long long s0 = a.w0 + r0;
  const unsigned long long c0 = s0 < r0;
  const unsigned long long t1 = a.w1 + r1;
  const unsigned long long c1 = t1 < r1;
  const unsigned long long s1 = t1 + c0;
  const unsigned long long c1b = s1 < c0;
  a.w0 = s0;
  a.w1 = s1;
  a.w2 = a.w2 + r2 + c1 + c1b;
#endif
}
// (w2:w1:w0) -= (r2:r1:r0) modulo 2^192
CCG_XHD void xacc_sub3(XAcc& a, unsigned long long r0, unsigned long long r1,
                       unsigned long long r2) {
#if defined(__CUDA_ARCH__)
  asm("sub.cc.u64 %0, %0, %3;\n\tsubc.cc.u64 %1, %1, %4;\n\tsubc.u64 %2, %2, %5;"
      : "+l"(a.w0), "+l"(a.w1), "+l"(a.w2) : "l"(r0), "l"(r1), "l"(r2));
#else
  xacc_add3(a, ~r0, ~r1, ~r2);
  xacc_add3(a, 1ull, 0ull, 0ull);
#endif
}

CCG_XHD void xacc_init(XAcc& a) {
  a.w0 = a.w1 = a.w2 = 0ull;
  a.K = -4096;
  a.bad = 0;
}
// arithmetic right shift of the accumulator by d >= 0 bits
CCG_XHD void xacc_shr(XAcc& a, int d) {
  const unsigned long long sg = (unsigned long long)((long long)a.w2 >> 63);
  if (d >= 192) {
    a.w0 = a.w1 = a.w2 = sg;
    return;
  }
  while (d >= 64) {
    a.w0 = a.w1;
    a.w1 = a.w2;
    a.w2 = sg;
    d -= 64;
  }
  if (d > 0) {
    a.w0 = (a.w0 >> d) | (a.w1 << (64 - d));
    a.w1 = (a.w1 >> d) | (a.w2 << (64 - d));
    a.w2 = (unsigned long long)((long long)a.w2 >> d);
  }
}
// w += x y exactly (within the window), moving the anchor up when a larger
// term arrives.
CCG_XHD void xacc_fma(XAcc& a, double x, double y) {
  const unsigned long long bx = xacc_bits(x), by = xacc_bits(y);
  const int ex = (int)(bx >> 52) & 0x7FF, ey = (int)(by >> 52) & 0x7FF;
  if ((ex == 0x7FF) | (ey == 0x7FF)) a.bad = 1;
  unsigned long long mx = bx & 0xFFFFFFFFFFFFFull, my = by & 0xFFFFFFFFFFFFFull;
  if (ex != 0) mx |= 1ull << 52;
  if (ey != 0) my |= 1ull << 52;
  if ((mx == 0ull) | (my == 0ull) | (a.bad != 0)) return;
  const int e = xacc_max(ex, 1) + xacc_max(ey, 1);
  if (e > a.K) {
    xacc_shr(a, e - a.K);
    a.K = e;
  }
  const int sh = a.K - e;
  const unsigned long long plo = mx * my, phi = xacc_mulhi(mx, my);
  unsigned long long q0, q1, q2 = 0ull;
  if (sh <= 53) {
    const int l = 53 - sh;  // 0..53
    q0 = plo << l;
    q1 = l ? (phi << l) | (plo >> (64 - l)) : phi;
    q2 = l ? (phi >> (64 - l)) : 0ull;
  } else {
    const int r = sh - 53;
    if (r >= 128) return;
    if (r >= 64) {
      q0 = phi >> (r - 64);
      q1 = 0ull;
    } else {
      q0 = r ? (plo >> r) | (phi << (64 - r)) : plo;
      q1 = phi >> r;
    }
  }
  if ((bx ^ by) >> 63) xacc_sub3(a, q0, q1, q2);
  else xacc_add3(a, q0, q1, q2);
}
// Biased exponent sum of a product (subnormals count as exponent 1): the
// anchor K of a sum fixed beforehand is the largest over its terms.
CCG_XHD int xacc_expsum(double x, double y) {
  const int ex = (int)(xacc_bits(x) >> 52) & 0x7FF;
  const int ey = (int)(xacc_bits(y) >> 52) & 0x7FF;
  return xacc_max(ex, 1) + xacc_max(ey, 1);
}
// An operand decoded once for many products: its significand with the hidden
// bit (bits 0-52) and its sign (bit 63) in one word, and its exponent (max(e,
// 1); 4096 for Inf and NaN, so that the exponent sum of any product with it
// is at least 4096 while finite sums stay below 4093).
CCG_XHD void xacc_decode(double x, unsigned long long& m, int& e) {
  const unsigned long long bx = xacc_bits(x);
  const int ex = (int)(bx >> 52) & 0x7FF;
  m = (bx & 0x800FFFFFFFFFFFFFull) | ((unsigned long long)(ex != 0) << 52);
  e = ex == 0x7FF ? 4096 : xacc_max(ex, 1);
}
// w += x y for decoded operands with exponent sum s, the anchor fixed
// beforehand (a.K >= every finite term's exponent sum): no re-anchoring and no
// branches, so unrolled terms interleave.  The product P enters as
// (P 2^53) >> (K - s), shifted by whole words and then bits with selects, and
// is added or subtracted through its two's complement.
CCG_XHD void xacc_fma_kd(XAcc& a, unsigned long long bx, unsigned long long by, int s) {
  a.bad |= (int)(s >= 4096);
  const unsigned long long mx = bx & 0x1FFFFFFFFFFFFFull, my = by & 0x1FFFFFFFFFFFFFull;
  const int sh = a.K - s;
  const unsigned long long plo = mx * my, phi = xacc_mulhi(mx, my);
  const unsigned long long q0 = plo << 53, q1 = (phi << 53) | (plo >> 11), q2 = phi >> 11;
  const int ws = xacc_min(sh >> 6, 3), bs = sh & 63;
  const unsigned long long w0 = ws == 0 ? q0 : ws == 1 ? q1 : ws == 2 ? q2 : 0ull;
  const unsigned long long w1 = ws == 0 ? q1 : ws == 1 ? q2 : 0ull;
  const unsigned long long w2 = ws == 0 ? q2 : 0ull;
  const unsigned long long m = 0ull - ((bx ^ by) >> 63);  // all ones: subtract
  const unsigned long long r0 = ((w0 >> bs) | ((w1 << 1) << (63 - bs))) ^ m;
  const unsigned long long r1 = ((w1 >> bs) | ((w2 << 1) << (63 - bs))) ^ m;
  const unsigned long long r2 = (w2 >> bs) ^ m;
  xacc_add3(a, r0, r1, r2);
  xacc_add3(a, m & 1ull, 0ull, 0ull);
}
// As xacc_fma with the anchor fixed beforehand, from the doubles themselves.
CCG_XHD void xacc_fma_k(XAcc& a, double x, double y) {
  unsigned long long mx, my;
  int ex, ey;
  xacc_decode(x, mx, ex);
  xacc_decode(y, my, ey);
  xacc_fma_kd(a, mx, my, ex + ey);
}
// 53 bits of the magnitude m starting at bit pos (zeros below bit 0)
CCG_XHD unsigned long long xacc_bits53(const unsigned long long m[3], int pos) {
  const unsigned long long kMask = (1ull << 53) - 1ull;
  if (pos <= -53) return 0ull;
  if (pos < 0) return (m[0] << (-pos)) & kMask;
  const int limb = pos >> 6, off = pos & 63;
  const unsigned long long lo = m[limb];
  const unsigned long long hi = limb < 2 ? m[limb + 1] : 0ull;
  return (off ? (lo >> off) | (hi << (64 - off)) : lo) & kMask;
}
CCG_XHD double xacc_from_bits(unsigned long long u) {
#if defined(__CUDA_ARCH__)
  return __longlong_as_double((long long)u);
#else
  double x;
  std::memcpy(&x, &u, sizeof x);
  return x;
#endif
}
// (-1)^sign m 2^s for an integer m < 2^53 (sgn: the sign bit).  A normal
// result is assembled from its bit fields (exact; integer operations only,
// where a conversion and ldexp cost several operations on the slow FP64
// pipe); a subnormal or overflowing one goes through ldexp, which rounds it.
CCG_XHD double xacc_scaled(unsigned long long m, int s, unsigned long long sgn) {
  if (m == 0ull) return xacc_from_bits(sgn);
  const int z = xacc_clz(m) - 11;    // leading zeros within the 53-bit field
  const int e = s + 52 - z + 1023;   // biased exponent once normalised
  if (e >= 1 && e <= 2046)
    return xacc_from_bits(sgn | ((unsigned long long)e << 52) | ((m << z) & 0xFFFFFFFFFFFFFull));
  const double v = ldexp((double)m, s);
  return sgn ? -v : v;
}
CCG_XHD DSum xacc_value(const XAcc& a) {
  if (a.bad) return DSum{NAN, 0.0};
  const bool neg = (long long)a.w2 < 0;
  XAcc mag = a;
  if (neg) {
    mag.w0 = ~a.w0;
    mag.w1 = ~a.w1;
    mag.w2 = ~a.w2;
    xacc_add3(mag, 1ull, 0ull, 0ull);
  }
  const unsigned long long m[3] = {mag.w0, mag.w1, mag.w2};
  int b;
  if (m[2]) b = 191 - xacc_clz(m[2]);
  else if (m[1]) b = 127 - xacc_clz(m[1]);
  else if (m[0]) b = 63 - xacc_clz(m[0]);
  else return DSum{0.0, 0.0};
  const unsigned long long sgn = neg ? 0x8000000000000000ull : 0ull;
  return DSum{xacc_scaled(xacc_bits53(m, b - 52), b - 52 + a.K - 2203, sgn),
              xacc_scaled(xacc_bits53(m, b - 105), b - 105 + a.K - 2203, sgn)};
}

}  // namespace ccg
