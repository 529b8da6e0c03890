// FP64 exponential for the coefficient field, table-driven after
// P. T. P. Tang, "Table-driven implementation of the exponential function in
// IEEE floating-point arithmetic", ACM TOMS 15(2), 1989:
//
//   t = (64 m + j) ln2/64 + r,   |r| <= ln2/128,   0 <= j < 64,
//   exp(t) = 2^m * 2^(j/64) * exp(r),
//
// with k = 64 m + j the nearest integer to t * 64/ln2, r from a two-part
// ln2/64 by fused multiply-adds, and exp(r) - 1 by its degree-5 Taylor
// polynomial (truncation below r^6/720 < 3.6e-17).  The 64 table values
// 2^(j/64) live in shared memory (the caller fills them with exp_table_fill).
// Error: below about 1.5 ulp for |t| <= 700; outside that range the CUDA
// library exp is used.  About 11 FP64 operations against the library's
// general-purpose routine, which matters on a part with a small FP64 pipe.
#pragma once
#include "common.cuh"

namespace stomsfem {

constexpr double kLn2 = 0.6931471805599453;                 // nearest double to ln 2
constexpr double kLn2Err = 2.3190468138462996e-17;          // ln 2 - kLn2
constexpr double kLn2By64Hi = kLn2 / 64.0;                  // exact division
constexpr double kLn2By64Lo = kLn2Err / 64.0;
constexpr double k64ByLn2 = 92.33248261689366;              // 64 / ln 2 (rounding is harmless)
constexpr double kRoundShift = 6755399441055744.0;          // 1.5 * 2^52: adding it rounds to an integer

// tab[j] = 2^(j/64), j = 0..63, for the block (all threads call, then sync).
__device__ __forceinline__ void exp_table_fill(double* tab) {
  for (int j = threadIdx.x; j < 64; j += blockDim.x) tab[j] = exp2((double)j / 64.0);
}

__device__ __forceinline__ double fexp(double t, const double* tab) {
  if (!(fabs(t) <= 700.0)) return exp(t);  // also NaN
  const double ks = fma(t, k64ByLn2, kRoundShift);
  const int k = __double2loint(ks);        // low word = the rounded integer (two's complement)
  const double kd = ks - kRoundShift;
  double r = fma(-kd, kLn2By64Hi, t);
  r = fma(-kd, kLn2By64Lo, r);
  double q = fma(r, 1.0 / 120.0, 1.0 / 24.0);
  q = fma(r, q, 1.0 / 6.0);
  q = fma(r, q, 0.5);
  q = fma(r, q, 1.0);
  const double p = r * q;                  // exp(r) - 1
  const double tj = tab[k & 63];
  const double v = fma(tj, p, tj);
  const int m = k >> 6;                    // floor(k / 64)
  return v * __longlong_as_double((long long)(m + 1023) << 52);
}

}  // namespace stomsfem
