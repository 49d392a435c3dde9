// Exact, order-independent accumulation of FP64 contributions into 128-bit
// fixed-point integers (DF-J gamma, J and gradient sums).  A value v is held
// as the two's-complement integer N = round(v * 2^kFixShift) in two 64-bit
// words {lo, hi}; contributions are added with two 64-bit integer atomics,
// the carry out of the low word going into the high word.  Integer addition
// is associative, so the final words -- and the FP64 value read back from
// them -- do not depend on the order in which the contributions arrive: two
// executions of the same plan give bitwise equal results.
//   resolution 2^-72 (2.1e-22); range |sum| < 2^55 (3.6e16), and every
//   partial sum and contribution must stay inside it.
#pragma once
#include <cuda_runtime.h>

namespace lx3c {

constexpr int kFixShift = 72;

// v -> N = round(v * 2^72) (round half away from zero), as {lo, hi}.
__device__ __forceinline__ void fix_encode(double v, unsigned long long& lo, unsigned long long& hi) {
  const long long bits = __double_as_longlong(v);
  const int e = (int)((bits >> 52) & 0x7FF);
  lo = hi = 0ULL;
  if (e == 0) return;  // zero or subnormal: far below the resolution
  const unsigned long long m = (bits & ((1ULL << 52) - 1)) | (1ULL << 52);  // v = +-m 2^(e-1075)
  const int sh = e - 1075 + kFixShift;                                      // |N| = m 2^sh
  if (sh >= 64) {
    hi = m << (sh - 64);
  } else if (sh > 0) {
    lo = m << sh;
    hi = m >> (64 - sh);
  } else if (sh == 0) {
    lo = m;
  } else if (sh > -64) {
    lo = (m + (1ULL << (-sh - 1))) >> (-sh);
  }
  if (bits < 0) {  // two's complement negation
    lo = ~lo + 1ULL;
    hi = ~hi + (lo == 0ULL ? 1ULL : 0ULL);
  }
}

__device__ __forceinline__ void fix_add(unsigned long long* acc, double v) {
  unsigned long long lo, hi;
  fix_encode(v, lo, hi);
  if ((lo | hi) == 0ULL) return;
  const unsigned long long old = atomicAdd(acc, lo);
  atomicAdd(acc + 1, hi + (old + lo < old ? 1ULL : 0ULL));
}

// {lo, hi} -> the nearest FP64 value of N 2^-72 (to within an ulp).
__device__ __forceinline__ double fix_decode(const unsigned long long* acc) {
  unsigned long long lo = acc[0], hi = acc[1];
  const bool neg = (long long)hi < 0;
  if (neg) {
    lo = ~lo + 1ULL;
    hi = ~hi + (lo == 0ULL ? 1ULL : 0ULL);
  }
  const double mag = fma((double)hi, 18446744073709551616.0, (double)lo);
  const double v = ldexp(mag, -kFixShift);
  return neg ? -v : v;
}

}  // namespace lx3c
