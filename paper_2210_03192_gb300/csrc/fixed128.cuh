// Exact, order-independent accumulation of FP64 contributions into
// fixed-point integers (DF-J gamma, J and gradient sums).  A contribution v
// is the two's-complement integer N = round(v * 2^kFixShift) of 128 bits,
// split as N = w2 2^64 + w1 2^32 + w0 with w0, w1 in [0, 2^32) and w2 the
// signed high word.  An accumulator is three 64-bit words {A0, A1, A2} that
// receive w0, w1 and w2 by three independent integer atomics (no return
// value, so no round trip: the adds are fire-and-forget reductions).  A0 and
// A1 take up to 2^32 contributions before a carry could be lost; the decode
// folds them, exactly, into the 128-bit total A2 2^64 + A1 2^32 + A0.
// Integer addition is associative, so the final words -- and the FP64 value
// read back from them -- do not depend on the order in which the
// contributions arrive: two executions of the same plan give bitwise equal
// results.
//   resolution 2^-72 (2.1e-22); range |sum| < 2^55 (3.6e16), and every
//   partial sum and contribution must stay inside it; at most 2^32
//   contributions per accumulator (the planners check the gradient's
//   per-atom counts; gamma and J elements get at most two per shell pair or
//   ket shell).
#pragma once
#include <cuda_runtime.h>

namespace lx3c {

constexpr int kFixShift = 72;
constexpr int kFixWords = 3;                     // 64-bit words per accumulator
constexpr int kFixBytes = 8 * kFixWords;         // bytes per accumulator
constexpr double kFixMaxAdds = 4294967296.0;     // contributions per accumulator

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
  const unsigned long long w0 = lo & 0xFFFFFFFFULL, w1 = lo >> 32;
  if (w0) atomicAdd(acc, w0);
  if (w1) atomicAdd(acc + 1, w1);
  if (hi) atomicAdd(acc + 2, hi);
}

// {A0, A1, A2} -> the nearest FP64 value of N 2^-72 (to within an ulp).
__device__ __forceinline__ double fix_decode(const unsigned long long* acc) {
  const unsigned long long a0 = acc[0], a1 = acc[1], a2 = acc[2];
  unsigned long long lo = a0 + (a1 << 32);
  unsigned long long hi = (a1 >> 32) + (lo < a0 ? 1ULL : 0ULL) + a2;
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
