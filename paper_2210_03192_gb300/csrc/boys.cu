// Host construction of the Boys-function interpolation tables used by the
// integral kernels (paper Sec. 2.5.2: 7th-order Chebyshev interpolation on
// intervals, upward recursion in m beyond x = 117).
//
// Design on GB300: the kernels evaluate only the highest order F_L(T) and
// exp(-T) from the table (two degree-7 polynomials) and obtain F_m for
// m = L-1 .. lc by the downward relation (2m+1) F_m = 2T F_{m+1} + exp(-T),
// which is stable.  For T >= 117 exp(-T) is negligible next to every
// F_m (m <= 24) in FP64 and F_L = Gamma(L+1/2)/2 * T^{-(L+1/2)} exactly to
// FP64, so the same downward relation with exp(-T) = 0 applies.
//
// Reference values for the fit: F_m(T) = exp(-T) sum_i (2T)^i /
// ((2m+1)(2m+3)...(2m+2i+1)), a series of positive terms, summed in long double.
#include <cmath>

#include "lx3c_internal.h"

namespace lx3c {

long double boys_ref(int m, long double T) {
  long double term = 1.0L / (2 * m + 1), sum = term;
  for (int i = 1; i < 20000; ++i) {
    term *= 2.0L * T / (long double)(2 * m + 2 * i + 1);
    sum += term;
    if (term < 1e-30L * sum) break;
  }
  return std::exp(-T) * sum;
}

double boys_large_const(int L) {
  // Gamma(L + 1/2) / 2 = (2L-1)!! / 2^{L+1} * sqrt(pi)
  long double g = std::sqrt(3.14159265358979323846264338327950288L);
  for (int k = 1; k <= L; ++k) g *= (k - 0.5L);
  return (double)(g / 2.0L);
}

// tab[(i*kBoysNF + f)*8 + j]: coefficient of (T - mid_i)^j for function f
// (f <= kBoysMmax: F_f, f = kBoysMmax+1: exp(-T)) on interval i.
void boys_tables(std::vector<double>& tab, std::vector<double>& mid) {
  const int n = kBoysDeg + 1;
  tab.assign((size_t)kBoysNInt * kBoysNF * 8, 0.0);
  mid.assign(kBoysNInt, 0.0);
  const long double pi = 3.14159265358979323846264338327950288L;
  const long double h = 0.5L / kBoysPerUnit;  // half width
  for (int i = 0; i < kBoysNInt; ++i) {
    long double c = (i + 0.5L) / kBoysPerUnit;
    mid[i] = (double)c;
    long double xk[n], Tk[n];
    for (int k = 0; k < n; ++k) {
      xk[k] = std::cos(pi * (k + 0.5L) / n);
      Tk[k] = c + h * xk[k];
    }
    for (int f = 0; f < kBoysNF; ++f) {
      long double fk[n];
      for (int k = 0; k < n; ++k) fk[k] = (f <= kBoysMmax) ? boys_ref(f, Tk[k]) : std::exp(-Tk[k]);
      // Chebyshev coefficients of the interpolant
      long double cc[n];
      for (int j = 0; j < n; ++j) {
        long double s = 0;
        for (int k = 0; k < n; ++k) s += fk[k] * std::cos(pi * j * (k + 0.5L) / n);
        cc[j] = s * 2.0L / n;
      }
      cc[0] *= 0.5L;
      // monomial coefficients in x = (T - c)/h: sum_j cc_j T_j(x)
      long double mono[n] = {0}, tm2[n] = {0}, tm1[n] = {0}, tcur[n];
      tm2[0] = 1;  // T_0
      tm1[1] = 1;  // T_1
      for (int k = 0; k < n; ++k) mono[k] += cc[0] * tm2[k];
      if (n > 1)
        for (int k = 0; k < n; ++k) mono[k] += cc[1] * tm1[k];
      for (int j = 2; j < n; ++j) {
        for (int k = 0; k < n; ++k) tcur[k] = -tm2[k] + (k > 0 ? 2 * tm1[k - 1] : 0);
        for (int k = 0; k < n; ++k) mono[k] += cc[j] * tcur[k];
        for (int k = 0; k < n; ++k) { tm2[k] = tm1[k]; tm1[k] = tcur[k]; }
      }
      // rescale to powers of (T - c)
      long double sc = 1;
      for (int k = 0; k < n; ++k) {
        tab[((size_t)i * kBoysNF + f) * 8 + k] = (double)(mono[k] / sc);
        sc *= h;
      }
    }
  }
}

}  // namespace lx3c
