// Hyperspherical-cap volume fraction in FP64 (host and device).
//
// Sec. 5 "Intersection Volume Approximation": the share of the ball B(q, rho)
// beyond a hyperplane at distance t from q is a cap; by Li (2010) its volume
// fraction is u = 1/2 I_x((d+1)/2, 1/2) with x = 1 - (t/rho)^2 (t < rho).
//
// I_x(a, b) is evaluated from the continued fraction of DLMF 8.17.22,
//   I_x(a,b) = x^a (1-x)^b / (a B(a,b)) * 1 / (1 + d1/(1 + d2/(1 + ...))),
//   d_{2m}   =  m (b - m) x / ((a + 2m - 1)(a + 2m)),
//   d_{2m+1} = -(a + m)(a + b + m) x / ((a + 2m)(a + 2m + 1)),
// summed by the modified Lentz method (Lentz 1976; Thompson & Barnett 1986),
// with the reflection I_x(a,b) = 1 - I_{1-x}(b,a) when x > (a+1)/(a+b+2), where
// the fraction converges slowly.  log B(a,b) comes from lgamma.
#pragma once

#include <math.h>

namespace qk {

constexpr int kBetaTablePoints = 1024;

// The continued fraction 1 + d1/(1 + d2/(1 + ...)) by modified Lentz.
__host__ __device__ inline double beta_cf_lentz(double a, double b, double x) {
  const double tiny = 1e-300;
  double f = 1.0, C = 1.0, D = 0.0;
  for (int j = 1; j <= 4000; ++j) {
    double dj;
    if (j & 1) {
      double m = 0.5 * (j - 1);
      dj = -(a + m) * (a + b + m) * x / ((a + 2.0 * m) * (a + 2.0 * m + 1.0));
    } else {
      double m = 0.5 * j;
      dj = m * (b - m) * x / ((a + 2.0 * m - 1.0) * (a + 2.0 * m));
    }
    D = 1.0 + dj * D;
    if (fabs(D) < tiny) D = tiny;
    D = 1.0 / D;
    C = 1.0 + dj / C;
    if (fabs(C) < tiny) C = tiny;
    double delta = C * D;
    f *= delta;
    if (fabs(delta - 1.0) < 1e-16) break;
  }
  return f;
}

// Regularised incomplete beta I_x(a, b) for x in [0, 1]; lnB = log B(a, b).
__host__ __device__ inline double inc_beta(double a, double b, double x, double lnB) {
  if (!(x > 0.0)) return 0.0;
  if (!(x < 1.0)) return 1.0;
  double lx = log(x), l1x = log1p(-x);
  double pre = exp(a * lx + b * l1x - lnB);
  if (x < (a + 1.0) / (a + b + 2.0)) return pre / (a * beta_cf_lentz(a, b, x));
  return 1.0 - pre / (b * beta_cf_lentz(b, a, 1.0 - x));
}

// Cap fraction u(t, rho) in dimension d (a = (d+1)/2, b = 1/2), exact mode.
__host__ __device__ inline double cap_fraction_exact(double t, double rho, double a, double lnB) {
  if (!(rho > 0.0) || !(t < rho)) return 0.0;
  double s = t / rho;
  return 0.5 * inc_beta(a, 0.5, 1.0 - s * s, lnB);
}

// Cap fraction with I_x linearly interpolated in the table at x_j = j/1023.
__host__ __device__ inline double cap_fraction_table(double t, double rho, const double* table) {
  if (!(rho > 0.0) || !(t < rho)) return 0.0;
  double s = t / rho;
  double x = 1.0 - s * s;
  double f = x * (kBetaTablePoints - 1);
  int j = static_cast<int>(floor(f));
  if (j < 0) j = 0;
  if (j > kBetaTablePoints - 2) j = kBetaTablePoints - 2;
  double w = f - j;
  double lo = table[j], hi = table[j + 1];
  return 0.5 * (lo + w * (hi - lo));
}

// The cap fraction as the search kernels evaluate it during Algorithm 1:
// inv = 1 / rho computed once per recompute by the caller; exact selects the
// continued fraction, else the table.  Every kernel that estimates p uses
// this one function, so they take identical decisions.
__device__ inline double cap_u(double t, double rho, double inv, bool exact, const double* table, double a,
                               double lnB) {
  if (!(rho > 0.0 && t < rho)) return 0.0;
  if (exact) return cap_fraction_exact(t, rho, a, lnB);
  const double sc = t * inv;
  const double x = 1.0 - sc * sc;
  const double f = x * (kBetaTablePoints - 1);
  int j = (int)f;
  if (j > kBetaTablePoints - 2) j = kBetaTablePoints - 2;
  const double lo = table[j], hi = table[j + 1];
  return 0.5 * (lo + (f - j) * (hi - lo));
}

}  // namespace qk
