// recurrence.h -- coefficients of the x^2 recurrence of Section 2.3, shared
// by the host and the device builders of the factorization.
#pragma once

#include <math.h>

#if defined(__CUDACC__)
#define SHT_HD __host__ __device__
#else
#define SHT_HD
#endif

namespace sht {

// x^2 P-bar^m_k = c_{k-2} P-bar^m_{k-2} + d_k P-bar^m_k + c_k P-bar^m_{k+2}
// (Section 2.3, eqs. c_rec, d_rec).
SHT_HD inline double rec_c(int k, int m) {
  const double a = (double)(k - m + 1) * (k - m + 2) * (double)(k + m + 1) * (k + m + 2);
  const double b = (2.0 * k + 1.0) * (2.0 * k + 3.0) * (2.0 * k + 3.0) * (2.0 * k + 5.0);
  return sqrt(a / b);
}
SHT_HD inline double rec_d(int k, int m) {
  return (2.0 * k * (k + 1.0) - 2.0 * (double)m * m - 1.0) / ((2.0 * k - 1.0) * (2.0 * k + 3.0));
}

}  // namespace sht
