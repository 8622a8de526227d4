// Device special functions for the 2D Helmholtz kernels.
//
//  * H_0, H_1 of the first kind: the CUDA math library's j0/y0/j1/y1 (FP64).
//  * H_m, m >= 2: upward three-term recurrence H_{m+1} = (2m/x) H_m - H_{m-1}
//    (DLMF 10.6.1), stable for the dominant Y part; the error of the J part
//    stays at rounding level relative to |H_m|.
//  * J_0..J_p: Miller's backward recurrence (DLMF 3.6(iii)) normalised by the
//    Neumann sum J_0 + 2 sum_{k>=1} J_{2k} = 1 (DLMF 10.12.4), with rescaling
//    against overflow; no library call.
#pragma once
#include "qbx_internal.h"

// H_0 and H_1 for 0 < x < 2 from the ascending series (DLMF 10.2.2 for J,
// DLMF 10.8.1 for Y, z = x^2/4):
//   J0 = sum (-z)^k / (k!)^2,            J1 = (x/2) sum (-z)^k / (k! (k+1)!),
//   Y0 = (2/pi)(ln(x/2) + gamma) J0 - (2/pi) sum_{k>=1} H_k (-z)^k / (k!)^2,
//   Y1 = -2/(pi x) + (2/pi) ln(x/2) J1 - (x/(2 pi)) sum (psi(k+1) + psi(k+2)) (-z)^k / (k! (k+1)!),
// with H_k the harmonic numbers and psi(m) = -gamma + H_{m-1}. For z < 1 the
// terms fall below 1e-17 by k = 13; the sums are taken forward with the term
// ratios (compile-time constants after unrolling).
__device__ __forceinline__ void hankel01_series(double x, cd& h0, cd& h1) {
  const double kGamma = 0.57721566490153286061;
  const double kTwoOverPi = 0.63661977236758134308;
  const double mz = -0.25 * x * x;
  double t0 = 1.0, t1 = 1.0;          // (-z)^k/(k!)^2 and (-z)^k/(k!(k+1)!)
  double sj0 = 1.0, sj1 = 1.0;        // J series
  double sy0 = 0.0;                   // sum H_k t0
  double sy1 = 1.0 - 2.0 * kGamma;    // sum (psi(k+1)+psi(k+2)) t1, k = 0 term: -2g + 1
  double hk = 0.0;                    // H_k (a compile-time constant in each unrolled step)
#pragma unroll
  for (int k = 1; k <= 14; ++k) {
    hk += 1.0 / (double)k;
    // reciprocals of the integer ratios are compile-time constants: no division
    t0 *= mz * (1.0 / ((double)k * (double)k));
    t1 *= mz * (1.0 / ((double)k * (double)(k + 1)));
    sj0 += t0;
    sj1 += t1;
    sy0 = fma(hk, t0, sy0);
    // psi(k+1) + psi(k+2) = -2 gamma + H_k + H_{k+1}
    sy1 = fma(-2.0 * kGamma + 2.0 * hk + 1.0 / (double)(k + 1), t1, sy1);
  }
  const double lx = log(0.5 * x);
  const double J0 = sj0, J1 = 0.5 * x * sj1;
  const double Y0 = kTwoOverPi * ((lx + kGamma) * J0 - sy0);
  const double Y1 = -kTwoOverPi / x + kTwoOverPi * lx * J1 - (0.5 * x) * (0.5 * kTwoOverPi) * sy1;
  h0 = mk(J0, Y0);
  h1 = mk(J1, Y1);
}

__device__ __forceinline__ void hankel01(double x, cd& h0, cd& h1) {
  if (x < 2.0) {
    hankel01_series(x, h0, h1);
    return;
  }
  h0 = mk(j0(x), y0(x));
  h1 = mk(j1(x), y1(x));
}

// Start index of the backward recurrence for orders 0..pmax at argument x:
// far enough above max(pmax, x) that the recurrence has converged to the
// minimal solution to full double precision.
__device__ __forceinline__ int miller_start(int pmax, double x) {
  int m = pmax > (int)x ? pmax : (int)x;
  int n = m + 20 + (int)(2.0 * sqrt(40.0 * (double)(m + 1)));
  return (n + 1) & ~1;  // even
}

// J_0..J_{PM} (entries above p are not used by callers; they are computed anyway).
template <int PM>
__device__ __forceinline__ void bessel_j_array(double x, double (&J)[PM + 1]) {
#pragma unroll
  for (int i = 0; i <= PM; ++i) J[i] = 0.0;
  if (x < 1e-8) {  // leading series terms (x/2)^n / n!, relative error O(x^2)
    double t = 1.0;
#pragma unroll
    for (int i = 0; i <= PM; ++i) {
      J[i] = t;
      t *= 0.5 * x / (double)(i + 1);
    }
    return;
  }
  const double inv = 2.0 / x;
  int N = miller_start(PM, x);
  double fn1 = 0.0, fn = 1e-280, sum = 0.0;  // f_{n+1}, f_n
  for (int n = N; n >= 1; --n) {
    // f_{n-1} = (2n/x) f_n - f_{n+1}
    double fm = (double)n * inv * fn - fn1;
    if ((n & 1) == 0) sum += fn;  // even index n >= 2 contributes 2 f_n (counted below)
    if (n <= PM + 1) {
#pragma unroll
      for (int i = 0; i <= PM; ++i)
        if (i == n - 1) J[i] = fm;
    }
    fn1 = fn;
    fn = fm;
    if (fabs(fn) > 1e250) {  // rescale everything kept so far
      const double s = 1e-250;
      fn *= s;
      fn1 *= s;
      sum *= s;
#pragma unroll
      for (int i = 0; i <= PM; ++i) J[i] *= s;
    }
  }
  // fn now holds f_0; Neumann sum: f_0 + 2 * sum_{k>=1} f_{2k}
  const double norm = 1.0 / (fn + 2.0 * sum);
#pragma unroll
  for (int i = 0; i <= PM; ++i) J[i] *= norm;
}
