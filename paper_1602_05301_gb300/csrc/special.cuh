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

__device__ __forceinline__ void hankel01(double x, cd& h0, cd& h1) {
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
