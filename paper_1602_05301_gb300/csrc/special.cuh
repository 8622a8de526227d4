// Device special functions for the 2D Helmholtz kernels.
//
//  * H_0, H_1 of the first kind: the ascending series below a series reach
//    (x < 5, or x < 8 for the mixed path), the CUDA math library's
//    j0/y0/j1/y1 (FP64) above it.
//  * H_m, m >= 2: upward three-term recurrence H_{m+1} = (2m/x) H_m - H_{m-1}
//    (DLMF 10.6.1), stable for the dominant Y part; the error of the J part
//    stays at rounding level relative to |H_m|.
//  * J_0..J_p: Miller's backward recurrence (DLMF 3.6(iii)) normalised by the
//    Neumann sum J_0 + 2 sum_{k>=1} J_{2k} = 1 (DLMF 10.12.4), with rescaling
//    against overflow; no library call.
#pragma once
#include "qbx_internal.h"

// Coefficients of the ascending series below, as compile-time constants:
// j0 = 1/(k!)^2, j1 = 1/(k!(k+1)!), h = H_k = 1 + 1/2 + ... + 1/k,
// y0 = H_k/(k!)^2, y1 = (psi(k+1) + psi(k+2))/(k!(k+1)!), psi(m) = -gamma + H_{m-1}.
constexpr double kEulerGamma = 0.57721566490153286061;
template <int K>
struct SeriesCoef {
  static constexpr double j0 = SeriesCoef<K - 1>::j0 / ((double)K * (double)K);
  static constexpr double j1 = SeriesCoef<K - 1>::j1 / ((double)K * (double)(K + 1));
  static constexpr double h = SeriesCoef<K - 1>::h + 1.0 / (double)K;
  static constexpr double y0 = h * j0;
  static constexpr double y1 = (-2.0 * kEulerGamma + h + (h + 1.0 / (double)(K + 1))) * j1;
};
template <>
struct SeriesCoef<0> {
  static constexpr double j0 = 1.0, j1 = 1.0, h = 0.0, y0 = 0.0;
  static constexpr double y1 = -2.0 * kEulerGamma + 1.0;
};

// Horner steps k = K, K-1, ..., 0 for the four polynomials in u.
template <int K>
struct SeriesHorner {
  __device__ __forceinline__ static void run(double u, double& pj0, double& pj1, double& py0,
                                             double& py1) {
    pj0 = fma(pj0, u, SeriesCoef<K>::j0);
    pj1 = fma(pj1, u, SeriesCoef<K>::j1);
    py0 = fma(py0, u, SeriesCoef<K>::y0);
    py1 = fma(py1, u, SeriesCoef<K>::y1);
    SeriesHorner<K - 1>::run(u, pj0, pj1, py0, py1);
  }
};
template <>
struct SeriesHorner<-1> {
  __device__ __forceinline__ static void run(double, double&, double&, double&, double&) {}
};

// H_0 and H_1 from the ascending series (DLMF 10.2.2 for J, DLMF 10.8.1 for
// Y), in u = -x^2/4:
//   J0 = sum u^k / (k!)^2,            J1 = (x/2) sum u^k / (k! (k+1)!),
//   Y0 = (2/pi)(ln(x/2) + gamma) J0 - (2/pi) sum_{k>=1} H_k u^k / (k!)^2,
//   Y1 = -2/(pi x) + (2/pi) ln(x/2) J1 - (x/(2 pi)) sum (psi(k+1) + psi(k+2)) u^k / (k! (k+1)!),
// each sum a polynomial in u of degree KTOP evaluated by Horner's rule (one
// FMA per term). The truncation error falls below rounding for x < 2 at
// KTOP = 14, x < 5 at 18 and x < 8 at 20; beyond x = 2 the sums cancel (their
// terms add up to about I_0(x)), which bounds the error relative to |H_0|,
// |H_1| by 1e-14 for x < 5 and 3e-13 for x < 8 (checked against the library's
// j0/y0/j1/y1 by tests/test_special_gpu.py).
// ix = 1/x is passed in (callers get it from one reciprocal square root of r^2).
template <int KTOP>
__device__ __forceinline__ void hankel01_series_n(double x, double ix, cd& h0, cd& h1) {
  constexpr double kTwoOverPi = 0.63661977236758134308;
  const double u = -0.25 * x * x;
  double pj0 = SeriesCoef<KTOP>::j0, pj1 = SeriesCoef<KTOP>::j1;
  double py0 = SeriesCoef<KTOP>::y0, py1 = SeriesCoef<KTOP>::y1;
  SeriesHorner<KTOP - 1>::run(u, pj0, pj1, py0, py1);
  const double lx = log(0.5 * x);
  const double J0 = pj0, J1 = 0.5 * x * pj1;
  const double Y0 = kTwoOverPi * ((lx + kEulerGamma) * J0 - py0);
  const double Y1 = -kTwoOverPi * ix + kTwoOverPi * lx * J1 - (0.5 * x) * (0.5 * kTwoOverPi) * py1;
  h0 = mk(J0, Y0);
  h1 = mk(J1, Y1);
}

__device__ __forceinline__ void hankel01_series(double x, double ix, cd& h0, cd& h1) {
  hankel01_series_n<14>(x, ix, h0, h1);
}
__device__ __forceinline__ void hankel01_series(double x, cd& h0, cd& h1) {
  hankel01_series_n<14>(x, 1.0 / x, h0, h1);
}

// Series reach of hankel01 (FP64 accuracy) and of hankel01_wide (relative
// error below 3e-13, for the mixed-precision path whose Hankel values are
// rounded to FP32 after the FP64 recurrence).
constexpr double kSeriesMax = 5.0, kSeriesMaxWide = 8.0;

// H_0, H_1 at x > 0. The lanes of a warp usually see arguments of one range:
// when all of them are below 2 the short series serves all, otherwise the
// longer one serves every lane below the series reach (one path, not two),
// and the library's j0/y0/j1/y1 the rest.
// NEED0 / NEED1: whether the caller reads h0 / h1 (the library calls of the
// other are skipped; the series parts it does not read are dead code).
template <bool WIDE, bool NEED0 = true, bool NEED1 = true>
__device__ __forceinline__ void hankel01_any(double x, double ix, cd& h0, cd& h1) {
  if (__all_sync(__activemask(), x < 2.0)) {
    hankel01_series_n<14>(x, ix, h0, h1);
    return;
  }
  if (x < (WIDE ? kSeriesMaxWide : kSeriesMax)) {
    if (WIDE)
      hankel01_series_n<20>(x, ix, h0, h1);
    else
      hankel01_series_n<18>(x, ix, h0, h1);
    return;
  }
  if (NEED0) h0 = mk(j0(x), y0(x));
  if (NEED1) h1 = mk(j1(x), y1(x));
}

__device__ __forceinline__ void hankel01(double x, double ix, cd& h0, cd& h1) {
  hankel01_any<false>(x, ix, h0, h1);
}
__device__ __forceinline__ void hankel01(double x, cd& h0, cd& h1) {
  hankel01_any<false>(x, 1.0 / x, h0, h1);
}
__device__ __forceinline__ void hankel01_wide(double x, double ix, cd& h0, cd& h1) {
  hankel01_any<true>(x, ix, h0, h1);
}

// An FP64 value rounded to FP32 with integer instructions only: on GB300 the
// conversion instruction occupies the FP64 pipe, which the mixed-precision
// kernels keep busy with their recurrences. IEEE binary64 -> binary32 by the
// bit fields: exponent rebiased (1023 -> 127), the top 23 of the 52 mantissa
// bits kept and the result rounded to nearest by adding the next bit (ties
// away from zero; a carry into the exponent is the correct result). Results
// below the FP32 normal range (|v| < 2^-126) become zero, above it infinity;
// NaN stays NaN.
__device__ __forceinline__ float f32_from_f64(double v) {
  const unsigned hi = (unsigned)__double2hiint(v), lo = (unsigned)__double2loint(v);
  const unsigned e64 = (hi >> 20) & 0x7FFu;
  const int e = (int)e64 - 896;  // 1023 - 127
  unsigned bits = ((unsigned)e << 23) + (((hi & 0xFFFFFu) << 3) | (lo >> 29)) + ((lo >> 28) & 1u);
  bits = e <= 0 ? 0u : bits;
  bits = e >= 255 ? 0x7F800000u : bits;
  bits = e64 == 0x7FFu && (((hi & 0xFFFFFu) | lo) != 0u) ? 0x7FC00000u : bits;
  return __uint_as_float(bits | (hi & 0x80000000u));
}

// f32_from_f64(v * 2^sh) without the multiplication: the exponent field is
// offset before the rounding (zero stays zero)
__device__ __forceinline__ float f32_from_f64_sh(double v, int sh) {
  const unsigned hi = (unsigned)__double2hiint(v), lo = (unsigned)__double2loint(v);
  const unsigned e64 = (hi >> 20) & 0x7FFu;
  const int e = (int)e64 - 896 + sh;
  unsigned bits = ((unsigned)e << 23) + (((hi & 0xFFFFFu) << 3) | (lo >> 29)) + ((lo >> 28) & 1u);
  bits = (e <= 0 || e64 == 0u) ? 0u : bits;
  bits = e >= 255 ? 0x7F800000u : bits;
  bits = e64 == 0x7FFu ? ((((hi & 0xFFFFFu) | lo) != 0u) ? 0x7FC00000u : 0x7F800000u) : bits;
  return __uint_as_float(bits | (hi & 0x80000000u));
}

// Split form of values whose range exceeds FP32: v = m 2^e with FP32
// mantissas m (the larger component's magnitude in [1, 2)) and an integer
// exponent e; zero (and FP64 subnormals) give m = 0, e = kZeroExp. Integer
// instructions only (field arithmetic on the IEEE bit patterns).
constexpr int kZeroExp = -(1 << 20);
// x (exponent field ex, high word hx) times 2^-(E - 1023), as FP32
__device__ __forceinline__ float split_part(double x, unsigned hx, int ex, int E) {
  const int f = ex - E + 1023;  // new exponent field
  if (ex == 0 || f < 1) return 0.f;
  const unsigned h2 = (hx & 0x800FFFFFu) | ((unsigned)f << 20);
  return f32_from_f64(__hiloint2double((int)h2, __double2loint(x)));
}
// two complex values sharing one exponent (e.g. H_m e^{+-i m th}, of equal modulus)
__device__ __forceinline__ void split_pair(cd a, cd b, float2& ma, float2& mb, int& e) {
  const unsigned h0 = (unsigned)__double2hiint(a.x), h1 = (unsigned)__double2hiint(a.y);
  const unsigned h2 = (unsigned)__double2hiint(b.x), h3 = (unsigned)__double2hiint(b.y);
  const int e0 = (h0 >> 20) & 0x7FF, e1 = (h1 >> 20) & 0x7FF;
  const int e2 = (h2 >> 20) & 0x7FF, e3 = (h3 >> 20) & 0x7FF;
  const int E = max(max(e0, e1), max(e2, e3));
  if (E == 0) {
    ma = mb = make_float2(0.f, 0.f);
    e = kZeroExp;
    return;
  }
  e = E - 1023;
  ma = make_float2(split_part(a.x, h0, e0, E), split_part(a.y, h1, e1, E));
  mb = make_float2(split_part(b.x, h2, e2, E), split_part(b.y, h3, e3, E));
}
__device__ __forceinline__ void split_one(cd a, float2& m, int& e) {
  float2 dummy;
  split_pair(a, mk(0.0, 0.0), m, dummy, e);
}
// 2^d as FP32 for d <= 127 (0 below the normal range)
__device__ __forceinline__ float pow2f(int d) {
  return d < -126 ? 0.f : __int_as_float((d + 127) << 23);
}
// 2^d as FP64 (0 below the normal range, infinity above it)
__device__ __forceinline__ double pow2d(int d) {
  if (d < -1022) return 0.0;
  if (d > 1023) return __longlong_as_double(0x7FF0000000000000ll);
  return __hiloint2double((d + 1023) << 20, 0);
}

// Start index of the backward recurrence for orders 0..pmax at argument x:
// far enough above m = max(pmax, x) that the recurrence has converged to the
// minimal solution to full double precision. The relative error of J_m from a
// start N is about (x/2)^{2(N-m)} (m!/N!)^2, so for x well below m a dozen
// orders suffice; the sqrt(40 x) term keeps the classical margin of order
// sqrt(m) where x approaches m (the transition region).
__device__ __forceinline__ int miller_start(int pmax, double x) {
  int m = pmax > (int)x ? pmax : (int)x;
  int n = m + 12 + (int)(2.0 * sqrt(40.0 * x));
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
