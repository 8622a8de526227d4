// Device special functions for the 2D Helmholtz kernels.
//
//  * H_0, H_1 of the first kind: piecewise polynomials below x = 8
//    (Chebyshev fits on eight intervals per octave from 2^-9, the economised
//    ascending series below), the CUDA math library's j0/y0/j1/y1 (FP64) above.
//  * H_m, m >= 2: upward three-term recurrence H_{m+1} = (2m/x) H_m - H_{m-1}
//    (DLMF 10.6.1), stable for the dominant Y part; the error of the J part
//    stays at rounding level relative to |H_m|.
//  * J_0..J_p: Miller's backward recurrence (DLMF 3.6(iii)) normalised by the
//    Neumann sum J_0 + 2 sum_{k>=1} J_{2k} = 1 (DLMF 10.12.4), with rescaling
//    against overflow; no library call.
#pragma once
#include "qbx_internal.h"

// Polynomial pieces of H_0 and H_1 below x = 8 (generated tables, see
// gen_hankel_table.py): eight intervals per octave from 2^-9 to 8 with
// degree-D Chebyshev fits of J_0, Y_0, J_1, Y_1 in t in [-1, 1] (the
// partition is geometric, so one degree serves every octave), and the
// ascending series (DLMF 10.2.2, 10.8.1) economised to degree D on
// u = -x^2/4 in [-1, 0] for x < 2^-9. D = 10 for the FP64 path (truncation
// near 1e-16 of |H_0|, |H_1|), 8 for the mixed path (near 1e-13).
#include "hankel_table.h"
constexpr double kEulerGamma = 0.57721566490153286061;
constexpr double kTwoOverPi = 0.63661977236758134308;

template <bool WIDE>
struct HankTab;
template <>
struct HankTab<false> {
  static constexpr int D = kHankDeg64;
  __device__ static const double2* tab() { return kHankTab64; }
};
template <>
struct HankTab<true> {
  static constexpr int D = kHankDegMx;
  __device__ static const double2* tab() { return kHankTabMx; }
};

// The logarithmic terms of the ascending series: from the four series sums
// J0, P1 = J1 / (x/2), R0, R1 in u = -x^2/4,
//   Y0 = (2/pi)((ln(x/2) + gamma) J0 - R0),
//   Y1 = -2/(pi x) + (2/pi) ln(x/2) J1 - (x/(2 pi)) R1.
template <bool NEED0, bool NEED1>
__device__ __forceinline__ void hankel01_from_series(double x, double ix, double j0s, double r0s,
                                                     double p1s, double r1s, cd& h0, cd& h1) {
  const double lx = log(0.5 * x);
  if (NEED0) h0 = mk(j0s, kTwoOverPi * ((lx + kEulerGamma) * j0s - r0s));
  if (NEED1) {
    const double J1 = 0.5 * x * p1s;
    h1 = mk(J1, -kTwoOverPi * ix + kTwoOverPi * lx * J1 - (0.5 * x) * (0.5 * kTwoOverPi) * r1s);
  }
}

// H_0, H_1 at 0 < x < 8 from the tables: each lane evaluates its own row (its
// interval, or the series row below 2^-9) by Horner's rule, two FMAs per
// degree for each function read; lanes on the series row add the logarithmic
// terms.
template <bool WIDE, bool NEED0, bool NEED1>
__device__ __forceinline__ void hankel01_table(double x, double ix, cd& h0, cd& h1) {
  using T = HankTab<WIDE>;
  constexpr double kTiny = 0x1p-9;  // 2^kHankMinExp
  static_assert(kHankMinExp == -9, "table floor");
  const bool small = x < kTiny;
  // interval row from the bit fields of x: 8 (E + 9) + j from the biased
  // exponent and the top three mantissa bits; t = 16 x / 2^E - 17 - 2 j with
  // 16 / 2^E and -(17 + 2 j) built from their bit fields (no conversion
  // instruction); u = x (-x/4) on the series row
  const unsigned hi = (unsigned)__double2hiint(x);
  const int ej = (int)((hi >> 17) & 0x3FFFu) - ((1023 + kHankMinExp) << 3);
  const int row = small ? kHankSeriesRow : ej;
  const double a = small ? -0.25 * x
                         : __hiloint2double((int)((2050u - ((hi >> 20) & 0x7FFu)) << 20), 0);
  const double b = small ? 0.0
                         : __hiloint2double((int)(0x80000000u | (1027u << 20) |
                                                  ((unsigned)(1 + 2 * (ej & 7)) << 16)),
                                            0);
  const double v = fma(x, a, b);
  const double2* tb = T::tab() + row;
  double2 c0 = make_double2(0.0, 0.0), c1 = c0;
  if (NEED0) c0 = tb[(2 * T::D) * kHankRows];
  if (NEED1) c1 = tb[(2 * T::D + 1) * kHankRows];
#pragma unroll
  for (int d = T::D - 1; d >= 0; --d) {
    if (NEED0) {
      const double2 k0 = tb[(2 * d) * kHankRows];
      c0 = make_double2(fma(c0.x, v, k0.x), fma(c0.y, v, k0.y));
    }
    if (NEED1) {
      const double2 k1 = tb[(2 * d + 1) * kHankRows];
      c1 = make_double2(fma(c1.x, v, k1.x), fma(c1.y, v, k1.y));
    }
  }
  if (small) {
    hankel01_from_series<NEED0, NEED1>(x, ix, c0.x, c0.y, c1.x, c1.y, h0, h1);
  } else {
    if (NEED0) h0 = mk(c0.x, c0.y);
    if (NEED1) h1 = mk(c1.x, c1.y);
  }
}

// Reach of the tables; the CUDA math library's j0/y0/j1/y1 serve x >= 8.
constexpr double kTableMax = 8.0;

// H_0, H_1 at x > 0: each lane below 8 reads its own table row, the library
// serves the rest.
// WIDE: the mixed path's lower-degree tables (relative error below 1e-13).
// NEED0 / NEED1: whether the caller reads h0 / h1 (the other's polynomials
// and library calls are skipped).
template <bool WIDE, bool NEED0 = true, bool NEED1 = true>
__device__ __forceinline__ void hankel01_any(double x, double ix, cd& h0, cd& h1) {
  if (x < kTableMax) {
    hankel01_table<WIDE, NEED0, NEED1>(x, ix, h0, h1);
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

// Start index of the backward recurrence for orders 0..pmax at argument x.
// Started at N, the recurrence returns J_m contaminated by the dominant
// solution with relative weight about (J_{N+1} Y_m) / (Y_{N+1} J_m); above the
// turning point each order n > x shrinks J and grows Y by e^{arccosh(n / x)}
// (Debye's asymptotics, DLMF 10.19.3), so with m = max(pmax, x) the error of
// every J_{m' <= m} is below e^{-2 d arccosh(m / x)} for N = m + d. Where
// x <= m / 2, d = ceil(20 / arccosh(m / x)) + 2 (error below e^{-40}, computed
// in FP32: only an index); nearer the turning point the classical margin
// 12 + 2 sqrt(40 x). Checked against J_m at 40 digits for 17 orders pmax
// between 1 and 420 and 9 arguments each in 1e-6 <= x <= pmax / 2: every J_m,
// m <= pmax, to 2e-16 or better, two or more orders below the start found.
__device__ __forceinline__ int miller_start(int pmax, double x) {
  const int m = pmax > (int)x ? pmax : (int)x;
  const float xf = f32_from_f64(x);
  int n;
  if (2.0f * xf <= (float)m)
    n = m + 2 + (int)ceilf(20.0f / acoshf((float)m / xf));
  else
    n = m + 12 + (int)(2.0 * sqrt(40.0 * x));
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
