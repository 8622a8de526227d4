// Entries of the sigma-normalised M2L operator of one (level, offset class),
//     T[n][lo] = sig_lo sig_n (-1)^lo W_{n+lo}(D) s^-|n+lo| (scale factors of
//     the level's power-scaled Hankel table What_m = s^|m| W_m(D)),
// computed in FP64 through logarithms (the table entries reach 1e155, the
// sigma products are tiny): of order one or smaller for every n, lo. Used by
// the FP32 M2L of the mixed path and by the tensor-core M2L of the FP64 path.
#pragma once
#include "qbx_internal.h"

struct M2lNorm {
  const cd* w;       // What_m at w[m], |m| <= 2 pbmax
  const double* sg;  // log sig_j of the level
  double ls;         // log s of the level
  bool used;         // the class is a V-list offset (max(|dx|, |dy|) >= 2)
  __device__ M2lNorm(const cd* t_m2l, const double* scale, const double* lsig, int l, int cls,
                     int pbmax)
      : w(t_m2l + ((size_t)l * 49 + cls) * (4 * pbmax + 1) + 2 * pbmax),
        sg(lsig + (size_t)l * (pbmax + 1)),
        ls(log(scale[l])) {
    const int dx = cls / 7 - 3, dy = cls % 7 - 3;
    used = max(abs(dx), abs(dy)) >= 2;
  }
  __device__ cd entry(int n, int lo) const {
    if (!used) return mk(0.0, 0.0);
    const cd v = w[n + lo];
    const double mag = hypot(v.x, v.y);  // no squares: entries reach 1e155
    if (!(mag > 0.0)) return mk(0.0, 0.0);
    const double lf = sg[abs(lo)] + sg[abs(n)] - abs(n + lo) * ls + log(mag);
    const double f = lf < -700.0 ? 0.0 : exp(lf) / mag;
    const double sgn = (lo & 1) ? -f : f;
    return mk(v.x * sgn, v.y * sgn);
  }
};
