// Level-dependent FMM expansion orders (Sec. 7.1, "Maintaining Expansion
// Accuracy"). For a box of half-side R the outgoing expansion is truncated at
// the smallest order p for which
//     max_{rho >= 3R, rho_j <= sqrt2 R, |n| > p} |H_n(k rho) J_n(k rho_j)| <= eps,
// and the box order used by the QBX translations is that p plus p_add.
// |H_n| decreases in its argument, so its maximum over rho >= 3R is at
// rho = 3R. For n above y = sqrt2 k R, J_n increases on [0, y] (its first
// maximum lies beyond n), so the maximum over rho_j is at rho_j = sqrt2 R;
// below y the bound 1 is used, which only matters for orders that the
// criterion rejects anyway.
//
// eps is not an input of the method: it is read off the order p_fmm, as the
// bound that p_fmm gives in the low-frequency regime, eps = max_{n > p_fmm} of
// the bound at k R = min(k R_finest, 1). The finest level then keeps p_fmm
// unless its boxes are themselves above k R = 1, and every coarser level gets
// the order that gives the same bound, which grows with k R once boxes span
// wavelengths.
//
// Host code only (plan construction): log-magnitudes of H_n and J_n from
// recurrences with rescaling, the starting values from the C library.
#include <algorithm>
#include <cmath>
#include <vector>

#include "qbx_internal.h"
#include "p_add_table.h"

namespace {

constexpr double kBig = 1e250;
const double kLogBig = std::log(kBig);

// log|H_n(a)|, n = 0..N, by the upward recurrence H_{n+1} = (2n/a) H_n - H_{n-1}
// (DLMF 10.6.1), which is stable for the Hankel function as a whole.
void log_abs_hankel(double a, int N, std::vector<double>& out) {
  out.assign(N + 1, 0.0);
  double hr0 = j0(a), hi0 = y0(a), hr1 = j1(a), hi1 = y1(a);
  double lsc = 0.0;  // log of the factor the stored pair has been divided by
  out[0] = 0.5 * std::log(hr0 * hr0 + hi0 * hi0);
  if (N >= 1) out[1] = 0.5 * std::log(hr1 * hr1 + hi1 * hi1);
  for (int n = 1; n < N; ++n) {
    const double f = 2.0 * n / a;
    const double hr2 = f * hr1 - hr0, hi2 = f * hi1 - hi0;
    hr0 = hr1; hi0 = hi1; hr1 = hr2; hi1 = hi2;
    const double m = std::fabs(hr1) + std::fabs(hi1);
    if (m > kBig) {
      hr0 /= kBig; hi0 /= kBig; hr1 /= kBig; hi1 /= kBig;
      lsc += kLogBig;
    }
    out[n + 1] = std::log(std::hypot(hr1, hi1)) + lsc;
  }
}

// log J_n(b), n = 0..N, b > 0, by Miller's backward recurrence normalised with
// J_0 + 2 sum_k J_2k = 1 (DLMF 10.12.4); values at orders where J_n(b) = 0
// come out as -inf. Tiny b uses the leading term (b/2)^n / n!.
void log_bessel_j(double b, int N, std::vector<double>& out) {
  out.assign(N + 1, 0.0);
  if (b < 1e-8) {
    for (int n = 0; n <= N; ++n) out[n] = n * std::log(0.5 * b) - std::lgamma(n + 1.0);
    return;
  }
  const int start = std::max(N + 20, (int)(b + 40.0 + 10.0 * std::cbrt(b)));
  std::vector<double> f(start + 2, 0.0), lsc_at(start + 2, 0.0);
  double fn1 = 0.0, fn = 1e-300, sum = 0.0, lsc = 0.0;  // lsc: log of the scale applied so far
  f[start] = fn;
  lsc_at[start] = 0.0;
  for (int n = start; n >= 1; --n) {
    const double fm = (2.0 * n / b) * fn - fn1;
    if ((n & 1) == 0) sum += fn;
    fn1 = fn;
    fn = fm;
    if (std::fabs(fn) > kBig) {
      fn /= kBig; fn1 /= kBig; sum /= kBig;
      lsc += kLogBig;
    }
    f[n - 1] = fn;
    lsc_at[n - 1] = lsc;
  }
  // true f_n = stored f_n * exp(lsc_at[n]); true norm = (f_0 + 2 sum) * exp(lsc)
  const double lnorm = std::log(std::fabs(fn + 2.0 * sum)) + lsc;
  for (int n = 0; n <= N; ++n)
    out[n] = (f[n] == 0.0 ? -INFINITY : std::log(std::fabs(f[n])) + lsc_at[n]) - lnorm;
}

// log of the bound for orders n = 0..N at half-side R: log|H_n(3kR)| + log max_{y<=sqrt2 kR}|J_n(y)|.
void log_bound(double kR, int N, std::vector<double>& out) {
  const double a = 3.0 * kR, b = std::sqrt(2.0) * kR;
  std::vector<double> lh, lj;
  log_abs_hankel(a, N, lh);
  log_bessel_j(b, N, lj);
  out.assign(N + 1, 0.0);
  for (int n = 0; n <= N; ++n) out[n] = lh[n] + ((double)n > b ? lj[n] : 0.0);
}

}  // namespace

// Smallest p >= p_min with max_{n > p} bound_n(kR) <= exp(log_eps); -1 if it
// exceeds p_cap. Beyond n = sqrt2 kR the bound decreases with n, so a window of
// orders above the candidate suffices.
int fmm_order_for(double kR, double log_eps, int p_min, int p_cap) {
  int N = std::max(p_min, (int)(std::sqrt(2.0) * kR)) + 64 + (int)(16.0 * std::cbrt(kR + 1.0));
  for (;;) {
    std::vector<double> lb;
    log_bound(kR, N, lb);
    // suffix maxima over (p, N]
    std::vector<double> sm(N + 2, -INFINITY);
    for (int n = N; n >= 0; --n) sm[n] = std::max(sm[n + 1], lb[n]);
    for (int p = p_min; p < N - 16; ++p)
      if (sm[p + 1] <= log_eps) return p > p_cap ? -1 : p;
    if (N > p_cap + 64) return -1;
    N *= 2;
  }
}

// log eps as defined above: the largest bound over orders n > p_fmm at kR_ref.
double fmm_log_eps(double kR_ref, int p_fmm) {
  const int N = p_fmm + 64 + (int)(16.0 * std::cbrt(kR_ref + 1.0)) +
                (int)(std::sqrt(2.0) * kR_ref);
  std::vector<double> lb;
  log_bound(kR_ref, N, lb);
  double m = -INFINITY;
  for (int n = p_fmm + 1; n <= N; ++n) m = std::max(m, lb[n]);
  return m;
}

extern "C" qbx_status qbx_fmm_level_orders(double k, double root_side, int32_t n_levels,
                                           int32_t p_fmm, int32_t p_add, int32_t* pb_out) {
  set_error("%s", "");
  if (!(k > 0.0) || !(root_side > 0.0) || n_levels < 1 || n_levels > 25 || p_fmm < 1 ||
      p_add < 0 || p_fmm + p_add > kMaxBoxOrder || !pb_out) {
    set_error("qbx_fmm_level_orders: bad arguments");
    return QBX_ERR_ARG;
  }
  for (int l = 0; l < n_levels; ++l) pb_out[l] = 0;
  if (n_levels < 3) return QBX_OK;  // no level carries expansions
  const int lf = n_levels - 1;
  const double kR_lf = 0.5 * k * root_side / (double)(1 << lf);
  const double log_eps = fmm_log_eps(std::min(kR_lf, 1.0), p_fmm);
  for (int l = 2; l < n_levels; ++l) {
    const double kR = 0.5 * k * root_side / (double)(1 << l);
    const int p = (l == lf && kR_lf <= 1.0) ? p_fmm
                                            : fmm_order_for(kR, log_eps, p_fmm, kMaxBoxOrder - p_add);
    if (p < 0) {
      set_error("level %d boxes (k*side = %.4g) need an expansion order above %d", l, 2.0 * kR,
                kMaxBoxOrder);
      return QBX_ERR_ARG;
    }
    pb_out[l] = p + p_add;
  }
  return QBX_OK;
}

// p_add for the default plan (p_add < 0 in the tree descriptor): measured
// with this library by the experiment of Sec. 7.1 (calibrate_p_add.py; the
// generated table below). Table 2 of the paper, measured the same way with
// the paper's own point-FMM orders, prints 5, 5, 15, 20 for p = 2, 4, 6, 8.
extern "C" int32_t qbx_default_p_add(int32_t p) {
  if (p < 0) return -1;
  return kPAddCalibrated[p > QBX_MAX_P ? QBX_MAX_P : p];
}
