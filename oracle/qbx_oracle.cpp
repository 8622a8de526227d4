// Plain FP64 CPU oracle for Global QBX of 2D Helmholtz layer potentials
// (Rachh, Kloeckner, O'Neil, "Fast algorithms for Quadrature by Expansion I:
// Globally valid expansions").
//
// TEST INFRASTRUCTURE ONLY. Only the test suite, the smoke check and the
// benchmark's CPU-baseline leg may load this library. It shares no code with
// the CUDA path: every quantity below is computed from its plain definition,
// with no tree and no translation operator.
//
// Special functions: every J_l / Y_l value is one call of the C++17 library
// routines std::cyl_bessel_j / std::cyl_neumann at that order (negative orders
// by the reflection Z_{-l} = (-1)^l Z_l). H_l = J_l + i Y_l is the Hankel
// function of the first kind. For the full-size workloads the Hankel tables of
// the QBX coefficients may instead come from H_0, H_1 and the upward
// recurrence (oracle_set_hankel_recurrence; off by default).
//
// Conventions (all from Sec. 1 and Sec. 2.1 of the paper):
//   G(x,y) = (i/4) H_0(k|x-y|)                       Eq. (helmholtz-ker)
//   S[s](x) = int G(x,y) s(y) ds(y)                   Eq. (slp)
//   D[s](x) = int dG/dn_y(x,y) s(y) ds(y), n outward  Eq. (dlp)
//   u(x) = sum_l alpha_l J_l(k rho) e^{-i l theta}    Eq. (jexp), (phiapprox)
//   alpha_l(c) = (i/4) int H_l(k|y-c|) e^{i l theta'} s(y) ds(y)
//                                                     Eq. (graf-coefficient)
// where (rho, theta) and (rho', theta') are polar coordinates of x-c and y-c.
// Complex arrays are interleaved (re, im) doubles.

#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdint>
#include <vector>
#include <limits>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef std::complex<double> cplx;
static const cplx I(0.0, 1.0);

// J_l(x) for integer l (any sign), x >= 0: one library call.
static double bessel_j(int l, double x) {
  int m = l < 0 ? -l : l;
  double v = std::cyl_bessel_j((double)m, x);
  return (l < 0 && (m & 1)) ? -v : v;
}

// H_l(x) = J_l(x) + i Y_l(x) for integer l (any sign), x > 0.
static cplx hankel1(int l, double x) {
  int m = l < 0 ? -l : l;
  double j = std::cyl_bessel_j((double)m, x);
  double y = std::cyl_neumann((double)m, x);
  cplx h(j, y);
  return (l < 0 && (m & 1)) ? -h : h;
}

// How hankel_table() fills orders m >= 2 (oracle_set_hankel_recurrence):
//  0 (default): one library call pair per order;
//  1: H_0 and H_1 from the library, then the upward three-term recurrence
//     H_{m+1}(x) = (2m/x) H_m(x) - H_{m-1}(x) (DLMF 10.6.1). |H_m| grows with m,
//     so the recurrence keeps every H_m to a few ulps of |H_m|; it is the
//     affordable route for the full-size workloads (2^20 sources per centre),
//     and it is checked against the per-order calls and mpmath by the pins.
static int g_hankel_recurrence = 0;

// H_m(x) for m = 0..M into h[0..M]; the value at a negative order follows by
// reflection, see hankel_from().
static void hankel_table(int M, double x, cplx* h) {
  if (!g_hankel_recurrence) {
    for (int m = 0; m <= M; ++m) h[m] = hankel1(m, x);
    return;
  }
  h[0] = hankel1(0, x);
  if (M >= 1) h[1] = hankel1(1, x);
  for (int m = 1; m < M; ++m) h[m + 1] = (2.0 * m / x) * h[m] - h[m - 1];
}
static inline cplx hankel_from(const cplx* h, int l) {
  int m = l < 0 ? -l : l;
  return (l < 0 && (m & 1)) ? -h[m] : h[m];
}

// n . grad_y [ H_l(k|y-c|) e^{i l arg(y-c)} ] at y, written out in polar
// coordinates about c: e^{i l th} [ k H_l'(k r) (n . rhat) + (i l / r) H_l(k r) (n . thhat) ]
// with H_l' = (H_{l-1} - H_{l+1}) / 2 (the derivative of Eq. (graf-coefficient)'s
// kernel along the source normal, as needed for the double layer of Eq. (dlp)).
// h holds H_m(k r) for m = 0..|l|+1 (hankel_table).
static cplx dn_hankel_wave(int l, const cplx* h, double k, double dx, double dy, double nx,
                           double ny) {
  double r = std::sqrt(dx * dx + dy * dy);
  double th = std::atan2(dy, dx);
  double c = std::cos(th), s = std::sin(th);
  double n_rhat = nx * c + ny * s;
  double n_thhat = -nx * s + ny * c;
  cplx hl = hankel_from(h, l);
  cplx hp = 0.5 * (hankel_from(h, l - 1) - hankel_from(h, l + 1));
  cplx e = std::polar(1.0, l * th);
  return e * (k * hp * n_rhat + (I * (double)l / r) * hl * n_thhat);
}

// The sums over sources below are split into fixed blocks of kBlock sources;
// each block is summed in source order and the block sums are added in block
// order. The split depends only on the number of sources, so results do not
// depend on the thread count, and a few centres or targets still keep every
// core busy.
static const int64_t kBlock = 2048;
// Upper bound on the partial sums held at once (complex values).
static const int64_t kPartialCap = (int64_t)1 << 22;

static inline cplx load_c(const double* a, int64_t i) { return cplx(a[2 * i], a[2 * i + 1]); }

extern "C" {

int oracle_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void oracle_set_num_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

void oracle_set_hankel_recurrence(int on) { g_hankel_recurrence = on ? 1 : 0; }
int oracle_hankel_recurrence(void) { return g_hankel_recurrence; }

// H_m(x), m = 0..M, for an array of x as hankel_table() forms them under the
// current method: h_out [n][M+1] complex (pins only).
void oracle_hankel_table(int M, int64_t n, const double* x, double* h_out) {
  std::vector<cplx> h(M + 1);
  for (int64_t i = 0; i < n; ++i) {
    hankel_table(M, x[i], h.data());
    for (int m = 0; m <= M; ++m) {
      h_out[2 * (i * (M + 1) + m)] = h[m].real();
      h_out[2 * (i * (M + 1) + m) + 1] = h[m].imag();
    }
  }
}

// Library values of J_l(x) and H_l(x) at one order for an array of x (pins only).
void oracle_bessel(int l, int64_t n, const double* x, double* j_out, double* h_out) {
  for (int64_t i = 0; i < n; ++i) {
    if (j_out) j_out[i] = bessel_j(l, x[i]);
    if (h_out) {
      cplx h = hankel1(l, x[i]);
      h_out[2 * i] = h.real();
      h_out[2 * i + 1] = h.imag();
    }
  }
}

// Expansion centres c = s + side (h_k / 2) n of Sec. 2.2 (one per density node
// and requested side; side +1 is the exterior side of an outward normal).
// Centre index convention: exterior centre of node j is j; when both sides are
// requested the interior centre of node j is n + j.
void oracle_centres(int64_t n, const double* node_xy, const double* normal_xy,
                    const int64_t* panel_of_node, const double* panel_h, int sides,
                    double* centre_xy, double* centre_radius) {
  for (int64_t j = 0; j < n; ++j) {
    double h = panel_h[panel_of_node[j]];
    for (int s = 0; s < sides; ++s) {
      double sgn = s == 0 ? 1.0 : -1.0;
      int64_t c = j + s * n;
      centre_xy[2 * c] = node_xy[2 * j] + sgn * 0.5 * h * normal_xy[2 * j];
      centre_xy[2 * c + 1] = node_xy[2 * j + 1] + sgn * 0.5 * h * normal_xy[2 * j + 1];
      centre_radius[c] = 0.5 * h;
    }
  }
}

// Global QBX coefficients alpha_{c,l}, l = -p..p, over ALL sources, the
// discrete sum of Eq. (localexpcoeffs) (Sec. 7) applied to the combined
// density  cS * S[sigma_S] + cD * D[sigma_D]:
//   alpha_l(c) = (i/4) sum_j w_j [ cS sS_j H_l(k|s_j-c|) e^{i l th_j}
//                                 + cD sD_j n_j . grad_s(H_l(k|s-c|) e^{i l th(s-c)})|s_j ]
// sigma_S / sigma_D may be NULL (that layer is absent).
// alpha_out: [n_ctr][2p+1] complex, l = -p..p in order.
void oracle_qbx_coefficients(int64_t n_src, const double* src_xy, const double* src_normal,
                             const double* weight, const double* sigma_S, const double* sigma_D,
                             double cS_re, double cS_im, double cD_re, double cD_im, double k,
                             int64_t n_ctr, const double* ctr_xy, int p, double* alpha_out) {
  const cplx cS(cS_re, cS_im), cD(cD_re, cD_im);
  const int P = 2 * p + 1;
  const int64_t nb = n_src > 0 ? (n_src + kBlock - 1) / kBlock : 0;
  const int64_t group = std::max<int64_t>(1, kPartialCap / std::max<int64_t>(1, nb * P));
  for (int64_t c0 = 0; c0 < n_ctr; c0 += group) {
    const int64_t c1 = std::min(n_ctr, c0 + group);
    std::vector<cplx> part((size_t)((c1 - c0) * nb * P), cplx(0.0, 0.0));
#pragma omp parallel for collapse(2) schedule(dynamic, 1)
    for (int64_t c = c0; c < c1; ++c) {
      for (int64_t blk = 0; blk < nb; ++blk) {
        cplx* acc = part.data() + ((c - c0) * nb + blk) * P;
        std::vector<cplx> h(p + 2);
        const int64_t j1 = std::min(n_src, (blk + 1) * kBlock);
        for (int64_t j = blk * kBlock; j < j1; ++j) {
          double dx = src_xy[2 * j] - ctr_xy[2 * c];
          double dy = src_xy[2 * j + 1] - ctr_xy[2 * c + 1];
          double r = std::sqrt(dx * dx + dy * dy);
          double th = std::atan2(dy, dx);
          hankel_table(sigma_D ? p + 1 : p, k * r, h.data());
          for (int l = -p; l <= p; ++l) {
            cplx term(0.0, 0.0);
            if (sigma_S)
              term += cS * load_c(sigma_S, j) * hankel_from(h.data(), l) * std::polar(1.0, l * th);
            if (sigma_D)
              term += cD * load_c(sigma_D, j) *
                      dn_hankel_wave(l, h.data(), k, dx, dy, src_normal[2 * j],
                                     src_normal[2 * j + 1]);
            acc[l + p] += weight[j] * term;
          }
        }
      }
    }
    for (int64_t c = c0; c < c1; ++c) {
      for (int l = 0; l < P; ++l) {
        cplx sum(0.0, 0.0);
        for (int64_t blk = 0; blk < nb; ++blk) sum += part[((c - c0) * nb + blk) * P + l];
        cplx a = 0.25 * I * sum;
        alpha_out[2 * (c * P + l)] = a.real();
        alpha_out[2 * (c * P + l) + 1] = a.imag();
      }
    }
  }
}

// Smooth Gauss quadrature of the layer potential at targets, Eq. (gauss-layerpot)
// (Sec. 3.2) / Eq. (QBXFMMpot) (Sec. 7), for the combined density:
//   u(t) = (i/4) sum_j w_j [ cS sS_j H_0(k r) + cD sD_j k H_1(k r) n_j.(t - s_j)/r ],
// r = |t - s_j|; the second term is dG/dn_y = (i/4) k H_1(kr) n_y.(x-y)/r.
void oracle_direct_potential(int64_t n_src, const double* src_xy, const double* src_normal,
                             const double* weight, const double* sigma_S, const double* sigma_D,
                             double cS_re, double cS_im, double cD_re, double cD_im, double k,
                             int64_t n_tgt, const double* tgt_xy, double* u_out) {
  const cplx cS(cS_re, cS_im), cD(cD_re, cD_im);
  const int64_t nb = n_src > 0 ? (n_src + kBlock - 1) / kBlock : 0;
  const int64_t group = std::max<int64_t>(1, kPartialCap / std::max<int64_t>(1, nb));
  for (int64_t t0 = 0; t0 < n_tgt; t0 += group) {
    const int64_t t1 = std::min(n_tgt, t0 + group);
    std::vector<cplx> part((size_t)((t1 - t0) * nb), cplx(0.0, 0.0));
#pragma omp parallel for collapse(2) schedule(dynamic, 1)
    for (int64_t t = t0; t < t1; ++t) {
      for (int64_t blk = 0; blk < nb; ++blk) {
        cplx acc(0.0, 0.0);
        const int64_t j1 = std::min(n_src, (blk + 1) * kBlock);
        for (int64_t j = blk * kBlock; j < j1; ++j) {
          double dx = tgt_xy[2 * t] - src_xy[2 * j];
          double dy = tgt_xy[2 * t + 1] - src_xy[2 * j + 1];
          double r = std::sqrt(dx * dx + dy * dy);
          cplx term(0.0, 0.0);
          if (sigma_S) term += cS * load_c(sigma_S, j) * hankel1(0, k * r);
          if (sigma_D) {
            double ndotd = src_normal[2 * j] * dx + src_normal[2 * j + 1] * dy;
            term += cD * load_c(sigma_D, j) * k * hankel1(1, k * r) * (ndotd / r);
          }
          acc += weight[j] * term;
        }
        part[(t - t0) * nb + blk] = acc;
      }
    }
    for (int64_t t = t0; t < t1; ++t) {
      cplx acc(0.0, 0.0);
      for (int64_t blk = 0; blk < nb; ++blk) acc += part[(t - t0) * nb + blk];
      acc *= 0.25 * I;
      u_out[2 * t] = acc.real();
      u_out[2 * t + 1] = acc.imag();
    }
  }
}

// Truncated QBX evaluation of Eq. (phiapprox): u(t) = sum_{|l|<=p} alpha_l J_l(k rho) e^{-i l theta},
// (rho, theta) the polar coordinates of t - c for the centre c = centre_of_target[t].
// Targets with centre_of_target[t] < 0 are skipped (u_out untouched).
void oracle_qbx_evaluate(int64_t n_tgt, const double* tgt_xy, const int32_t* centre_of_target,
                         const double* ctr_xy, const double* alpha, int p, double k,
                         double* u_out) {
  const int P = 2 * p + 1;
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t t = 0; t < n_tgt; ++t) {
    int64_t c = centre_of_target[t];
    if (c < 0) continue;
    double dx = tgt_xy[2 * t] - ctr_xy[2 * c];
    double dy = tgt_xy[2 * t + 1] - ctr_xy[2 * c + 1];
    double rho = std::sqrt(dx * dx + dy * dy);
    double th = std::atan2(dy, dx);
    cplx acc(0.0, 0.0);
    for (int l = -p; l <= p; ++l)
      acc += load_c(alpha, c * P + (l + p)) * bessel_j(l, k * rho) * std::polar(1.0, -l * th);
    u_out[2 * t] = acc.real();
    u_out[2 * t + 1] = acc.imag();
  }
}

// Brute-force target association of Sec. 6.1 ("Associate volume/surface targets
// with QBX expansions"), over all centres instead of through a tree:
//  * a target that lies on the surface (on_surface_node[t] = j >= 0) takes the
//    centre of its own node on the requested side (side preference, Sec. 6.1);
//  * otherwise the nearest centre c with |t-c| <= (1+eps_assoc) r_c, ties to the
//    smaller index; squared distances are compared, (dx*dx + dy*dy) against
//    ((1+eps) r)^2, without fused multiply-add;
//  * if there is none and t is in Gamma_near, approximated (as the paper allows)
//    by min_j |t - s_j| <= h_{panel(j)}/4 over density nodes, association fails;
//  * else the target is evaluated by direct quadrature (-1).
// centre_of_target receives the centre index, -1 (direct) or -2 (failure).
// Returns the number of failures.
int64_t oracle_associate(int64_t n_tgt, const double* tgt_xy, const int64_t* on_surface_node,
                         const int8_t* on_surface_side, int64_t n_nodes, const double* node_xy,
                         const int64_t* panel_of_node, const double* panel_h, int64_t n_ctr,
                         const double* ctr_xy, const double* ctr_radius, double eps_assoc,
                         int32_t* centre_of_target) {
  int64_t fails = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : fails)
  for (int64_t t = 0; t < n_tgt; ++t) {
    if (on_surface_node && on_surface_node[t] >= 0) {
      int64_t j = on_surface_node[t];
      int side = on_surface_side ? on_surface_side[t] : 1;
      centre_of_target[t] = (int32_t)(side >= 0 ? j : n_nodes + j);
      continue;
    }
    const double tx = tgt_xy[2 * t], ty = tgt_xy[2 * t + 1];
    int64_t best = -1;
    double best_d2 = std::numeric_limits<double>::infinity();
    for (int64_t c = 0; c < n_ctr; ++c) {
      volatile double dx = tx - ctr_xy[2 * c];
      volatile double dy = ty - ctr_xy[2 * c + 1];
      volatile double dx2 = dx * dx;
      volatile double dy2 = dy * dy;
      double d2 = dx2 + dy2;
      volatile double lim = (1.0 + eps_assoc) * ctr_radius[c];
      double lim2 = lim * lim;
      if (d2 <= lim2 && d2 < best_d2) {
        best = c;
        best_d2 = d2;
      }
    }
    if (best >= 0) {
      centre_of_target[t] = (int32_t)best;
      continue;
    }
    bool near = false;
    for (int64_t j = 0; j < n_nodes && !near; ++j) {
      volatile double dx = tx - node_xy[2 * j];
      volatile double dy = ty - node_xy[2 * j + 1];
      volatile double dx2 = dx * dx;
      volatile double dy2 = dy * dy;
      double d2 = dx2 + dy2;
      volatile double q = 0.25 * panel_h[panel_of_node[j]];
      double q2 = q * q;
      if (d2 <= q2) near = true;
    }
    if (near) {
      centre_of_target[t] = -2;
      fails += 1;
    } else {
      centre_of_target[t] = -1;
    }
  }
  return fails;
}

}  // extern "C"
