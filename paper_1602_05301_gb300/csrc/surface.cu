// The source discretisation made by the library (Sec. 2.2 and Sec. 3.2): the
// same panels as the density grid, each with q_src Gauss-Legendre nodes, and
// the density values there obtained from the q density nodes of the panel by
// polynomial interpolation. Also the node counts of Table 1.
//
// Each panel of the density grid is a set of q Gauss-Legendre nodes of some
// smooth parametrisation; in the panel's reference variable u in [-1, 1] the
// coordinates x(u), y(u) are interpolated by the degree q-1 polynomial through
// the nodes, so the source nodes, their tangents (the derivative of that
// polynomial) and their weights w_j^src |gamma'(u_j)| follow from the density
// grid alone. The outward normal is the rotated unit tangent, with the sign of
// the interpolated caller normals.
#include <algorithm>
#include <cmath>
#include <vector>

#include "qbx_internal.h"

namespace {

inline unsigned nblk(int64_t n, int b) { return (unsigned)std::max<int64_t>(1, (n + b - 1) / b); }

// P_n(z) and P_n'(z) by the three-term recurrence.
void legendre(int n, double z, double& pn, double& dpn) {
  double p0 = 1.0, p1 = z;
  for (int k = 2; k <= n; ++k) {
    const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
    p0 = p1;
    p1 = p2;
  }
  pn = n == 0 ? 1.0 : p1;
  dpn = n == 0 ? 0.0 : n * (z * p1 - p0) / (z * z - 1.0);
}

// Gauss-Legendre nodes (ascending) and weights on [-1, 1]: Newton's method on
// P_n from the usual cosine starting values, w = 2 / ((1 - x^2) P_n'(x)^2).
void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  for (int i = 0; i < n; ++i) {
    double z = std::cos(M_PI * (i + 0.75) / (n + 0.5)), pn, dp;
    for (int it = 0; it < 100; ++it) {
      legendre(n, z, pn, dp);
      const double dz = pn / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    legendre(n, z, pn, dp);
    x[n - 1 - i] = z;
    w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

// L[j][i] = l_i(u_j) and D[j][i] = l_i'(u_j) for the Lagrange basis l_i of the
// nodes x (q of them) at the points u (m of them); the derivative is the
// product rule written without divisions by (u - x_r), so coinciding nodes
// are harmless.
void lagrange_matrices(const std::vector<double>& x, const std::vector<double>& u,
                       std::vector<double>& L, std::vector<double>& D) {
  const int q = (int)x.size(), m = (int)u.size();
  L.assign((size_t)m * q, 0.0);
  D.assign((size_t)m * q, 0.0);
  for (int j = 0; j < m; ++j)
    for (int i = 0; i < q; ++i) {
      double li = 1.0;
      for (int r = 0; r < q; ++r)
        if (r != i) li *= (u[j] - x[r]) / (x[i] - x[r]);
      double di = 0.0;
      for (int s = 0; s < q; ++s) {
        if (s == i) continue;
        double t = 1.0 / (x[i] - x[s]);
        for (int r = 0; r < q; ++r)
          if (r != i && r != s) t *= (u[j] - x[r]) / (x[i] - x[r]);
        di += t;
      }
      L[(size_t)j * q + i] = li;
      D[(size_t)j * q + i] = di;
    }
}

// One thread per source node: position, unit outward normal and weight from
// the q density nodes of its panel.
__global__ void upsample_geometry_kernel(int64_t n_panels, int q, int qs,
                                         const double* __restrict__ L,
                                         const double* __restrict__ D,
                                         const double* __restrict__ ws,
                                         const double* __restrict__ node_xy,
                                         const double* __restrict__ node_nrm,
                                         double* __restrict__ src_xy, double* __restrict__ src_nrm,
                                         double* __restrict__ src_w) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n_panels * qs) return;
  const int64_t k = i / qs;
  const int j = (int)(i % qs);
  const double* Lj = L + (size_t)j * q;
  const double* Dj = D + (size_t)j * q;
  const double* xy = node_xy + 2 * k * q;
  const double* nn = node_nrm + 2 * k * q;
  double x = 0.0, y = 0.0, dx = 0.0, dy = 0.0, nx = 0.0, ny = 0.0;
  for (int r = 0; r < q; ++r) {
    x = fma(Lj[r], xy[2 * r], x);
    y = fma(Lj[r], xy[2 * r + 1], y);
    dx = fma(Dj[r], xy[2 * r], dx);
    dy = fma(Dj[r], xy[2 * r + 1], dy);
    nx = fma(Lj[r], nn[2 * r], nx);
    ny = fma(Lj[r], nn[2 * r + 1], ny);
  }
  const double sp = hypot(dx, dy);
  double ox = dy / sp, oy = -dx / sp;
  if (ox * nx + oy * ny < 0.0) ox = -ox, oy = -oy;
  src_xy[2 * i] = x;
  src_xy[2 * i + 1] = y;
  src_nrm[2 * i] = ox;
  src_nrm[2 * i + 1] = oy;
  src_w[i] = ws[j] * sp;
}

// Strengths on the library-made source grid: the densities (given on the
// density grid) interpolated to source node i of panel k, times the weight and
// the kernel's factor i/4 (as for a caller's grid):
// q_i = (i/4) w_i cS sigma_S(s_i), d_i = (i/4) w_i cD sigma_D(s_i).
__global__ void strengths_upsampled_kernel(int64_t n_panels, int q, int qs,
                                           const double* __restrict__ L,
                                           const double* __restrict__ w, cd cS,
                                           const cd* __restrict__ sS, cd cD,
                                           const cd* __restrict__ sD, cd* __restrict__ qo,
                                           cd* __restrict__ dout) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n_panels * qs) return;
  const int64_t k = i / qs;
  const int j = (int)(i % qs);
  const double* Lj = L + (size_t)j * q;
  cd a = mk(0.0, 0.0), b = mk(0.0, 0.0);
  for (int r = 0; r < q; ++r) {
    if (sS) a = mk(fma(Lj[r], sS[k * q + r].x, a.x), fma(Lj[r], sS[k * q + r].y, a.y));
    if (sD) b = mk(fma(Lj[r], sD[k * q + r].x, b.x), fma(Lj[r], sD[k * q + r].y, b.y));
  }
  const cd i4 = mk(0.0, 0.25 * w[i]);
  qo[i] = sS ? cmul(i4, cmul(cS, a)) : mk(0.0, 0.0);
  dout[i] = sD ? cmul(i4, cmul(cD, b)) : mk(0.0, 0.0);
}

}  // namespace

void gl_nodes(int n, std::vector<double>& x, std::vector<double>& w) { gauss_legendre(n, x, w); }

qbx_status upsample_geometry(qbx_handle* h) {
  const int q = h->q, qs = h->q_src;
  std::vector<double> xq, wq, xs, ws, L, D;
  gauss_legendre(q, xq, wq);
  gauss_legendre(qs, xs, ws);
  lagrange_matrices(xq, xs, L, D);
  DevBuf<double> dD, dw;
  QBX_CUDA_TRY(h->up_L.alloc(L.size()));
  QBX_CUDA_TRY(dD.alloc(D.size()));
  QBX_CUDA_TRY(dw.alloc(ws.size()));
  QBX_CUDA_TRY(cudaMemcpy(h->up_L.ptr, L.data(), L.size() * 8, cudaMemcpyHostToDevice));
  QBX_CUDA_TRY(cudaMemcpy(dD.ptr, D.data(), D.size() * 8, cudaMemcpyHostToDevice));
  QBX_CUDA_TRY(cudaMemcpy(dw.ptr, ws.data(), ws.size() * 8, cudaMemcpyHostToDevice));
  QBX_CUDA_TRY(h->src_xy.alloc(2 * h->n_src));
  QBX_CUDA_TRY(h->src_nrm.alloc(2 * h->n_src));
  QBX_CUDA_TRY(h->src_w.alloc(h->n_src));
  upsample_geometry_kernel<<<nblk(h->n_src, 128), 128>>>(h->n_panels, q, qs, h->up_L.ptr, dD.ptr,
                                                         dw.ptr, h->node_xy.ptr, h->node_nrm.ptr,
                                                         h->src_xy.ptr, h->src_nrm.ptr,
                                                         h->src_w.ptr);
  QBX_CUDA_TRY(cudaGetLastError());
  QBX_CUDA_TRY(cudaDeviceSynchronize());  // before the temporaries are freed
  return QBX_OK;
}

qbx_status launch_strengths_upsampled(qbx_handle* h, cd cS, const cd* sigS, cd cD,
                                      const cd* sigD, cudaStream_t s) {
  if (h->n_src == 0) return QBX_OK;
  strengths_upsampled_kernel<<<nblk(h->n_src, 256), 256, 0, s>>>(
      h->n_panels, h->q, h->q_src, h->up_L.ptr, h->src_w.ptr, cS, sigS, cD, sigD, h->q_str.ptr,
      h->d_str.ptr);
  QBX_CUDA_TRY(cudaGetLastError());
  h->launches += 1;
  return QBX_OK;
}

extern "C" qbx_status qbx_get_source_grid(const qbx_handle* h, double* src_xy,
                                          double* src_normal_xy, double* src_weight) {
  if (!h) {
    set_error("qbx_get_source_grid: NULL handle");
    return QBX_ERR_ARG;
  }
  const int64_t n = h->n_src;
  if (src_xy) QBX_CUDA_TRY(cudaMemcpy(src_xy, h->src_xy.ptr, 2 * n * 8, cudaMemcpyDefault));
  if (src_normal_xy)
    QBX_CUDA_TRY(cudaMemcpy(src_normal_xy, h->src_nrm.ptr, 2 * n * 8, cudaMemcpyDefault));
  if (src_weight) QBX_CUDA_TRY(cudaMemcpy(src_weight, h->src_w.ptr, n * 8, cudaMemcpyDefault));
  return QBX_OK;
}

// Table 1 (Sec. 3.2): source nodes per panel for q density nodes and a
// requested precision eps. Rows q = 2, 4, 8, 16; columns eps = 1e-3, 1e-6,
// 1e-9, 1e-12.
extern "C" int32_t qbx_table1_q_src(int32_t q, double eps) {
  static const int rows[4] = {2, 4, 8, 16};
  static const int tab[4][4] = {{8, 16, 24, 32}, {12, 24, 32, 40}, {16, 32, 40, 48},
                                {32, 48, 64, 64}};
  static const double cols[4] = {1e-3, 1e-6, 1e-9, 1e-12};
  if (q < 1 || q > 16 || !(eps > 0.0) || eps < 1e-12 * (1.0 - 1e-9)) return -1;
  int r = 0;
  while (rows[r] < q) ++r;             // the next tabulated density order
  int c = 0;
  while (cols[c] > eps * (1.0 + 1e-9)) ++c;   // the first column at least as strict
  return tab[r][c];
}
