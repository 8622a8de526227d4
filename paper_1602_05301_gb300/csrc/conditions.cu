// Accuracy conditions of the geometry and source refinement (Sec. 3.1-3.3,
// Sec. 4 and Sec. 5 of the paper).
//
// Every panel is described by the Legendre expansion of its coordinates in
// the reference variable u in [-1, 1] (the interpolating polynomial through
// its q Gauss-Legendre nodes; Sec. 5: "the Legendre expansion describing the
// panel's parametrization"). Distances from a point to a panel are distances
// to that curve: the nearest point of the polygon through the nodes and the
// end points, then Newton's method on (x(u) - c) . x'(u) = 0 when the answer
// is close to the threshold being tested.
//
// Area queries (Sec. 4): the paper finds the panels near a centre through
// peer boxes of a quadtree. Here the panels' bounding squares (enlarged by
// h/4, the reach of Condition 3) are the leaves of a bounding-volume tree over
// the panels in Morton order of their centres of mass (a complete binary tree
// in heap order, each node the union of its children's squares); each centre
// walks it with a small stack and visits the panels whose square meets its
// query square. Same result as the paper's queries (every panel that can be
// closer than the threshold is visited), suited to one thread per centre.
//
// Refinement (Sec. 5): a flagged panel is bisected at the parameter u* that
// halves its arclength (Newton's method on the Gauss-Legendre arclength
// integral); the two halves get new Gauss-Legendre nodes, normals and weights
// from the parent's expansion.
#include <cub/cub.cuh>

#include <algorithm>
#include <cmath>
#include <vector>

#include "qbx_internal.h"

namespace {

constexpr int kT = 128;
constexpr int kMaxQ = 32;        // density nodes per panel handled here
constexpr int kStack = 40;       // bounding-volume tree depth bound (2^39 panels)

inline unsigned nblk(int64_t n, int b) { return (unsigned)std::max<int64_t>(1, (n + b - 1) / b); }

// x(u) = sum_n c_n P_n(u) and its first two derivatives (three-term
// recurrences for P_n, P_n' = P_{n-2}' + (2n-1) P_{n-1}, same for P_n'').
struct Curve {
  const double2* c;  // [q] coefficients (x, y)
  int q;
  __device__ void eval(double u, double2& x, double2& d1, double2& d2) const {
    double p0 = 1.0, p1 = u, dp0 = 0.0, dp1 = 1.0, ddp0 = 0.0, ddp1 = 0.0;
    x = make_double2(c[0].x, c[0].y);
    d1 = make_double2(0.0, 0.0);
    d2 = make_double2(0.0, 0.0);
    if (q > 1) {
      x.x += c[1].x * u; x.y += c[1].y * u;
      d1.x += c[1].x; d1.y += c[1].y;
    }
    for (int n = 2; n < q; ++n) {
      const double p2 = ((2.0 * n - 1.0) * u * p1 - (n - 1.0) * p0) / n;
      const double dp2 = dp0 + (2.0 * n - 1.0) * p1;
      const double ddp2 = ddp0 + (2.0 * n - 1.0) * dp1;
      x.x += c[n].x * p2; x.y += c[n].y * p2;
      d1.x += c[n].x * dp2; d1.y += c[n].y * dp2;
      d2.x += c[n].x * ddp2; d2.y += c[n].y * ddp2;
      p0 = p1; p1 = p2; dp0 = dp1; dp1 = dp2; ddp0 = ddp1; ddp1 = ddp2;
    }
  }
  __device__ double2 pos(double u) const {
    double2 x, a, b;
    eval(u, x, a, b);
    return x;
  }
};

__device__ __forceinline__ double seg_dist2(double2 c, double2 a, double2 b) {
  const double ex = b.x - a.x, ey = b.y - a.y, wx = c.x - a.x, wy = c.y - a.y;
  const double L = ex * ex + ey * ey;
  double t = L > 0.0 ? (wx * ex + wy * ey) / L : 0.0;
  t = fmin(1.0, fmax(0.0, t));
  const double dx = wx - t * ex, dy = wy - t * ey;
  return dx * dx + dy * dy;
}

// Distance from c to a panel: the polygon through the end points and the
// nodes (node u values gl), refined by Newton's method on the curve when it
// is within 2% of one of the thresholds t1, t2 (so that comparisons with them
// are decided on the curve itself).
__device__ double panel_distance(const Curve& C, const double2* nodes, const double* gl,
                                 double2 e0, double2 e1, double2 c, double t1, double t2) {
  double best = seg_dist2(c, e0, nodes[0]);
  double ub = 0.5 * (-1.0 + gl[0]);
  for (int j = 0; j + 1 < C.q; ++j) {
    const double d = seg_dist2(c, nodes[j], nodes[j + 1]);
    if (d < best) { best = d; ub = 0.5 * (gl[j] + gl[j + 1]); }
  }
  {
    const double d = seg_dist2(c, nodes[C.q - 1], e1);
    if (d < best) { best = d; ub = 0.5 * (gl[C.q - 1] + 1.0); }
  }
  const double dist = sqrt(best);
  if (fabs(dist - t1) > 0.02 * t1 && fabs(dist - t2) > 0.02 * t2) return dist;
  double u = ub;
  for (int it = 0; it < 12; ++it) {
    double2 x, d1, d2;
    C.eval(u, x, d1, d2);
    const double rx = x.x - c.x, ry = x.y - c.y;
    const double g = rx * d1.x + ry * d1.y;
    const double gp = d1.x * d1.x + d1.y * d1.y + rx * d2.x + ry * d2.y;
    if (!(gp > 0.0)) break;
    const double un = fmin(1.0, fmax(-1.0, u - g / gp));
    if (fabs(un - u) < 1e-15) { u = un; break; }
    u = un;
  }
  const double2 x = C.pos(u);
  return fmin(dist, hypot(x.x - c.x, x.y - c.y));
}

// Legendre coefficients of the panel coordinates and normals:
// c_n = (2n + 1)/2 sum_j w_j P_n(u_j) x_j (A[n][j] holds the factors).
__global__ void legendre_kernel(int64_t n_panels, int q, const double* __restrict__ A,
                                const double* __restrict__ xy, const double* __restrict__ nrm,
                                double2* __restrict__ cx, double2* __restrict__ cn) {
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= n_panels) return;
  for (int n = 0; n < q; ++n) {
    double2 a = make_double2(0.0, 0.0), b = make_double2(0.0, 0.0);
    for (int j = 0; j < q; ++j) {
      const double f = A[n * q + j];
      const int64_t i = k * q + j;
      a.x = fma(f, xy[2 * i], a.x); a.y = fma(f, xy[2 * i + 1], a.y);
      b.x = fma(f, nrm[2 * i], b.x); b.y = fma(f, nrm[2 * i + 1], b.y);
    }
    cx[k * q + n] = a;
    cn[k * q + n] = b;
  }
}

// Per panel: end points, centre of mass, bounding square (of 4q + 1 curve
// points, enlarged by 1% of h for the parts between samples) and that square
// enlarged by h/4 (the reach of Condition 3); Morton key of the centre of mass.
__global__ void panel_box_kernel(int64_t n_panels, int q, const double2* __restrict__ cx,
                                 const double* __restrict__ xy, const double* __restrict__ w,
                                 const double* __restrict__ h, double2* __restrict__ ends,
                                 double4* __restrict__ box, double4 dom,
                                 unsigned long long* __restrict__ key, int* __restrict__ id) {
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= n_panels) return;
  const Curve C{cx + k * q, q};
  double mx = 0.0, my = 0.0, ws = 0.0;
  for (int j = 0; j < q; ++j) {
    const int64_t i = k * q + j;
    mx += w[i] * xy[2 * i];
    my += w[i] * xy[2 * i + 1];
    ws += w[i];
  }
  mx /= ws;
  my /= ws;
  double r = 0.0;
  const int ns = 4 * q;
  for (int s = 0; s <= ns; ++s) {
    const double2 x = C.pos(-1.0 + 2.0 * s / ns);
    r = fmax(r, fmax(fabs(x.x - mx), fabs(x.y - my)));
  }
  r += 0.01 * h[k];
  const double R = r + 0.25 * h[k];
  box[k] = make_double4(mx - R, my - R, mx + R, my + R);
  ends[2 * k] = C.pos(-1.0);
  ends[2 * k + 1] = C.pos(1.0);
  // Morton key (16 bits per axis) of the centre of mass in the domain square
  const double sx = fmin(fmax((mx - dom.x) / (dom.z - dom.x), 0.0), 1.0);
  const double sy = fmin(fmax((my - dom.y) / (dom.w - dom.y), 0.0), 1.0);
  unsigned ix = (unsigned)(sx * 65535.0), iy = (unsigned)(sy * 65535.0);
  unsigned long long m = 0;
  for (int b = 0; b < 16; ++b)
    m |= (unsigned long long)((ix >> b) & 1u) << (2 * b) |
         (unsigned long long)((iy >> b) & 1u) << (2 * b + 1);
  key[k] = m;
  id[k] = (int)k;
}

// Bounding-volume tree in heap order: node 1 is the root, node j has children
// 2j and 2j + 1, the leaves are nodes 2^L + i for the panels in Morton order.
__global__ void bvh_leaves_kernel(int64_t n, int64_t nl, const int* __restrict__ order,
                                  const double4* __restrict__ box, double4* __restrict__ node) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= nl) return;
  node[nl + i] = i < n ? box[order[i]] : make_double4(1e300, 1e300, -1e300, -1e300);
}
__global__ void bvh_level_kernel(int64_t first, int64_t count, double4* __restrict__ node) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= count) return;
  const int64_t j = first + t;
  const double4 a = node[2 * j], b = node[2 * j + 1];
  node[j] = make_double4(fmin(a.x, b.x), fmin(a.y, b.y), fmax(a.z, b.z), fmax(a.w, b.w));
}

struct Geo {
  int q;
  const double2* cx;     // Legendre coefficients [n_panels][q]
  const double* xy;      // density nodes
  const double2* ends;   // [n_panels][2]
  const double* h;       // panel lengths
  const int* curve;      // curve of each panel
  const long long* coff; // [n_curves + 1] first panel of each curve
  const double* gl;      // Gauss-Legendre nodes on [-1, 1]
};

__device__ __forceinline__ bool adjacent(const Geo& G, int a, int b) {
  if (G.curve[a] != G.curve[b]) return false;
  const long long c0 = G.coff[G.curve[a]], n = G.coff[G.curve[a] + 1] - c0;
  if (n <= 1) return false;
  const long long d = (a - b + n) % n;
  return d == 1 || d == n - 1;
}

// Conditions 1 and 3 for every centre (one thread each): centre i of panel n,
// side sgn; visits the panels whose enlarged square meets the square of
// half-side h_n/2 about the centre.
__global__ void __launch_bounds__(kT) cond13_kernel(Geo G, int64_t n_ctr, int64_t n_nodes,
                                                    const double* __restrict__ ctr_xy,
                                                    int64_t nl, const double4* __restrict__ node,
                                                    const int* __restrict__ order,
                                                    const double4* __restrict__ pbox,
                                                    int* __restrict__ flags,
                                                    int* __restrict__ err) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n_ctr) return;
  const int n = (int)((i % n_nodes) / G.q);
  const double2 c = make_double2(ctr_xy[2 * i], ctr_xy[2 * i + 1]);
  const double r1 = 0.5 * G.h[n];
  const double4 Qb = make_double4(c.x - r1, c.y - r1, c.x + r1, c.y + r1);
  int64_t stack[kStack];
  int sp = 0;
  stack[sp++] = 1;
  bool f1 = false;
  while (sp > 0) {
    const int64_t j = stack[--sp];
    const double4 b = node[j];
    if (b.x > Qb.z || b.z < Qb.x || b.y > Qb.w || b.w < Qb.y) continue;
    if (j < nl) {
      if (sp + 2 > kStack) { atomicExch(err, 1); return; }
      stack[sp++] = 2 * j + 1;
      stack[sp++] = 2 * j;
      continue;
    }
    const int m = order[j - nl];
    if (m == n) continue;
    // Condition 3 needs the centre inside panel m's enlarged square
    const double4 pb = pbox[m];
    const bool in3 = c.x >= pb.x && c.x <= pb.z && c.y >= pb.y && c.y <= pb.w && !adjacent(G, n, m);
    const double r3 = 0.25 * G.h[m];
    const Curve C{G.cx + (int64_t)m * G.q, G.q};
    const double d = panel_distance(C, reinterpret_cast<const double2*>(G.xy) + (int64_t)m * G.q,
                                    G.gl, G.ends[2 * m], G.ends[2 * m + 1], c, r1,
                                    in3 ? r3 : r1);
    if (!f1 && d < r1) f1 = true;
    if (in3 && d < r3) atomicOr(&flags[m], QBX_COND3);
  }
  if (f1) atomicOr(&flags[n], QBX_COND1);
}

// Conditions 2 and 4 per panel.
__global__ void cond24_kernel(Geo G, int64_t n_panels, double k, int* __restrict__ flags) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= n_panels) return;
  if (k * G.h[p] > 5.0) atomicOr(&flags[p], QBX_COND4);
  const int cv = G.curve[p];
  const long long c0 = G.coff[cv], n = G.coff[cv + 1] - c0;
  if (n <= 1) return;
  const long long nx = c0 + (p - c0 + 1) % n;
  const double a = G.h[p], b = G.h[nx];
  if (a > 2.0 * b) atomicOr(&flags[p], QBX_COND2);
  if (b > 2.0 * a) atomicOr(&flags[nx], QBX_COND2);
}

// u* in (-1, 1) with arclength(-1, u*) = arclength(-1, 1) / 2 for every
// flagged panel (Newton's method; arclengths by q-point Gauss-Legendre).
__device__ double arclength(const Curve& C, const double* gl, const double* gw, double a,
                            double b) {
  double s = 0.0;
  for (int j = 0; j < C.q; ++j) {
    double2 x, d1, d2;
    C.eval(a + (b - a) * 0.5 * (gl[j] + 1.0), x, d1, d2);
    s += gw[j] * hypot(d1.x, d1.y);
  }
  return 0.5 * (b - a) * s;
}
__global__ void split_point_kernel(int64_t n, const int* __restrict__ which,
                                   const double2* __restrict__ cx, int q,
                                   const double* __restrict__ gl, const double* __restrict__ gw,
                                   double* __restrict__ ustar) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= n) return;
  const Curve C{cx + (int64_t)which[t] * q, q};
  const double half = 0.5 * arclength(C, gl, gw, -1.0, 1.0);
  double u = 0.0;
  for (int it = 0; it < 30; ++it) {
    double2 x, d1, d2;
    C.eval(u, x, d1, d2);
    const double f = arclength(C, gl, gw, -1.0, u) - half;
    const double un = fmin(0.99, fmax(-0.99, u - f / hypot(d1.x, d1.y)));
    if (fabs(un - u) < 1e-14) { u = un; break; }
    u = un;
  }
  ustar[t] = u;
}

// Nodes, normals and weights of the new panels: new panel p is the part
// [a, b] of old panel parent[p] (reference variable).
__global__ void new_nodes_kernel(int64_t n_new, int q, const int* __restrict__ parent,
                                 const double2* __restrict__ ab, const double2* __restrict__ cx,
                                 const double2* __restrict__ cn, const double* __restrict__ gl,
                                 const double* __restrict__ gw, double* __restrict__ xy,
                                 double* __restrict__ nrm, double* __restrict__ w) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n_new * q) return;
  const int64_t p = i / q;
  const int j = (int)(i % q);
  const Curve C{cx + (int64_t)parent[p] * q, q};
  const Curve N{cn + (int64_t)parent[p] * q, q};
  const double a = ab[p].x, b = ab[p].y;
  const double u = a + (b - a) * 0.5 * (gl[j] + 1.0);
  double2 x, d1, d2;
  C.eval(u, x, d1, d2);
  const double sp = hypot(d1.x, d1.y);
  double ox = d1.y / sp, oy = -d1.x / sp;
  const double2 nn = N.pos(u);
  if (ox * nn.x + oy * nn.y < 0.0) ox = -ox, oy = -oy;
  xy[2 * i] = x.x;
  xy[2 * i + 1] = x.y;
  nrm[2 * i] = ox;
  nrm[2 * i + 1] = oy;
  w[i] = gw[j] * sp * 0.5 * (b - a);
}

}  // namespace

// ---------------------------------------------------------------- host side
namespace {

struct PanelData {
  DevBuf<double2> cx, cn, ends;
  DevBuf<double4> box;
  DevBuf<double> gl, gw, w;
  DevBuf<int> curve;
  DevBuf<long long> coff;
};

qbx_status prepare(qbx_handle* h, PanelData& D) {
  const int q = h->q;
  std::vector<double> x, w;
  gl_nodes(q, x, w);
  std::vector<double> A((size_t)q * q);
  for (int j = 0; j < q; ++j) {  // P_n(u_j) by the recurrence
    double p0 = 1.0, p1 = x[j];
    for (int n = 0; n < q; ++n) {
      double pn;
      if (n == 0) pn = 1.0;
      else if (n == 1) pn = x[j];
      else {
        pn = ((2.0 * n - 1.0) * x[j] * p1 - (n - 1.0) * p0) / n;
        p0 = p1;
        p1 = pn;
      }
      A[(size_t)n * q + j] = 0.5 * (2.0 * n + 1.0) * w[j] * pn;
    }
  }
  DevBuf<double> dA;
  QBX_CUDA_TRY(dA.alloc(A.size()));
  QBX_CUDA_TRY(cudaMemcpy(dA.ptr, A.data(), A.size() * 8, cudaMemcpyHostToDevice));
  QBX_CUDA_TRY(D.gl.alloc(q));
  QBX_CUDA_TRY(D.gw.alloc(q));
  QBX_CUDA_TRY(cudaMemcpy(D.gl.ptr, x.data(), q * 8, cudaMemcpyHostToDevice));
  QBX_CUDA_TRY(cudaMemcpy(D.gw.ptr, w.data(), q * 8, cudaMemcpyHostToDevice));
  const int64_t np = h->n_panels;
  QBX_CUDA_TRY(D.cx.alloc(np * q));
  QBX_CUDA_TRY(D.cn.alloc(np * q));
  legendre_kernel<<<nblk(np, kT), kT>>>(np, q, dA.ptr, h->node_xy.ptr, h->node_nrm.ptr, D.cx.ptr,
                                        D.cn.ptr);
  QBX_CUDA_TRY(cudaGetLastError());
  // the curve of every panel
  std::vector<int> cur(np);
  for (int c = 0; c + 1 < (int)h->curve_off.size(); ++c)
    for (int64_t p = h->curve_off[c]; p < h->curve_off[c + 1]; ++p) cur[p] = c;
  QBX_CUDA_TRY(D.curve.alloc(np));
  QBX_CUDA_TRY(cudaMemcpy(D.curve.ptr, cur.data(), np * 4, cudaMemcpyHostToDevice));
  QBX_CUDA_TRY(D.coff.alloc(h->curve_off.size()));
  QBX_CUDA_TRY(cudaMemcpy(D.coff.ptr, h->curve_off.data(), h->curve_off.size() * 8,
                          cudaMemcpyHostToDevice));
  QBX_CUDA_TRY(cudaDeviceSynchronize());
  return QBX_OK;
}

// Density-grid weights w_j |dx/du| of every node, from the panels' expansions.
qbx_status expansion_weights(qbx_handle* h, PanelData& D, DevBuf<double>& wn) {
  const int64_t np = h->n_panels;
  const int q = h->q;
  QBX_CUDA_TRY(wn.alloc(h->n_nodes));
  {
    DevBuf<double> tmp_xy, tmp_n;
    DevBuf<int> par;
    DevBuf<double2> ab;
    QBX_CUDA_TRY(tmp_xy.alloc(2 * h->n_nodes));
    QBX_CUDA_TRY(tmp_n.alloc(2 * h->n_nodes));
    std::vector<int> pp(np);
    std::vector<double2> iv(np, make_double2(-1.0, 1.0));
    for (int64_t p = 0; p < np; ++p) pp[p] = (int)p;
    QBX_CUDA_TRY(par.alloc(np));
    QBX_CUDA_TRY(ab.alloc(np));
    QBX_CUDA_TRY(cudaMemcpy(par.ptr, pp.data(), np * 4, cudaMemcpyHostToDevice));
    QBX_CUDA_TRY(cudaMemcpy(ab.ptr, iv.data(), np * sizeof(double2), cudaMemcpyHostToDevice));
    new_nodes_kernel<<<nblk(np * q, kT), kT>>>(np, q, par.ptr, ab.ptr, D.cx.ptr, D.cn.ptr,
                                               D.gl.ptr, D.gw.ptr, tmp_xy.ptr, tmp_n.ptr, wn.ptr);
    QBX_CUDA_TRY(cudaGetLastError());
    QBX_CUDA_TRY(cudaDeviceSynchronize());
  }
  return QBX_OK;
}

qbx_status check(qbx_handle* h, PanelData& D, DevBuf<int>& flags) {
  const int64_t np = h->n_panels;
  const int q = h->q;
  if (q > kMaxQ) {
    set_error("qbx_check_conditions: q = %d above %d", q, kMaxQ);
    return QBX_ERR_ARG;
  }
  DevBuf<double> wn;  // for the centres of mass
  {
    const qbx_status st = expansion_weights(h, D, wn);
    if (st != QBX_OK) return st;
  }
  // domain square of the nodes
  std::vector<double> hxy(2 * h->n_nodes);
  QBX_CUDA_TRY(cudaMemcpy(hxy.data(), h->node_xy.ptr, hxy.size() * 8, cudaMemcpyDeviceToHost));
  double x0 = 1e300, y0 = 1e300, x1 = -1e300, y1 = -1e300;
  for (int64_t i = 0; i < h->n_nodes; ++i) {
    x0 = std::min(x0, hxy[2 * i]); x1 = std::max(x1, hxy[2 * i]);
    y0 = std::min(y0, hxy[2 * i + 1]); y1 = std::max(y1, hxy[2 * i + 1]);
  }
  const double side = std::max(x1 - x0, y1 - y0) * (1.0 + 1e-9) + 1e-300;
  const double4 dom = make_double4(x0, y0, x0 + side, y0 + side);
  QBX_CUDA_TRY(D.ends.alloc(2 * np));
  QBX_CUDA_TRY(D.box.alloc(np));
  DevBuf<unsigned long long> key, key2;
  DevBuf<int> id, order;
  QBX_CUDA_TRY(key.alloc(np));
  QBX_CUDA_TRY(key2.alloc(np));
  QBX_CUDA_TRY(id.alloc(np));
  QBX_CUDA_TRY(order.alloc(np));
  panel_box_kernel<<<nblk(np, kT), kT>>>(np, q, D.cx.ptr, h->node_xy.ptr, wn.ptr, h->panel_h.ptr,
                                         D.ends.ptr, D.box.ptr, dom, key.ptr, id.ptr);
  QBX_CUDA_TRY(cudaGetLastError());
  size_t tb = 0;
  QBX_CUDA_TRY(cub::DeviceRadixSort::SortPairs(nullptr, tb, key.ptr, key2.ptr, id.ptr, order.ptr,
                                               (int)np, 0, 32));
  DevBuf<unsigned char> tmp;
  QBX_CUDA_TRY(tmp.alloc(std::max<size_t>(1, tb)));
  QBX_CUDA_TRY(cub::DeviceRadixSort::SortPairs(tmp.ptr, tb, key.ptr, key2.ptr, id.ptr, order.ptr,
                                               (int)np, 0, 32));
  int L = 0;
  while ((int64_t(1) << L) < np) ++L;
  if (L + 2 > kStack) {
    set_error("qbx_check_conditions: too many panels");
    return QBX_ERR_ARG;
  }
  const int64_t nl = int64_t(1) << L;
  DevBuf<double4> node;
  QBX_CUDA_TRY(node.alloc(2 * nl));
  bvh_leaves_kernel<<<nblk(nl, kT), kT>>>(np, nl, order.ptr, D.box.ptr, node.ptr);
  QBX_CUDA_TRY(cudaGetLastError());
  for (int lev = L - 1; lev >= 0; --lev) {
    const int64_t first = int64_t(1) << lev;
    bvh_level_kernel<<<nblk(first, kT), kT>>>(first, first, node.ptr);
    QBX_CUDA_TRY(cudaGetLastError());
  }
  QBX_CUDA_TRY(flags.alloc(np));
  QBX_CUDA_TRY(cudaMemset(flags.ptr, 0, np * sizeof(int)));
  DevBuf<int> err;
  QBX_CUDA_TRY(err.alloc(1));
  QBX_CUDA_TRY(cudaMemset(err.ptr, 0, sizeof(int)));
  const Geo G{q, D.cx.ptr, h->node_xy.ptr, D.ends.ptr, h->panel_h.ptr, D.curve.ptr, D.coff.ptr,
              D.gl.ptr};
  if (np == 1) {
    // a single panel: no other panel to test against
  } else {
    cond13_kernel<<<nblk(h->n_ctr, kT), kT>>>(G, h->n_ctr, h->n_nodes, h->ctr_xy.ptr, nl,
                                              node.ptr, order.ptr, D.box.ptr, flags.ptr, err.ptr);
    QBX_CUDA_TRY(cudaGetLastError());
  }
  cond24_kernel<<<nblk(np, kT), kT>>>(G, np, h->k, flags.ptr);
  QBX_CUDA_TRY(cudaGetLastError());
  int herr = 0;
  QBX_CUDA_TRY(cudaMemcpy(&herr, err.ptr, sizeof(int), cudaMemcpyDeviceToHost));
  if (herr) {
    set_error("qbx_check_conditions: area query stack overflow");
    return QBX_ERR_CUDA;
  }
  return QBX_OK;
}

}  // namespace

// Density-grid weights of a handle whose geometry came without them.
qbx_status density_weights(qbx_handle* h) {
  if (h->q > kMaxQ) {
    set_error("q = %d above %d", h->q, kMaxQ);
    return QBX_ERR_ARG;
  }
  PanelData D;
  qbx_status st = prepare(h, D);
  if (st != QBX_OK) return st;
  return expansion_weights(h, D, h->node_w);
}

extern "C" qbx_status qbx_check_conditions(qbx_handle* h, int32_t* panel_flags, int64_t* counts) {
  set_error("%s", "");
  if (!h) {
    set_error("qbx_check_conditions: NULL handle");
    return QBX_ERR_ARG;
  }
  PanelData D;
  qbx_status st = prepare(h, D);
  if (st != QBX_OK) return st;
  DevBuf<int> flags;
  st = check(h, D, flags);
  if (st != QBX_OK) return st;
  std::vector<int> f(h->n_panels);
  QBX_CUDA_TRY(cudaMemcpy(f.data(), flags.ptr, f.size() * 4, cudaMemcpyDeviceToHost));
  if (panel_flags)
    QBX_CUDA_TRY(cudaMemcpy(panel_flags, f.data(), f.size() * 4, cudaMemcpyDefault));
  if (counts) {
    for (int c = 0; c < 4; ++c) counts[c] = 0;
    for (int v : f)
      for (int c = 0; c < 4; ++c)
        if (v & (1 << c)) counts[c] += 1;
  }
  return QBX_OK;
}

extern "C" qbx_status qbx_refine(qbx_handle* h, int32_t max_rounds, int32_t* rounds,
                                 int64_t* n_panels_out) {
  set_error("%s", "");
  if (!h || max_rounds < 0) {
    set_error("qbx_refine: bad arguments");
    return QBX_ERR_ARG;
  }
  if (h->own_src) {
    set_error("qbx_refine: the handle has a caller-supplied source grid, which the library "
              "cannot refine");
    return QBX_ERR_STATE;
  }
  const int q = h->q;
  int r = 0;
  for (;; ++r) {
    PanelData D;
    qbx_status st = prepare(h, D);
    if (st != QBX_OK) return st;
    DevBuf<int> flags;
    st = check(h, D, flags);
    if (st != QBX_OK) return st;
    const int64_t np = h->n_panels;
    std::vector<int> f(np);
    QBX_CUDA_TRY(cudaMemcpy(f.data(), flags.ptr, np * 4, cudaMemcpyDeviceToHost));
    std::vector<int> which;
    for (int64_t p = 0; p < np; ++p)
      if (f[p]) which.push_back((int)p);
    if (which.empty()) break;
    if (r >= max_rounds) {
      if (rounds) *rounds = r;
      if (n_panels_out) *n_panels_out = np;
      set_error("qbx_refine: %zu panels still break a condition after %d rounds", which.size(),
                r);
      return QBX_ERR_CONDITION;
    }
    // split points, then the new panel list (a flagged panel becomes two)
    DevBuf<int> dwhich;
    DevBuf<double> du;
    QBX_CUDA_TRY(dwhich.alloc(which.size()));
    QBX_CUDA_TRY(du.alloc(which.size()));
    QBX_CUDA_TRY(cudaMemcpy(dwhich.ptr, which.data(), which.size() * 4, cudaMemcpyHostToDevice));
    split_point_kernel<<<nblk((int64_t)which.size(), kT), kT>>>((int64_t)which.size(), dwhich.ptr,
                                                                D.cx.ptr, q, D.gl.ptr, D.gw.ptr,
                                                                du.ptr);
    QBX_CUDA_TRY(cudaGetLastError());
    std::vector<double> us(which.size());
    QBX_CUDA_TRY(cudaMemcpy(us.data(), du.ptr, us.size() * 8, cudaMemcpyDeviceToHost));
    std::vector<int> parent;
    std::vector<double2> ab;
    std::vector<long long> origin;
    std::vector<double2> interval;
    std::vector<long long> coff(1, 0);
    size_t wi = 0;
    for (int c = 0; c + 1 < (int)h->curve_off.size(); ++c) {
      for (int64_t p = h->curve_off[c]; p < h->curve_off[c + 1]; ++p) {
        const double2 I = h->panel_interval[p];
        auto push = [&](double a, double b) {
          parent.push_back((int)p);
          ab.push_back(make_double2(a, b));
          origin.push_back(h->panel_origin[p]);
          interval.push_back(make_double2(I.x + (I.y - I.x) * 0.5 * (a + 1.0),
                                          I.x + (I.y - I.x) * 0.5 * (b + 1.0)));
        };
        if (wi < which.size() && which[wi] == p) {
          push(-1.0, us[wi]);
          push(us[wi], 1.0);
          ++wi;
        } else {
          push(-1.0, 1.0);
        }
      }
      coff.push_back((long long)parent.size());
    }
    const int64_t nn = (int64_t)parent.size();
    DevBuf<int> dpar;
    DevBuf<double2> dab;
    DevBuf<double> nxy, nnrm, nw;
    QBX_CUDA_TRY(dpar.alloc(nn));
    QBX_CUDA_TRY(dab.alloc(nn));
    QBX_CUDA_TRY(nxy.alloc(2 * nn * q));
    QBX_CUDA_TRY(nnrm.alloc(2 * nn * q));
    QBX_CUDA_TRY(nw.alloc(nn * q));
    QBX_CUDA_TRY(cudaMemcpy(dpar.ptr, parent.data(), nn * 4, cudaMemcpyHostToDevice));
    QBX_CUDA_TRY(cudaMemcpy(dab.ptr, ab.data(), nn * sizeof(double2), cudaMemcpyHostToDevice));
    new_nodes_kernel<<<nblk(nn * q, kT), kT>>>(nn, q, dpar.ptr, dab.ptr, D.cx.ptr, D.cn.ptr,
                                               D.gl.ptr, D.gw.ptr, nxy.ptr, nnrm.ptr, nw.ptr);
    QBX_CUDA_TRY(cudaGetLastError());
    std::vector<double> hw(nn * q), hh(nn, 0.0);
    QBX_CUDA_TRY(cudaMemcpy(hw.data(), nw.ptr, hw.size() * 8, cudaMemcpyDeviceToHost));
    for (int64_t p = 0; p < nn; ++p)
      for (int j = 0; j < q; ++j) hh[p] += hw[p * q + j];
    h->panel_origin = origin;
    h->panel_interval = interval;
    h->curve_off = coff;
    st = replace_geometry(h, nn, nxy, nnrm, nw, hh);
    if (st != QBX_OK) return st;
  }
  if (rounds) *rounds = r;
  if (n_panels_out) *n_panels_out = h->n_panels;
  return QBX_OK;
}

extern "C" qbx_status qbx_get_geometry(const qbx_handle* h, int64_t* n_panels, double* node_xy,
                                       double* normal_xy, double* weight, double* panel_h,
                                       int64_t* panel_origin, double* panel_interval,
                                       int64_t* curve_panel_offset) {
  if (!h || !n_panels) {
    set_error("qbx_get_geometry: NULL argument");
    return QBX_ERR_ARG;
  }
  *n_panels = h->n_panels;
  const int64_t nn = h->n_nodes;
  if (node_xy) QBX_CUDA_TRY(cudaMemcpy(node_xy, h->node_xy.ptr, 2 * nn * 8, cudaMemcpyDefault));
  if (normal_xy)
    QBX_CUDA_TRY(cudaMemcpy(normal_xy, h->node_nrm.ptr, 2 * nn * 8, cudaMemcpyDefault));
  if (weight) QBX_CUDA_TRY(cudaMemcpy(weight, h->node_w.ptr, nn * 8, cudaMemcpyDefault));
  if (panel_h)
    QBX_CUDA_TRY(cudaMemcpy(panel_h, h->panel_h.ptr, h->n_panels * 8, cudaMemcpyDefault));
  if (panel_origin)
    QBX_CUDA_TRY(cudaMemcpy(panel_origin, h->panel_origin.data(), h->n_panels * 8,
                            cudaMemcpyDefault));
  if (panel_interval)
    QBX_CUDA_TRY(cudaMemcpy(panel_interval, h->panel_interval.data(), h->n_panels * 16,
                            cudaMemcpyDefault));
  if (curve_panel_offset)
    QBX_CUDA_TRY(cudaMemcpy(curve_panel_offset, h->curve_off.data(), h->curve_off.size() * 8,
                            cudaMemcpyDefault));
  return QBX_OK;
}
