// The exterior Dirichlet (sound-soft scattering) problem of Sec. 1 and
// Sec. 8.3: with the scattered field represented as u = D[sigma] + i k S[sigma],
// the boundary condition gives the second-kind equation (Eq. (extdir),
// Eq. (int_eq))
//     (1/2) sigma + D*[sigma] + i k S*[sigma] = f   on the curves.
// Its left side is the exterior one-sided limit of D[sigma] + i k S[sigma]
// (Sec. 2, Eq. (oneside), exterior limit D* + sigma/2), which is what Global
// QBX evaluates at a node from its exterior centre: one matrix-vector product
// is one qbx_layer_potential_eval with every density node as an on-surface
// target on the exterior side.
//
// The solver is restarted GMRES (Saad and Schultz, SIAM J. Sci. Stat. Comput.
// 7 (1986)) with classical Gram-Schmidt applied twice per Arnoldi step (two
// reductions per step instead of one per basis vector); the Krylov vectors
// live on the device and all vector arithmetic runs in the kernels below
// (dot products reduced in a fixed order, so results repeat bit for bit); the
// small Hessenberg least-squares problem is solved on the host with Givens
// rotations.
#include <algorithm>
#include <cmath>
#include <complex>
#include <vector>

#include "qbx_internal.h"

namespace {

constexpr int kT = 256;
constexpr int kBlocks = 304;   // 2 x 152 SMs: partial sums per dot product

inline unsigned nblk(int64_t n, int b) { return (unsigned)std::max<int64_t>(1, (n + b - 1) / b); }

__device__ cd block_sum(cd v, cd* sh) {
  for (int o = 16; o > 0; o >>= 1) {
    v.x += __shfl_down_sync(0xffffffffu, v.x, o);
    v.y += __shfl_down_sync(0xffffffffu, v.y, o);
  }
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  cd s = mk(0.0, 0.0);
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s = cadd(s, sh[w]);
  return s;
}

// part[i][b] = sum over block b's share of conj(V_i) w, for i < m (grid.y = m)
__global__ void __launch_bounds__(kT) dots_kernel(int64_t n, const cd* __restrict__ V,
                                                  int64_t ldv, const cd* __restrict__ w,
                                                  cd* __restrict__ part) {
  __shared__ cd sh[kT / 32];
  const int i = blockIdx.y;
  const cd* v = V + (int64_t)i * ldv;
  cd s = mk(0.0, 0.0);
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n;
       j += (int64_t)gridDim.x * blockDim.x)
    cfma(s, cconj(v[j]), w[j]);
  s = block_sum(s, sh);
  if (threadIdx.x == 0) part[(int64_t)i * gridDim.x + blockIdx.x] = s;
}
// out[i] = sum_b part[i][b], in block order
__global__ void sum_parts_kernel(int m, int nb, const cd* __restrict__ part, cd* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  cd s = mk(0.0, 0.0);
  for (int b = 0; b < nb; ++b) s = cadd(s, part[(int64_t)i * nb + b]);
  out[i] = s;
}
// w -= sum_{i < m} c_i V_i
__global__ void sub_combo_kernel(int64_t n, int m, const cd* __restrict__ V, int64_t ldv,
                                 const cd* __restrict__ c, cd* __restrict__ w) {
  const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= n) return;
  cd s = w[j];
  for (int i = 0; i < m; ++i) {
    const cd ci = c[i];
    const cd v = V[(int64_t)i * ldv + j];
    s = csub(s, cmul(ci, v));
  }
  w[j] = s;
}
// y = a x (+ y if add)
__global__ void scale_kernel(int64_t n, cd a, const cd* __restrict__ x, cd* __restrict__ y,
                             int add) {
  const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= n) return;
  const cd v = cmul(a, x[j]);
  y[j] = add ? cadd(y[j], v) : v;
}
// r = b - r
__global__ void residual_kernel(int64_t n, const cd* __restrict__ b, cd* __restrict__ r) {
  const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j < n) r[j] = csub(b[j], r[j]);
}

struct Krylov {
  int64_t n;
  cudaStream_t s;
  DevBuf<cd> part, dots;
  std::vector<cd> host;
  // c_i = <V_i, w>, i < m (fixed-order reduction), copied to host
  qbx_status dot(const cd* V, int64_t ldv, int m, const cd* w) {
    if (part.n < (size_t)m * kBlocks) QBX_CUDA_TRY(part.alloc((size_t)m * kBlocks));
    if (dots.n < (size_t)m) QBX_CUDA_TRY(dots.alloc(std::max(m, 64)));
    dots_kernel<<<dim3(kBlocks, m), kT, 0, s>>>(n, V, ldv, w, part.ptr);
    QBX_CUDA_TRY(cudaGetLastError());
    sum_parts_kernel<<<nblk(m, 64), 64, 0, s>>>(m, kBlocks, part.ptr, dots.ptr);
    QBX_CUDA_TRY(cudaGetLastError());
    host.resize(m);
    QBX_CUDA_TRY(cudaMemcpyAsync(host.data(), dots.ptr, m * sizeof(cd), cudaMemcpyDeviceToHost, s));
    QBX_CUDA_TRY(cudaStreamSynchronize(s));
    return QBX_OK;
  }
};

}  // namespace

extern "C" qbx_status qbx_solve_dirichlet(qbx_handle* h, const double* rhs, double* sigma_out,
                                          int32_t mode, int32_t p_fmm, int32_t precision,
                                          double tol, int32_t max_iter, int32_t restart,
                                          int32_t* iters_out, double* resid_out,
                                          void* cuda_stream) {
  set_error("%s", "");
  if (!h || !rhs || !sigma_out || !(tol > 0.0) || max_iter < 1 || restart < 1 || restart > 500) {
    set_error("qbx_solve_dirichlet: bad arguments");
    return QBX_ERR_ARG;
  }
  if (h->own_src) {
    set_error("qbx_solve_dirichlet: the unknowns live on the density nodes; a caller-supplied "
              "source grid takes densities on its own nodes");
    return QBX_ERR_STATE;
  }
  const int64_t n = h->n_nodes;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  // the plan: every density node an on-surface target, exterior side
  {
    std::vector<int64_t> on(n);
    std::vector<int8_t> side(n, 1);
    for (int64_t j = 0; j < n; ++j) on[j] = j;
    qbx_tree_desc d{};
    d.n_targets = n;
    d.target_xy = h->node_xy.ptr;
    d.on_surface_node = on.data();
    d.on_surface_side = side.data();
    d.mode = mode;
    d.p_fmm = p_fmm;
    d.p_add = -1;
    d.n_max = 0;
    d.eps_assoc = 0.0;
    d.assoc_out = nullptr;
    const qbx_status st = qbx_tree_build(h, &d);
    if (st != QBX_OK) return st;
  }
  const int m = std::min<int64_t>(restart, n);
  DevBuf<cd> V, w, b, x;
  QBX_CUDA_TRY(V.alloc((size_t)(m + 1) * n));
  QBX_CUDA_TRY(w.alloc(n));
  QBX_CUDA_TRY(b.alloc(n));
  QBX_CUDA_TRY(x.alloc(n));
  QBX_CUDA_TRY(cudaMemcpyAsync(b.ptr, rhs, n * sizeof(cd), cudaMemcpyDefault, s));
  QBX_CUDA_TRY(cudaMemsetAsync(x.ptr, 0, n * sizeof(cd), s));
  const double ikr = h->k;
  auto apply = [&](const cd* in, cd* out) -> qbx_status {  // out = A in
    return qbx_layer_potential_eval(h, 0.0, ikr, (const double*)in, 1.0, 0.0, (const double*)in,
                                    (double*)out, nullptr, precision, s);
  };
  Krylov K{n, s, {}, {}, {}};
  qbx_status st = K.dot(b.ptr, n, 1, b.ptr);
  if (st != QBX_OK) return st;
  const double bnorm = std::sqrt(K.host[0].x);
  int it = 0;
  double rel = 0.0;
  if (bnorm == 0.0) {
    const std::vector<cd> zero(n, mk(0.0, 0.0));
    QBX_CUDA_TRY(cudaMemcpyAsync(sigma_out, zero.data(), n * sizeof(cd), cudaMemcpyDefault, s));
    QBX_CUDA_TRY(cudaStreamSynchronize(s));
    if (iters_out) *iters_out = 0;
    if (resid_out) *resid_out = 0.0;
    return QBX_OK;
  }
  typedef std::complex<double> C;
  bool done = false;
  while (!done) {
    // r = b - A x into V_0
    if ((st = apply(x.ptr, V.ptr)) != QBX_OK) return st;
    residual_kernel<<<nblk(n, kT), kT, 0, s>>>(n, b.ptr, V.ptr);
    QBX_CUDA_TRY(cudaGetLastError());
    if ((st = K.dot(V.ptr, n, 1, V.ptr)) != QBX_OK) return st;
    const double beta = std::sqrt(K.host[0].x);
    rel = beta / bnorm;
    if (rel <= tol || it >= max_iter) break;
    scale_kernel<<<nblk(n, kT), kT, 0, s>>>(n, mk(1.0 / beta, 0.0), V.ptr, V.ptr, 0);
    QBX_CUDA_TRY(cudaGetLastError());
    std::vector<C> H((size_t)(m + 1) * m, C(0.0)), cs(m), sn(m), g(m + 1, C(0.0));
    g[0] = beta;
    int j = 0;
    for (; j < m && it < max_iter; ++j, ++it) {
      cd* vj1 = V.ptr + (int64_t)(j + 1) * n;
      if ((st = apply(V.ptr + (int64_t)j * n, vj1)) != QBX_OK) return st;
      // classical Gram-Schmidt, twice
      std::vector<C> hc(j + 1, C(0.0));
      for (int pass = 0; pass < 2; ++pass) {
        if ((st = K.dot(V.ptr, n, j + 1, vj1)) != QBX_OK) return st;
        std::vector<cd> c(K.host);
        for (int i = 0; i <= j; ++i) hc[i] += C(c[i].x, c[i].y);
        QBX_CUDA_TRY(cudaMemcpyAsync(K.dots.ptr, c.data(), (j + 1) * sizeof(cd),
                                     cudaMemcpyHostToDevice, s));
        sub_combo_kernel<<<nblk(n, kT), kT, 0, s>>>(n, j + 1, V.ptr, n, K.dots.ptr, vj1);
        QBX_CUDA_TRY(cudaGetLastError());
      }
      if ((st = K.dot(vj1, n, 1, vj1)) != QBX_OK) return st;
      const double hn = std::sqrt(K.host[0].x);
      for (int i = 0; i <= j; ++i) H[(size_t)i * m + j] = hc[i];
      H[(size_t)(j + 1) * m + j] = hn;
      if (hn > 0.0) {
        scale_kernel<<<nblk(n, kT), kT, 0, s>>>(n, mk(1.0 / hn, 0.0), vj1, vj1, 0);
        QBX_CUDA_TRY(cudaGetLastError());
      }
      // apply the earlier rotations to column j, then a new one
      for (int i = 0; i < j; ++i) {
        const C a = H[(size_t)i * m + j], bb = H[(size_t)(i + 1) * m + j];
        H[(size_t)i * m + j] = std::conj(cs[i]) * a + std::conj(sn[i]) * bb;
        H[(size_t)(i + 1) * m + j] = -sn[i] * a + cs[i] * bb;
      }
      const C a = H[(size_t)j * m + j], bb = H[(size_t)(j + 1) * m + j];
      const double r = std::sqrt(std::norm(a) + std::norm(bb));
      cs[j] = r > 0.0 ? a / r : C(1.0);
      sn[j] = r > 0.0 ? bb / r : C(0.0);
      H[(size_t)j * m + j] = r;
      H[(size_t)(j + 1) * m + j] = 0.0;
      g[j + 1] = -sn[j] * g[j];
      g[j] = std::conj(cs[j]) * g[j];
      rel = std::abs(g[j + 1]) / bnorm;
      if (rel <= tol || hn == 0.0) {
        ++j;
        ++it;
        break;
      }
    }
    // x += V y, H y = g (upper triangular j x j)
    std::vector<C> y(j);
    for (int i = j - 1; i >= 0; --i) {
      C t = g[i];
      for (int l = i + 1; l < j; ++l) t -= H[(size_t)i * m + l] * y[l];
      y[i] = t / H[(size_t)i * m + i];
    }
    for (int i = 0; i < j; ++i) {
      scale_kernel<<<nblk(n, kT), kT, 0, s>>>(n, mk(y[i].real(), y[i].imag()),
                                             V.ptr + (int64_t)i * n, x.ptr, 1);
      QBX_CUDA_TRY(cudaGetLastError());
    }
    if (rel <= tol || it >= max_iter) {
      // the true residual of the final iterate
      if ((st = apply(x.ptr, w.ptr)) != QBX_OK) return st;
      residual_kernel<<<nblk(n, kT), kT, 0, s>>>(n, b.ptr, w.ptr);
      QBX_CUDA_TRY(cudaGetLastError());
      if ((st = K.dot(w.ptr, n, 1, w.ptr)) != QBX_OK) return st;
      rel = std::sqrt(K.host[0].x) / bnorm;
      done = true;
    }
  }
  QBX_CUDA_TRY(cudaMemcpyAsync(sigma_out, x.ptr, n * sizeof(cd), cudaMemcpyDefault, s));
  QBX_CUDA_TRY(cudaStreamSynchronize(s));
  if (iters_out) *iters_out = it;
  if (resid_out) *resid_out = rel;
  return QBX_OK;
}
