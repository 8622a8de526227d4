// All-pairs ("direct") kernels of Global QBX, FP64:
//   strengths      per-source charge / dipole strengths
//   p2qbxl_direct  QBX coefficients at every centre from every source
//                  (Sec. 7, Eq. (localexpcoeffs); double layer by the normal
//                  derivative of the Graf kernel)
//   p2p_direct     smooth Gauss quadrature at unassociated targets
//                  (Sec. 3.2, Eq. (gauss-layerpot))
//   qbxl2p         truncated J-expansion at associated targets (Sec. 2.1, Eq. (phiapprox))
//   associate      target association (Sec. 6.1) by exhaustive search
//   place_centres  c = s + side (h/2) n (Sec. 2.2)
#include <cstdio>

#include "qbx_internal.h"
#include "special.cuh"

namespace {

constexpr int kTile = 128;

// q_j = (i/4) w_j cS sigmaS_j,  d_j = (i/4) w_j cD sigmaD_j
__global__ void strengths_kernel(int64_t n, const double* __restrict__ w, cd cS,
                                 const cd* __restrict__ sS, cd cD, const cd* __restrict__ sD,
                                 cd* __restrict__ q, cd* __restrict__ d) {
  int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= n) return;
  const cd i4 = mk(0.0, 0.25 * w[j]);
  q[j] = sS ? cmul(i4, cmul(cS, sS[j])) : mk(0.0, 0.0);
  d[j] = sD ? cmul(i4, cmul(cD, sD[j])) : mk(0.0, 0.0);
}

// One thread per centre; sources streamed through shared memory.
// With W_m = H_m(k r) e^{i m th} (th = arg(s - c)) and the complex normal
// nu = n_x + i n_y, the double-layer kernel of order m is
//   n . grad_s W_m = (k/2) (nu W_{m-1} - conj(nu) W_{m+1}),
// from (d_x +- i d_y) [Z_m(kr) e^{i m th}] = -+ k Z_{m+-1}(kr) e^{i(m+-1) th}
// (DLMF 10.6.2 in polar form). W_{-m} = (-1)^m H_m conj(e^{i m th}).
template <int PM, bool HS, bool HD>
__global__ void __launch_bounds__(kTile) p2qbxl_direct_kernel(
    int64_t n_ctr, const double* __restrict__ ctr_xy, int64_t n_src,
    const double* __restrict__ src_xy, const double* __restrict__ src_nrm,
    const cd* __restrict__ qs, const cd* __restrict__ ds, double k, int p,
    cd* __restrict__ alpha) {
  __shared__ double2 s_xy[kTile];
  __shared__ double2 s_nu[kTile];
  __shared__ cd s_q[kTile];
  __shared__ cd s_d[kTile];
  const int64_t c = blockIdx.x * (int64_t)kTile + threadIdx.x;
  const bool active = c < n_ctr;
  const double cx = active ? ctr_xy[2 * c] : 0.0;
  const double cy = active ? ctr_xy[2 * c + 1] : 0.0;
  const double hk = 0.5 * k;
  cd acc[2 * PM + 1];
#pragma unroll
  for (int i = 0; i <= 2 * PM; ++i) acc[i] = mk(0.0, 0.0);

  for (int64_t base = 0; base < n_src; base += kTile) {
    const int64_t j = base + threadIdx.x;
    if (j < n_src) {
      s_xy[threadIdx.x] = make_double2(src_xy[2 * j], src_xy[2 * j + 1]);
      if (HD) {
        s_nu[threadIdx.x] = make_double2(src_nrm[2 * j], src_nrm[2 * j + 1]);
        s_d[threadIdx.x] = ds[j];
      }
      if (HS) s_q[threadIdx.x] = qs[j];
    }
    __syncthreads();
    const int cnt = (int)min((int64_t)kTile, n_src - base);
    if (active) {
      for (int jj = 0; jj < cnt; ++jj) {
        const double dx = s_xy[jj].x - cx, dy = s_xy[jj].y - cy;
        const double r = sqrt(dx * dx + dy * dy);
        if (r == 0.0) continue;  // a source on a centre has no expansion (Condition 1)
        const double ir = 1.0 / r, x = k * r, ix2 = 2.0 / x;
        const cd e1 = mk(dx * ir, dy * ir);
        cd h0, h1;
        hankel01(x, h0, h1);
        cd q = HS ? s_q[jj] : mk(0.0, 0.0);
        cd dk = HD ? cscale(s_d[jj], hk) : mk(0.0, 0.0);
        cd nu = HD ? mk(s_nu[jj].x, s_nu[jj].y) : mk(0.0, 0.0);
        cd nub = cconj(nu);
        // m = 0
        cd w1 = cmul(h1, e1);              // W_1
        cd wm1 = cscale(cmul(h1, cconj(e1)), -1.0);  // W_{-1} = -H_1 conj(e1)
        if (HS) cfma(acc[PM], q, h0);
        if (HD) cfma(acc[PM], dk, csub(cmul(nu, wm1), cmul(nub, w1)));
        // running values: H_{m-1}, H_m, e^{i(m-1)th}, e^{i m th}
        cd hprev = h0, hcur = h1, eprev = mk(1.0, 0.0), ecur = e1;
        double sgn = -1.0;  // (-1)^m for m = 1
#pragma unroll
        for (int m = 1; m <= PM; ++m) {
          if (m > p) break;
          cd hnext = csub(cscale(hcur, (double)m * ix2), hprev);  // H_{m+1}
          cd enext = cmul(ecur, e1);
          cd w_m = cmul(hcur, ecur);
          cd w_p = cmul(hnext, enext);
          cd w_pm = cmul(hprev, eprev);
          // negative orders: W_{-m} = (-1)^m H_m conj(e_m)
          cd v_m = cscale(cmul(hcur, cconj(ecur)), sgn);
          cd v_p = cscale(cmul(hnext, cconj(enext)), -sgn);   // W_{-(m+1)}
          cd v_pm = cscale(cmul(hprev, cconj(eprev)), -sgn);  // W_{-(m-1)}
          if (HS) {
            cfma(acc[PM + m], q, w_m);
            cfma(acc[PM - m], q, v_m);
          }
          if (HD) {
            cfma(acc[PM + m], dk, csub(cmul(nu, w_pm), cmul(nub, w_p)));
            cfma(acc[PM - m], dk, csub(cmul(nu, v_p), cmul(nub, v_pm)));
          }
          hprev = hcur;
          hcur = hnext;
          eprev = ecur;
          ecur = enext;
          sgn = -sgn;
        }
      }
    }
    __syncthreads();
  }
  if (active) {
    const int P = 2 * p + 1;
#pragma unroll
    for (int l = -PM; l <= PM; ++l)
      if (l >= -p && l <= p) alpha[c * P + (l + p)] = acc[PM + l];
  }
}

// Smooth quadrature: u(t) = sum_j q_j H_0(k r) + d_j k H_1(k r) n_j.(t - s_j)/r
template <bool HS, bool HD>
__global__ void __launch_bounds__(kTile) p2p_direct_kernel(
    int64_t n_list, const int32_t* __restrict__ list, const double* __restrict__ tgt_xy,
    int64_t n_src, const double* __restrict__ src_xy, const double* __restrict__ src_nrm,
    const cd* __restrict__ qs, const cd* __restrict__ ds, double k, cd* __restrict__ out) {
  __shared__ double2 s_xy[kTile];
  __shared__ double2 s_n[kTile];
  __shared__ cd s_q[kTile];
  __shared__ cd s_d[kTile];
  const int64_t i = blockIdx.x * (int64_t)kTile + threadIdx.x;
  const bool active = i < n_list;
  const int64_t t = active ? list[i] : 0;
  const double tx = active ? tgt_xy[2 * t] : 0.0;
  const double ty = active ? tgt_xy[2 * t + 1] : 0.0;
  cd acc = mk(0.0, 0.0);
  for (int64_t base = 0; base < n_src; base += kTile) {
    const int64_t j = base + threadIdx.x;
    if (j < n_src) {
      s_xy[threadIdx.x] = make_double2(src_xy[2 * j], src_xy[2 * j + 1]);
      if (HS) s_q[threadIdx.x] = qs[j];
      if (HD) {
        s_n[threadIdx.x] = make_double2(src_nrm[2 * j], src_nrm[2 * j + 1]);
        s_d[threadIdx.x] = ds[j];
      }
    }
    __syncthreads();
    const int cnt = (int)min((int64_t)kTile, n_src - base);
    if (active) {
      for (int jj = 0; jj < cnt; ++jj) {
        const double dx = tx - s_xy[jj].x, dy = ty - s_xy[jj].y;
        const double r = sqrt(dx * dx + dy * dy);
        if (r == 0.0) continue;
        const double x = k * r;
        cd h0, h1;
        hankel01_any<false, HS, HD>(x, 1.0 / x, h0, h1);
        if (HS) cfma(acc, s_q[jj], h0);
        if (HD) cfma(acc, s_d[jj], cscale(h1, k * (s_n[jj].x * dx + s_n[jj].y * dy) / r));
      }
    }
    __syncthreads();
  }
  if (active) out[t] = acc;
}

// u(t) = sum_{|l| <= p} alpha_l(c) J_l(k rho) e^{-i l theta}, (rho, theta) the
// polar coordinates of t - c (Eq. (phiapprox)); J_{-m} = (-1)^m J_m.
template <int PM>
__device__ __forceinline__ cd qbx_local_eval(double tx, double ty, const double* __restrict__ ctr_xy,
                                             int64_t c, const cd* __restrict__ alpha, double k,
                                             int p) {
  const double dx = tx - ctr_xy[2 * c];
  const double dy = ty - ctr_xy[2 * c + 1];
  const double rho = sqrt(dx * dx + dy * dy);
  const cd e1 = rho > 0.0 ? mk(dx / rho, dy / rho) : mk(1.0, 0.0);
  double J[PM + 1];
  bessel_j_array<PM>(k * rho, J);
  const int P = 2 * p + 1;
  const cd* a = alpha + c * P + p;  // a[l], l = -p..p
  cd u = cscale(a[0], J[0]);
  cd e = mk(1.0, 0.0);
  double sgn = 1.0;
#pragma unroll
  for (int m = 1; m <= PM; ++m) {
    if (m > p) break;
    e = cmul(e, e1);
    sgn = -sgn;
    cfma(u, cscale(a[m], J[m]), cconj(e));
    cfma(u, cscale(a[-m], sgn * J[m]), e);
  }
  return u;
}

// QBX evaluation at the associated targets. A target marked in avg (an
// on-surface target asking for the on-surface value) gets the mean of its
// node's exterior (assoc) and interior (assoc + n_nodes) one-sided limits
// (Sec. 2, Eq. (oneside): the two limits differ by the jump of D).
template <int PM>
__global__ void __launch_bounds__(128) qbxl2p_kernel(int64_t n_list, const int32_t* __restrict__ list,
                                                     const double* __restrict__ tgt_xy,
                                                     const int32_t* __restrict__ assoc,
                                                     const int8_t* __restrict__ avg,
                                                     int64_t n_nodes,
                                                     const double* __restrict__ ctr_xy,
                                                     const cd* __restrict__ alpha, double k,
                                                     int p, cd* __restrict__ out) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n_list) return;
  const int64_t t = list[i];
  const int64_t c = assoc[t];
  const double tx = tgt_xy[2 * t], ty = tgt_xy[2 * t + 1];
  cd u = qbx_local_eval<PM>(tx, ty, ctr_xy, c, alpha, k, p);
  if (avg && avg[t]) {
    const cd v = qbx_local_eval<PM>(tx, ty, ctr_xy, c + n_nodes, alpha, k, p);
    u = mk(0.5 * (u.x + v.x), 0.5 * (u.y + v.y));
  }
  out[t] = u;
}

// Exhaustive association, arithmetic without contraction so that ties and
// boundaries are decided exactly as in a plain IEEE evaluation.
__global__ void associate_direct_kernel(int64_t n_tgt, const double* __restrict__ tgt_xy,
                                        const int64_t* __restrict__ on_node,
                                        const int8_t* __restrict__ on_side, int64_t n_nodes,
                                        const double* __restrict__ node_xy,
                                        const double* __restrict__ panel_h, int q,
                                        int64_t n_ctr, const double* __restrict__ ctr_xy,
                                        const double* __restrict__ ctr_r, double eps,
                                        int32_t* __restrict__ assoc, int32_t* __restrict__ ctrs) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= n_tgt) return;
  if (on_node && on_node[t] >= 0) {
    const int64_t j = on_node[t];
    const int side = on_side ? on_side[t] : 1;
    assoc[t] = (int32_t)(side >= 0 ? j : n_nodes + j);
    return;
  }
  const double tx = tgt_xy[2 * t], ty = tgt_xy[2 * t + 1];
  const double one_eps = __dadd_rn(1.0, eps);
  int64_t best = -1;
  double best_d2 = 1.0 / 0.0;
  for (int64_t c = 0; c < n_ctr; ++c) {
    const double dx = __dsub_rn(tx, ctr_xy[2 * c]);
    const double dy = __dsub_rn(ty, ctr_xy[2 * c + 1]);
    const double d2 = __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
    const double lim = __dmul_rn(one_eps, ctr_r[c]);
    if (d2 <= __dmul_rn(lim, lim) && d2 < best_d2) {
      best = c;
      best_d2 = d2;
    }
  }
  if (best >= 0) {
    assoc[t] = (int32_t)best;
    return;
  }
  for (int64_t j = 0; j < n_nodes; ++j) {
    const double dx = __dsub_rn(tx, node_xy[2 * j]);
    const double dy = __dsub_rn(ty, node_xy[2 * j + 1]);
    const double d2 = __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
    const double qh = __dmul_rn(0.25, panel_h[j / q]);
    if (d2 <= __dmul_rn(qh, qh)) {
      assoc[t] = -2;
      atomicAdd(&ctrs[0], 1);
      atomicMin(&ctrs[1], (int32_t)t);
      return;
    }
  }
  assoc[t] = -1;
}

__global__ void place_centres_kernel(int64_t n, int q, int sides, const double* __restrict__ node_xy,
                                     const double* __restrict__ node_nrm,
                                     const double* __restrict__ panel_h,
                                     double* __restrict__ ctr_xy, double* __restrict__ ctr_r) {
  const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= n) return;
  const double h = panel_h[j / q];
  for (int s = 0; s < sides; ++s) {
    const double a = (s == 0 ? 0.5 : -0.5) * h;  // exact: power-of-two scaling
    const int64_t c = j + s * n;
    ctr_xy[2 * c] = __dadd_rn(node_xy[2 * j], __dmul_rn(a, node_nrm[2 * j]));
    ctr_xy[2 * c + 1] = __dadd_rn(node_xy[2 * j + 1], __dmul_rn(a, node_nrm[2 * j + 1]));
    ctr_r[c] = 0.5 * h;
  }
}

inline unsigned nblk(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

template <int PM>
void p2qbxl_dispatch_flags(qbx_handle* h, bool S, bool D, cudaStream_t s) {
  dim3 g(nblk(h->n_ctr, kTile));
  if (S && D)
    p2qbxl_direct_kernel<PM, true, true><<<g, kTile, 0, s>>>(
        h->n_ctr, h->ctr_xy.ptr, h->n_src, h->src_xy.ptr, h->src_nrm.ptr, h->q_str.ptr,
        h->d_str.ptr, h->k, h->p, h->alpha.ptr);
  else if (S)
    p2qbxl_direct_kernel<PM, true, false><<<g, kTile, 0, s>>>(
        h->n_ctr, h->ctr_xy.ptr, h->n_src, h->src_xy.ptr, h->src_nrm.ptr, h->q_str.ptr,
        h->d_str.ptr, h->k, h->p, h->alpha.ptr);
  else
    p2qbxl_direct_kernel<PM, false, true><<<g, kTile, 0, s>>>(
        h->n_ctr, h->ctr_xy.ptr, h->n_src, h->src_xy.ptr, h->src_nrm.ptr, h->q_str.ptr,
        h->d_str.ptr, h->k, h->p, h->alpha.ptr);
}

}  // namespace

qbx_status launch_strengths(qbx_handle* h, cd cS, const cd* sigS, cd cD, const cd* sigD,
                            cudaStream_t s) {
  if (h->n_src == 0) return QBX_OK;
  strengths_kernel<<<nblk(h->n_src, 256), 256, 0, s>>>(h->n_src, h->src_w.ptr, cS, sigS, cD, sigD,
                                                     h->q_str.ptr, h->d_str.ptr);
  QBX_CUDA_TRY(cudaGetLastError());
  h->launches += 1;
  return QBX_OK;
}

qbx_status launch_p2qbxl_direct(qbx_handle* h, bool S, bool D, int precision, cudaStream_t s) {
  (void)precision;
  if (h->n_ctr == 0) return QBX_OK;
  if (!S && !D) {
    QBX_CUDA_TRY(cudaMemsetAsync(h->alpha.ptr, 0, h->alpha.n * sizeof(cd), s));
    return QBX_OK;
  }
  if (h->p <= 4) p2qbxl_dispatch_flags<4>(h, S, D, s);
  else if (h->p <= 8) p2qbxl_dispatch_flags<8>(h, S, D, s);
  else if (h->p <= 12) p2qbxl_dispatch_flags<12>(h, S, D, s);
  else p2qbxl_dispatch_flags<16>(h, S, D, s);
  QBX_CUDA_TRY(cudaGetLastError());
  h->launches += 1;
  return QBX_OK;
}

qbx_status launch_p2p_direct(qbx_handle* h, bool S, bool D, cd* out, int precision,
                             cudaStream_t s) {
  (void)precision;
  const int64_t n = h->n_direct_tgt;
  if (n == 0) return QBX_OK;
  dim3 g(nblk(n, kTile));
  if (S && D)
    p2p_direct_kernel<true, true><<<g, kTile, 0, s>>>(n, h->direct_tgt_list.ptr, h->tgt_xy.ptr,
                                                      h->n_src, h->src_xy.ptr, h->src_nrm.ptr,
                                                      h->q_str.ptr, h->d_str.ptr, h->k, out);
  else if (S)
    p2p_direct_kernel<true, false><<<g, kTile, 0, s>>>(n, h->direct_tgt_list.ptr, h->tgt_xy.ptr,
                                                       h->n_src, h->src_xy.ptr, h->src_nrm.ptr,
                                                       h->q_str.ptr, h->d_str.ptr, h->k, out);
  else if (D)
    p2p_direct_kernel<false, true><<<g, kTile, 0, s>>>(n, h->direct_tgt_list.ptr, h->tgt_xy.ptr,
                                                       h->n_src, h->src_xy.ptr, h->src_nrm.ptr,
                                                       h->q_str.ptr, h->d_str.ptr, h->k, out);
  else
    p2p_direct_kernel<false, false><<<g, kTile, 0, s>>>(n, h->direct_tgt_list.ptr, h->tgt_xy.ptr,
                                                        h->n_src, h->src_xy.ptr, h->src_nrm.ptr,
                                                        h->q_str.ptr, h->d_str.ptr, h->k, out);
  QBX_CUDA_TRY(cudaGetLastError());
  h->launches += 1;
  return QBX_OK;
}

qbx_status launch_qbxl2p(qbx_handle* h, cd* out, cudaStream_t s) {
  const int64_t n = h->n_qbx_tgt;
  if (n == 0) return QBX_OK;
  dim3 g(nblk(n, 128));
  const int8_t* avg = h->has_avg ? h->avg.ptr : nullptr;
#define QBXL2P_LAUNCH(PM)                                                                  \
  qbxl2p_kernel<PM><<<g, 128, 0, s>>>(n, h->qbx_tgt_list.ptr, h->tgt_xy.ptr, h->assoc.ptr, \
                                      avg, h->n_nodes, h->ctr_xy.ptr, h->alpha.ptr, h->k,  \
                                      h->p, out)
  if (h->p <= 4) QBXL2P_LAUNCH(4);
  else if (h->p <= 8) QBXL2P_LAUNCH(8);
  else if (h->p <= 12) QBXL2P_LAUNCH(12);
  else QBXL2P_LAUNCH(16);
#undef QBXL2P_LAUNCH
  QBX_CUDA_TRY(cudaGetLastError());
  h->launches += 1;
  return QBX_OK;
}

qbx_status launch_associate_direct(qbx_handle* h, const int64_t* on_node, const int8_t* on_side,
                                   double eps, cudaStream_t s) {
  if (h->n_tgt == 0) return QBX_OK;
  associate_direct_kernel<<<nblk(h->n_tgt, 128), 128, 0, s>>>(
      h->n_tgt, h->tgt_xy.ptr, on_node, on_side, h->n_nodes, h->node_xy.ptr, h->panel_h.ptr,
      h->q, h->n_ctr, h->ctr_xy.ptr, h->ctr_r.ptr, eps, h->assoc.ptr, h->counters.ptr);
  QBX_CUDA_TRY(cudaGetLastError());
  return QBX_OK;
}

qbx_status launch_place_centres(qbx_handle* h, cudaStream_t s) {
  if (h->n_nodes == 0) return QBX_OK;
  place_centres_kernel<<<nblk(h->n_nodes, 256), 256, 0, s>>>(
      h->n_nodes, h->q, h->sides, h->node_xy.ptr, h->node_nrm.ptr, h->panel_h.ptr, h->ctr_xy.ptr,
      h->ctr_r.ptr);
  QBX_CUDA_TRY(cudaGetLastError());
  return QBX_OK;
}

// ---------------------------------------------------------------- allocation-free entry point
// qbx_direct_qbx_eval_noalloc: the direct QBX evaluation (strengths -> coefficients
// at every centre from every source -> J-expansion at each target) for callers
// that may not allocate device memory. Its scratch (strengths and coefficients)
// is the file-scope array below, reserved once per device when the library's
// module loads and shared by every call on that device.
#include <mutex>

namespace {

constexpr int64_t kNoAllocScratch = int64_t(1) << 19;  // complex doubles = 8 MiB per device
static __device__ __align__(256) cd g_noalloc_scratch[kNoAllocScratch];

constexpr int kNoAllocMaxDevices = 128;
std::mutex g_noalloc_mu;
cd* g_noalloc_ptr[kNoAllocMaxDevices] = {};

// J-expansion of centre centre[t] at target t (Eq. (phiapprox)); an out-of-range
// centre index yields NaN for that target.
template <int PM>
__global__ void __launch_bounds__(128) qbxl2p_each_kernel(int64_t n_tgt,
                                                          const double* __restrict__ tgt_xy,
                                                          const int32_t* __restrict__ centre,
                                                          int64_t n_ctr,
                                                          const double* __restrict__ ctr_xy,
                                                          const cd* __restrict__ alpha, double k,
                                                          int p, cd* __restrict__ out) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= n_tgt) return;
  const int64_t c = centre[t];
  if (c < 0 || c >= n_ctr) {
    out[t] = mk(__longlong_as_double(0x7ff8000000000000LL), __longlong_as_double(0x7ff8000000000000LL));
    return;
  }
  const double dx = tgt_xy[2 * t] - ctr_xy[2 * c];
  const double dy = tgt_xy[2 * t + 1] - ctr_xy[2 * c + 1];
  const double rho = sqrt(dx * dx + dy * dy);
  const cd e1 = rho > 0.0 ? mk(dx / rho, dy / rho) : mk(1.0, 0.0);
  double J[PM + 1];
  bessel_j_array<PM>(k * rho, J);
  const int P = 2 * p + 1;
  const cd* a = alpha + c * P + p;
  cd u = cscale(a[0], J[0]);
  cd e = mk(1.0, 0.0);
  double sgn = 1.0;
#pragma unroll
  for (int m = 1; m <= PM; ++m) {
    if (m > p) break;
    e = cmul(e, e1);
    sgn = -sgn;
    cfma(u, cscale(a[m], J[m]), cconj(e));
    cfma(u, cscale(a[-m], sgn * J[m]), e);
  }
  out[t] = u;
}

// True if p is device (or managed) memory that belongs to device `dev`: a
// pointer into another GPU's memory would be dereferenced through peer access
// (or fault without it), so it is rejected like host memory.
bool on_device(const void* p, int dev) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) && a.device == dev;
}

template <int PM>
void noalloc_launch(int64_t n_src, const double* sxy, const double* snrm, const cd* q,
                    const cd* d, bool S, bool D, double k, int64_t n_ctr, const double* cxy,
                    int p, cd* alpha, int64_t n_tgt, const double* txy, const int32_t* tc,
                    cd* out, cudaStream_t s) {
  if (n_ctr > 0) {
    dim3 g(nblk(n_ctr, kTile));
    if (S && D)
      p2qbxl_direct_kernel<PM, true, true><<<g, kTile, 0, s>>>(n_ctr, cxy, n_src, sxy, snrm, q,
                                                               d, k, p, alpha);
    else if (S)
      p2qbxl_direct_kernel<PM, true, false><<<g, kTile, 0, s>>>(n_ctr, cxy, n_src, sxy, snrm, q,
                                                                d, k, p, alpha);
    else
      p2qbxl_direct_kernel<PM, false, true><<<g, kTile, 0, s>>>(n_ctr, cxy, n_src, sxy, snrm, q,
                                                                d, k, p, alpha);
  }
  if (n_tgt > 0)
    qbxl2p_each_kernel<PM><<<nblk(n_tgt, 128), 128, 0, s>>>(n_tgt, txy, tc, n_ctr, cxy, alpha, k,
                                                            p, out);
}

}  // namespace

extern "C" qbx_status qbx_direct_qbx_eval_noalloc(
    int64_t n_src, const double* src_xy, const double* src_normal_xy, const double* src_weight,
    double k, double cS_re, double cS_im, const double* sigma_S, double cD_re, double cD_im,
    const double* sigma_D, int64_t n_ctr, const double* ctr_xy, int32_t p, int64_t n_tgt,
    const double* tgt_xy, const int32_t* tgt_centre, double* out, void* cuda_stream) {
  set_error("%s", "");
  if (n_src < 0 || n_ctr < 0 || n_tgt < 0 || p < 0 || p > QBX_MAX_P || !(k > 0.0)) {
    set_error("qbx_direct_qbx_eval_noalloc: invalid size, order or wavenumber");
    return QBX_ERR_ARG;
  }
  if (!sigma_S && !sigma_D) {
    set_error("qbx_direct_qbx_eval_noalloc: at least one of sigma_S, sigma_D is required");
    return QBX_ERR_ARG;
  }
  const int64_t P = 2 * (int64_t)p + 1;
  // 2 n_src + n_ctr P <= kNoAllocScratch, checked term by term so that no
  // product can overflow
  if (n_src > kNoAllocScratch / 2 || n_ctr > (kNoAllocScratch - 2 * n_src) / P) {
    set_error("qbx_direct_qbx_eval_noalloc: n_src = %lld and n_ctr = %lld at p = %d need "
              "2*n_src + n_ctr*(2p+1) complex scratch values but the static scratch holds %lld",
              (long long)n_src, (long long)n_ctr, p, (long long)kNoAllocScratch);
    return QBX_ERR_ARG;
  }
  int dev = 0;
  QBX_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kNoAllocMaxDevices) {
    set_error("qbx_direct_qbx_eval_noalloc: device ordinal %d not supported", dev);
    return QBX_ERR_ARG;
  }
  static const char* const names[] = {"src_xy", "src_normal_xy", "src_weight", "ctr_xy",
                                      "tgt_xy", "tgt_centre", "out", "sigma_S", "sigma_D"};
  const void* dev_ptrs[] = {src_xy, src_normal_xy, src_weight, ctr_xy, tgt_xy,
                            tgt_centre, out, sigma_S, sigma_D};
  const int64_t sizes[] = {n_src, n_src, n_src, n_ctr, n_tgt, n_tgt, n_tgt,
                           sigma_S ? n_src : 0, sigma_D ? n_src : 0};
  for (int i = 0; i < 9; ++i)
    if (sizes[i] > 0 && (!dev_ptrs[i] || !on_device(dev_ptrs[i], dev))) {
      set_error("qbx_direct_qbx_eval_noalloc: %s must be device memory on the current "
                "device (%d)", names[i], dev);
      return QBX_ERR_ARG;
    }
  cd* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
      void* ptr = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
      if (e != cudaSuccess || !ptr) {
        set_error("qbx_direct_qbx_eval_noalloc: cudaGetSymbolAddress failed: %s",
                  cudaGetErrorString(e));
        return QBX_ERR_CUDA;
      }
      g_noalloc_ptr[dev] = (cd*)ptr;
    }
    scratch = g_noalloc_ptr[dev];
  }
  if (n_src == 0 && n_tgt == 0) return QBX_OK;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  cd* q = scratch;
  cd* d = scratch + n_src;
  cd* alpha = scratch + 2 * n_src;
  if (n_src > 0)
    strengths_kernel<<<nblk(n_src, 256), 256, 0, s>>>(
        n_src, src_weight, mk(cS_re, cS_im), (const cd*)sigma_S, mk(cD_re, cD_im),
        (const cd*)sigma_D, q, d);
  const bool S = sigma_S != nullptr, D = sigma_D != nullptr;
  const cd* cq = q;
  const cd* cdd = d;
  cd* o = (cd*)out;
  if (p <= 4)
    noalloc_launch<4>(n_src, src_xy, src_normal_xy, cq, cdd, S, D, k, n_ctr, ctr_xy, p, alpha,
                      n_tgt, tgt_xy, tgt_centre, o, s);
  else if (p <= 8)
    noalloc_launch<8>(n_src, src_xy, src_normal_xy, cq, cdd, S, D, k, n_ctr, ctr_xy, p, alpha,
                      n_tgt, tgt_xy, tgt_centre, o, s);
  else if (p <= 12)
    noalloc_launch<12>(n_src, src_xy, src_normal_xy, cq, cdd, S, D, k, n_ctr, ctr_xy, p, alpha,
                       n_tgt, tgt_xy, tgt_centre, o, s);
  else
    noalloc_launch<16>(n_src, src_xy, src_normal_xy, cq, cdd, S, D, k, n_ctr, ctr_xy, p, alpha,
                       n_tgt, tgt_xy, tgt_centre, o, s);
  QBX_CUDA_TRY(cudaGetLastError());
  return QBX_OK;
}
