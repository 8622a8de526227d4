// Mixed-precision kernels (QBX_MIXED): the M2L translation of Stage 4 in complex
// FP32 with compensated (Kahan) accumulation.
//
// FP32 cannot hold the power-scaled expansions of the FP64 path (their
// translation entries still grow like a factorial), so the FP32 operators act
// on sigma-normalised coefficients
//     mu_n = a_n / sig_|n|,   lam_l = gamma_l sig_|l|,
//     sig_j = min(1, (x/2)^j / j!),  x = k * side  (the size of J_j at a box),
// for which every M2L entry sig_l sig_n (-1)^l W_{n+l}(D) is of order one or
// smaller. The entries are computed in FP64 (through logarithms of the scale
// factors) and stored as FP32 matrices, one per (level, offset class); the
// coefficient conversions between the two normalisations are FP64.
#include <algorithm>
#include <cmath>
#include <vector>

#include "tree.cuh"

namespace {

constexpr int kT = 128;

inline unsigned nblk(int64_t n, int b) { return (unsigned)std::max<int64_t>(1, (n + b - 1) / b); }

// per level: lsig[j] = log sig_j, conv[j] = s^j / sig_j  (j = 0..pb_l; stride pbmax + 1)
__global__ void sigma_tables_kernel(int n_levels, int pbmax, const int* __restrict__ lpb,
                                    double k, double side, const double* __restrict__ scale,
                                    double* __restrict__ lsig, double* __restrict__ conv) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= n_levels) return;
  const double x = k * side / (double)(1 << l);
  const double ls = log(scale[l]);
  for (int j = 0; j <= lpb[l]; ++j) {
    const double v = fmin(0.0, j * log(0.5 * x) - lgamma((double)j + 1.0));
    lsig[(size_t)l * (pbmax + 1) + j] = v;
    conv[(size_t)l * (pbmax + 1) + j] = exp(j * ls - v);
  }
}

// Level l's matrices Tm[cls][n][lo] = sig_lo sig_n (-1)^lo W_{n+lo}(D) (orders
// up to pb = pb_l), from the FP64 scaled Hankel vectors What_m = s^|m| W_m(D)
// (row stride 4 pbmax + 1, order m at m + 2 pbmax). Grid: (cls, n), threads over lo.
__global__ void m2l_f32_matrix_kernel(int l, int pb, int pbmax, const cd* __restrict__ t_m2l,
                                      const double* __restrict__ scale,
                                      const double* __restrict__ lsig, float2* __restrict__ Tm) {
  const int cls = blockIdx.x;
  const int n = (int)blockIdx.y - pb;
  const int Q = 2 * pb + 1;
  const cd* w = t_m2l + ((size_t)l * 49 + cls) * (4 * pbmax + 1) + 2 * pbmax;
  const double ls = log(scale[l]);
  const double* sg = lsig + (size_t)l * (pbmax + 1);
  float2* dst = Tm + ((size_t)cls * Q + (n + pb)) * Q;
  const int dx = cls / 7 - 3, dy = cls % 7 - 3;
  const bool used = max(abs(dx), abs(dy)) >= 2;  // V-list offsets only
  for (int lo = (int)threadIdx.x - pb; lo <= pb; lo += blockDim.x) {
    float2 out = make_float2(0.f, 0.f);
    if (used) {
      const cd v = w[n + lo];
      const double mag = hypot(v.x, v.y);  // entries reach 1e155: no squares
      if (mag > 0.0) {
        const double lf = sg[abs(lo)] + sg[abs(n)] - abs(n + lo) * ls + log(mag);
        const double f = lf < -700.0 ? 0.0 : exp(lf) / mag;
        const double sgn = (lo & 1) ? -f : f;
        out = make_float2((float)(v.x * sgn), (float)(v.y * sgn));
      }
    }
    dst[lo + pb] = out;
  }
}

__device__ __forceinline__ void kahan_add(float& s, float& c, float v) {
  const float y = v - c;
  const float t = s + y;
  c = (t - s) - y;
  s = t;
}

// CTA per box with a V list; threads over output orders lo, with the
// compensated sums (re, im, their compensations) of each order kept in shared
// memory.
__global__ void __launch_bounds__(kT) m2l_f32_kernel(
    int pbmax, const int* __restrict__ boxes, const int* __restrict__ level,
    const int* __restrict__ lpb, const long long* __restrict__ tm_off,
    const long long* __restrict__ eoff, const int* __restrict__ voff, const int* __restrict__ vidx,
    const int* __restrict__ vcls, const float2* __restrict__ tm, const double* __restrict__ conv,
    const cd* __restrict__ mpole, cd* __restrict__ local) {
  extern __shared__ float4 sacc[];               // [Q] (sum re, sum im, comp re, comp im)
  const int b = boxes[blockIdx.x];
  const int l = level[b];
  const int pb = lpb[l], Q = 2 * pb + 1;
  float2* mu = (float2*)(sacc + Q);              // [Q]
  const float2* Tm = tm + tm_off[l];
  const double* cv = conv + (size_t)l * (pbmax + 1);
  for (int i = threadIdx.x; i < Q; i += kT) sacc[i] = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int e = voff[b]; e < voff[b + 1]; ++e) {
    const cd* mp = mpole + eoff[vidx[e]];
    for (int i = threadIdx.x; i < Q; i += kT) {
      const cd a = mp[i];
      const double f = cv[abs(i - pb)];
      mu[i] = make_float2((float)(a.x * f), (float)(a.y * f));
    }
    __syncthreads();
    const float2* M = Tm + (size_t)vcls[e] * Q * Q;
    for (int lo = (int)threadIdx.x - pb; lo <= pb; lo += kT) {
      float4 acc = sacc[lo + pb];
      for (int n = 0; n < Q; ++n) {
        const float2 t = M[(size_t)n * Q + lo + pb];
        const float2 m = mu[n];
        kahan_add(acc.x, acc.z, fmaf(t.x, m.x, -t.y * m.y));
        kahan_add(acc.y, acc.w, fmaf(t.x, m.y, t.y * m.x));
      }
      sacc[lo + pb] = acc;
    }
    __syncthreads();
  }
  cd* dst = local + eoff[b];
  for (int lo = (int)threadIdx.x - pb; lo <= pb; lo += kT) {
    const float4 acc = sacc[lo + pb];
    const double f = cv[abs(lo)];
    dst[lo + pb].x += ((double)acc.x - (double)acc.z) * f;
    dst[lo + pb].y += ((double)acc.y - (double)acc.w) * f;
  }
}

}  // namespace

qbx_status configure_mixed_kernels(int smem_optin) {
  QBX_CUDA_TRY(cudaFuncSetAttribute((const void*)m2l_f32_kernel,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, smem_optin));
  return QBX_OK;
}

qbx_status mixed_plan_build(qbx_handle* h, FmmPlan* f) {
  const int pbm = f->pb_max;
  QBX_CUDA_TRY(f->lsig.alloc((size_t)f->n_levels * (pbm + 1)));
  QBX_CUDA_TRY(f->conv.alloc((size_t)f->n_levels * (pbm + 1)));
  sigma_tables_kernel<<<1, 64>>>(f->n_levels, pbm, f->lpb.ptr, h->k, f->side, f->scale.ptr,
                                 f->lsig.ptr, f->conv.ptr);
  QBX_CUDA_TRY(cudaGetLastError());
  // matrices for the levels that have V lists
  std::vector<long long> off(f->n_levels, 0);
  long long tot = 0;
  for (int l = 0; l < f->n_levels; ++l) {
    off[l] = tot;
    if (f->vbox_off[l + 1] > f->vbox_off[l]) {
      const long long Q = 2 * f->h_pb[l] + 1;
      tot += 49 * Q * Q;
    }
  }
  QBX_CUDA_TRY(f->tm_f32.alloc(std::max<long long>(1, tot)));
  QBX_CUDA_TRY(f->tm_off.alloc(f->n_levels));
  QBX_CUDA_TRY(cudaMemcpy(f->tm_off.ptr, off.data(), off.size() * sizeof(long long),
                          cudaMemcpyHostToDevice));
  f->h_tm_off = off;
  for (int l = 2; l < f->n_levels; ++l) {
    if (f->vbox_off[l + 1] == f->vbox_off[l]) continue;
    const int pb = f->h_pb[l];
    dim3 grid(49, 2 * pb + 1);
    m2l_f32_matrix_kernel<<<grid, kT>>>(l, pb, pbm, f->t_m2l.ptr, f->scale.ptr, f->lsig.ptr,
                                        f->tm_f32.ptr + off[l]);
    QBX_CUDA_TRY(cudaGetLastError());
  }
  return QBX_OK;
}

qbx_status launch_m2l_f32(qbx_handle* h, FmmPlan* f, cudaStream_t s) {
  if (f->n_vbox == 0) return QBX_OK;
  int pbv = 0;  // largest order among levels with V lists (vbox runs coarse to fine)
  for (int l = 0; l < f->n_levels; ++l)
    if (f->vbox_off[l + 1] > f->vbox_off[l]) pbv = std::max(pbv, f->h_pb[l]);
  const size_t sm = (size_t)(2 * pbv + 1) * (sizeof(float4) + sizeof(float2));
  m2l_f32_kernel<<<f->n_vbox, kT, sm, s>>>(
      f->pb_max, f->vbox.ptr, f->box.level.ptr, f->lpb.ptr, f->tm_off.ptr, f->eoff.ptr,
      f->V.off.ptr, f->V.idx.ptr, f->V_cls.ptr, f->tm_f32.ptr, f->conv.ptr, f->mpole.ptr,
      f->local.ptr);
  QBX_CUDA_TRY(cudaGetLastError());
  h->launches += 1;
  return QBX_OK;
}
