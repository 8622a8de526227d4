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

// per level: lsig[j] = log sig_j, conv[j] = s^j / sig_j  (j = 0..pb)
__global__ void sigma_tables_kernel(int n_levels, int pb, double k, double side,
                                    const double* __restrict__ scale, double* __restrict__ lsig,
                                    double* __restrict__ conv) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= n_levels) return;
  const double x = k * side / (double)(1 << l);
  const double ls = log(scale[l]);
  for (int j = 0; j <= pb; ++j) {
    const double v = fmin(0.0, j * log(0.5 * x) - lgamma((double)j + 1.0));
    lsig[(size_t)l * (pb + 1) + j] = v;
    conv[(size_t)l * (pb + 1) + j] = exp(j * ls - v);
  }
}

// Tm[l][cls][n][lo] = sig_lo sig_n (-1)^lo W_{n+lo}(D), from the FP64 scaled
// Hankel vectors What_m = s^|m| W_m(D). Grid: (l*49 + cls, n), threads over lo.
__global__ void m2l_f32_matrix_kernel(int pb, const cd* __restrict__ t_m2l,
                                      const double* __restrict__ scale,
                                      const double* __restrict__ lsig, float2* __restrict__ Tm) {
  const int lc = blockIdx.x;            // l * 49 + cls
  const int l = lc / 49;
  const int n = (int)blockIdx.y - pb;
  const int Q = 2 * pb + 1, T = 4 * pb + 1;
  const cd* w = t_m2l + (size_t)lc * T;
  const double ls = log(scale[l]);
  const double* sg = lsig + (size_t)l * (pb + 1);
  float2* dst = Tm + ((size_t)lc * Q + (n + pb)) * Q;
  for (int lo = (int)threadIdx.x - pb; lo <= pb; lo += blockDim.x) {
    const cd v = w[n + lo + 2 * pb];
    const double mag = hypot(v.x, v.y);  // entries reach 1e155: no squares
    float2 out = make_float2(0.f, 0.f);
    if (mag > 0.0) {
      const double lf = sg[abs(lo)] + sg[abs(n)] - abs(n + lo) * ls + log(mag);
      const double f = lf < -700.0 ? 0.0 : exp(lf) / mag;
      const double sgn = (lo & 1) ? -f : f;
      out = make_float2((float)(v.x * sgn), (float)(v.y * sgn));
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

// CTA per box with a V list; threads over output orders lo.
__global__ void __launch_bounds__(kT) m2l_f32_kernel(
    int pb, const int* __restrict__ boxes, const int* __restrict__ level,
    const int* __restrict__ voff, const int* __restrict__ vidx, const int* __restrict__ vcls,
    const float2* __restrict__ Tm, const double* __restrict__ conv, const cd* __restrict__ mpole,
    cd* __restrict__ local) {
  extern __shared__ float2 mu[];  // [Q]
  const int Q = 2 * pb + 1;
  const int b = boxes[blockIdx.x];
  const int l = level[b];
  const double* cv = conv + (size_t)l * (pb + 1);
  float sr[2] = {0.f, 0.f}, si[2] = {0.f, 0.f}, cr[2] = {0.f, 0.f}, ci[2] = {0.f, 0.f};
  for (int e = voff[b]; e < voff[b + 1]; ++e) {
    const int c = vidx[e];
    for (int i = threadIdx.x; i < Q; i += kT) {
      const cd a = mpole[(size_t)c * Q + i];
      const double f = cv[abs(i - pb)];
      mu[i] = make_float2((float)(a.x * f), (float)(a.y * f));
    }
    __syncthreads();
    const float2* M = Tm + ((size_t)l * 49 + vcls[e]) * Q * Q;
    for (int o = 0; o < 2; ++o) {
      const int lo = (int)threadIdx.x + o * kT - pb;
      if (lo > pb) continue;
      for (int n = 0; n < Q; ++n) {
        const float2 t = M[(size_t)n * Q + lo + pb];
        const float2 m = mu[n];
        kahan_add(sr[o], cr[o], fmaf(t.x, m.x, -t.y * m.y));
        kahan_add(si[o], ci[o], fmaf(t.x, m.y, t.y * m.x));
      }
    }
    __syncthreads();
  }
  for (int o = 0; o < 2; ++o) {
    const int lo = (int)threadIdx.x + o * kT - pb;
    if (lo > pb) continue;
    const double f = cv[abs(lo)];
    cd* dst = local + (size_t)b * Q + lo + pb;
    dst->x += ((double)sr[o] - (double)cr[o]) * f;
    dst->y += ((double)si[o] - (double)ci[o]) * f;
  }
}

}  // namespace

qbx_status mixed_plan_build(qbx_handle* h, FmmPlan* f) {
  const int pb = f->pb, Q = f->Q;
  QBX_CUDA_TRY(f->lsig.alloc((size_t)f->n_levels * (pb + 1)));
  QBX_CUDA_TRY(f->conv.alloc((size_t)f->n_levels * (pb + 1)));
  sigma_tables_kernel<<<1, 64>>>(f->n_levels, pb, h->k, f->side, f->scale.ptr, f->lsig.ptr,
                                 f->conv.ptr);
  QBX_CUDA_TRY(cudaGetLastError());
  QBX_CUDA_TRY(f->tm_f32.alloc((size_t)f->n_levels * 49 * Q * Q));
  dim3 grid(f->n_levels * 49, Q);
  m2l_f32_matrix_kernel<<<grid, kT>>>(pb, f->t_m2l.ptr, f->scale.ptr, f->lsig.ptr,
                                      f->tm_f32.ptr);
  QBX_CUDA_TRY(cudaGetLastError());
  return QBX_OK;
}

qbx_status launch_m2l_f32(qbx_handle* h, FmmPlan* f, cudaStream_t s) {
  if (f->n_vbox == 0) return QBX_OK;
  m2l_f32_kernel<<<f->n_vbox, kT, f->Q * sizeof(float2), s>>>(
      f->pb, f->vbox.ptr, f->box.level.ptr, f->V.off.ptr, f->V.idx.ptr, f->V_cls.ptr,
      f->tm_f32.ptr, f->conv.ptr, f->mpole.ptr, f->local.ptr);
  QBX_CUDA_TRY(cudaGetLastError());
  h->launches += 1;
  return QBX_OK;
}
