// qbx_hankel01: the device evaluation of H_0 and H_1 of the first kind that
// every kernel of the library uses (piecewise polynomials below x = 8, the
// CUDA math library above), exposed so that it can be checked on its own.
#include <cmath>

#include "special.cuh"

namespace {

template <bool WIDE>
__global__ void hankel01_kernel(const double* __restrict__ x, int64_t n, double4* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double xi = x[i];
  cd h0, h1;
  if (WIDE)
    hankel01_wide(xi, 1.0 / xi, h0, h1);
  else
    hankel01(xi, 1.0 / xi, h0, h1);
  out[i] = make_double4(h0.x, h0.y, h1.x, h1.y);
}

}  // namespace

extern "C" qbx_status qbx_hankel01(const double* x, int64_t n, int32_t variant, double* out) {
  set_error("%s", "");
  if (n < 0 || (n > 0 && (!x || !out)) || (variant != 0 && variant != 1)) {
    set_error("qbx_hankel01: bad arguments (n = %lld, variant = %d)", (long long)n, variant);
    return QBX_ERR_ARG;
  }
  if (n == 0) return QBX_OK;
  for (int64_t i = 0; i < n; ++i)
    if (!(x[i] > 0.0) || !std::isfinite(x[i])) {
      set_error("qbx_hankel01: x[%lld] = %g is not a positive finite number", (long long)i, x[i]);
      return QBX_ERR_ARG;
    }
  DevBuf<double> dx;
  DevBuf<double4> dout;
  QBX_CUDA_TRY(dx.alloc(n));
  QBX_CUDA_TRY(dout.alloc(n));
  QBX_CUDA_TRY(cudaMemcpy(dx.ptr, x, n * sizeof(double), cudaMemcpyHostToDevice));
  const unsigned blocks = (unsigned)((n + 127) / 128);
  if (variant == 1)
    hankel01_kernel<true><<<blocks, 128>>>(dx.ptr, n, dout.ptr);
  else
    hankel01_kernel<false><<<blocks, 128>>>(dx.ptr, n, dout.ptr);
  QBX_CUDA_TRY(cudaGetLastError());
  QBX_CUDA_TRY(cudaMemcpy(out, dout.ptr, n * sizeof(double4), cudaMemcpyDeviceToHost));
  return QBX_OK;
}

namespace {
__global__ void f32_from_f64_kernel(const double* __restrict__ x, int64_t n, float* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = f32_from_f64(x[i]);
}
}  // namespace

extern "C" qbx_status qbx_f32_from_f64(const double* x, int64_t n, float* out) {
  set_error("%s", "");
  if (n < 0 || (n > 0 && (!x || !out))) {
    set_error("qbx_f32_from_f64: bad arguments (n = %lld)", (long long)n);
    return QBX_ERR_ARG;
  }
  if (n == 0) return QBX_OK;
  DevBuf<double> dx;
  DevBuf<float> dout;
  QBX_CUDA_TRY(dx.alloc(n));
  QBX_CUDA_TRY(dout.alloc(n));
  QBX_CUDA_TRY(cudaMemcpy(dx.ptr, x, n * sizeof(double), cudaMemcpyHostToDevice));
  f32_from_f64_kernel<<<(unsigned)((n + 127) / 128), 128>>>(dx.ptr, n, dout.ptr);
  QBX_CUDA_TRY(cudaGetLastError());
  QBX_CUDA_TRY(cudaMemcpy(out, dout.ptr, n * sizeof(float), cudaMemcpyDeviceToHost));
  return QBX_OK;
}

namespace {
// Independent FMA chains per thread (kChains), kIters steps each; the inputs
// come from the caller so that nothing folds, and the result is stored only
// when it equals a value it cannot reach.
constexpr int kChains = 8;
template <typename T>
__global__ void __launch_bounds__(256) fma_rate_kernel(T b, T c, int iters, T* __restrict__ sink) {
  T a[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) a[i] = (T)(threadIdx.x + i);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < kChains; ++i) a[i] = fma(a[i], b, c);
  }
  T s = 0;
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += a[i];
  if (s == (T)-1.2345e30) *sink = s;
}

template <typename T>
qbx_status time_fma(int iters, double& tflops, T* sink) {
  int sms = 0, dev = 0;
  QBX_CUDA_TRY(cudaGetDevice(&dev));
  QBX_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const unsigned blocks = (unsigned)sms * 8, threads = 256;
  cudaEvent_t e0, e1;
  QBX_CUDA_TRY(cudaEventCreate(&e0));
  QBX_CUDA_TRY(cudaEventCreate(&e1));
  float best = 1e30f;
  for (int rep = 0; rep < 4; ++rep) {  // first launch warms up; best of the rest
    cudaEventRecord(e0);
    fma_rate_kernel<T><<<blocks, threads>>>((T)0.999999, (T)1e-7, iters, sink);
    cudaEventRecord(e1);
    QBX_CUDA_TRY(cudaGetLastError());
    QBX_CUDA_TRY(cudaEventSynchronize(e1));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (rep > 0) best = ms < best ? ms : best;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  tflops = 2.0 * kChains * (double)iters * blocks * threads / (best * 1e-3) / 1e12;
  return QBX_OK;
}
}  // namespace

extern "C" qbx_status qbx_measure_fma_rates(double* fp64_tflops, double* fp32_tflops) {
  set_error("%s", "");
  if (!fp64_tflops || !fp32_tflops) {
    set_error("qbx_measure_fma_rates: NULL output");
    return QBX_ERR_ARG;
  }
  DevBuf<double> sink;
  QBX_CUDA_TRY(sink.alloc(2));
  qbx_status s = time_fma<double>(2048, *fp64_tflops, sink.ptr);
  if (s != QBX_OK) return s;
  return time_fma<float>(65536, *fp32_tflops, reinterpret_cast<float*>(sink.ptr + 1));
}
