// qbx_hankel01: the device evaluation of H_0 and H_1 of the first kind that
// every kernel of the library uses (ascending series, DLMF 10.2.2 and 10.8.1,
// below the series reach; the CUDA math library above), exposed so that it
// can be checked on its own.
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
