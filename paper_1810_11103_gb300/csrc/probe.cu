// probe.cu -- FMA throughput probe used as the ALU roof of the roofline: eight
// independent multiply-add chains per thread keep the FP64 (or FP32) pipe saturated.
#include "fsp_internal.h"

namespace fsp {

template <typename T>
__global__ void __launch_bounds__(256) fma_peak_kernel(int iters, T* sink) {
  T x[8];
  const T a = T(0.9999999), b = T(1e-7);
#pragma unroll
  for (int k = 0; k < 8; ++k) x[k] = T(threadIdx.x + k) * T(1e-3);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = fma(x[k], a, b);
  }
  T s = T(0);
#pragma unroll
  for (int k = 0; k < 8; ++k) s += x[k];
  sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void round_to_float_kernel(const double* in, float* oi, float* oh, long long n) {
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
    oi[k] = from_f64_int(in[k]);
    oh[k] = __double2float_rn(in[k]);
  }
}

cudaError_t launch_round_to_float(const double* in, float* oi, float* oh, long long n, cudaStream_t st) {
  if (n > 0) round_to_float_kernel<<<(int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096), 256, 0, st>>>(in, oi, oh, n);
  return cudaGetLastError();
}

__global__ void widen_to_double_kernel(const float* in, double* oi, double* oh, long long n) {
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
    oi[k] = to_f64_int(in[k]);
    oh[k] = (double)in[k];
  }
}

cudaError_t launch_widen_to_double(const float* in, double* oi, double* oh, long long n, cudaStream_t st) {
  if (n > 0) widen_to_double_kernel<<<(int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096), 256, 0, st>>>(in, oi, oh, n);
  return cudaGetLastError();
}

// out[0..n): rcp_nr, [n..2n): 1/x; [2n..3n): rsq_nr, [3n..4n): 1/sqrt(x) (two IEEE roundings)
__global__ void reciprocal_check_kernel(const double* in, double* out, long long n) {
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
    const double x = in[k];
    out[k] = rcp_nr(x);
    out[n + k] = 1.0 / x;
    out[2 * n + k] = x > 0.0 ? rsq_nr(x) : 0.0;
    out[3 * n + k] = x > 0.0 ? 1.0 / sqrt(x) : 0.0;
  }
}

cudaError_t launch_reciprocal_check(const double* in, double* out, long long n, cudaStream_t st) {
  if (n > 0) reciprocal_check_kernel<<<(int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096), 256, 0, st>>>(in, out, n);
  return cudaGetLastError();
}

cudaError_t launch_fma_peak(int precision, int blocks, int iters, void* sink, cudaStream_t st) {
  if (precision == FSP_FP64)
    fma_peak_kernel<double><<<blocks, 256, 0, st>>>(iters, static_cast<double*>(sink));
  else
    fma_peak_kernel<float><<<blocks, 256, 0, st>>>(iters, static_cast<float*>(sink));
  return cudaGetLastError();
}

}  // namespace fsp
