// Adaptive Dormand-Prince 5(4) steps of the moment ODE (FP64): the stage
// combinations y + h sum_j a_j k_j and the max-norm error of a step,
//   err = max_i |h sum_j e_j k_j[i]| / (atol + rtol max(|y_i|, |y5_i|)).
// The state y = (x, M) lives in two arrays (x: 2n values, M: K n values); a
// stage derivative k_j is one flat array of L = 2n + K n values, x part first.
#include <algorithm>

#include "particle_kernels.h"

namespace mmvm {

namespace {

__global__ void dp_combine_kernel(int n2, int L, const double* __restrict__ y_x,
                                  const double* __restrict__ y_M, const double* __restrict__ ks,
                                  DPCoef c, const double* h_dev, double* __restrict__ out_x,
                                  double* __restrict__ out_M) {
  const double h = *h_dev;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < L; i += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int j = 0; j < c.count; ++j) s = fma(c.w[j], ks[(size_t)j * L + i], s);
    if (i < n2)
      out_x[i] = fma(h, s, y_x[i]);
    else
      out_M[i - n2] = fma(h, s, y_M[i - n2]);
  }
}

__global__ void dp_error_kernel(int n2, int L, const double* __restrict__ y_x,
                                const double* __restrict__ y_M, const double* __restrict__ y5_x,
                                const double* __restrict__ y5_M, const double* __restrict__ ks,
                                DPCoef c, const double* h_dev, double rtol, double atol,
                                unsigned long long* err_bits) {
  __shared__ double red[32];
  const double h = *h_dev;
  double worst = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < L; i += gridDim.x * blockDim.x) {
    double e = 0.0;
    for (int j = 0; j < c.count; ++j) e = fma(c.w[j], ks[(size_t)j * L + i], e);
    const double y = i < n2 ? y_x[i] : y_M[i - n2];
    const double y5 = i < n2 ? y5_x[i] : y5_M[i - n2];
    const double v = fabs(h * e) / (atol + rtol * fmax(fabs(y), fabs(y5)));
    worst = (v > worst || v != v) ? v : worst;  // a NaN wins
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double w = __shfl_xor_sync(0xffffffffu, worst, o);
    worst = (w > worst || w != w) ? w : worst;
  }
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = worst;
  __syncthreads();
  if (threadIdx.x == 0) {
    double b = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) b = (red[i] > b || red[i] != red[i]) ? red[i] : b;
    // non-negative doubles (and NaN, whose bits are larger than +inf's) order
    // like their bit patterns
    atomicMax(err_bits, (unsigned long long)__double_as_longlong(b));
  }
}

}  // namespace

cudaError_t launch_dp_combine(int n, int K, const double* y_x, const double* y_M,
                              const double* ks, const DPCoef& c, const double* h_dev,
                              double* out_x, double* out_M, cudaStream_t st) {
  const int L = n * (2 + K);
  const int blocks = std::max(1, std::min((L + 255) / 256, 2048));
  dp_combine_kernel<<<blocks, 256, 0, st>>>(2 * n, L, y_x, y_M, ks, c, h_dev, out_x, out_M);
  return cudaGetLastError();
}

cudaError_t launch_dp_error(int n, int K, const double* y_x, const double* y_M,
                            const double* y5_x, const double* y5_M, const double* ks,
                            const DPCoef& c, const double* h_dev, double rtol, double atol,
                            unsigned long long* err_bits, cudaStream_t st) {
  const int L = n * (2 + K);
  const int blocks = std::max(1, std::min((L + 255) / 256, 1024));
  cudaError_t e = cudaMemsetAsync(err_bits, 0, sizeof(unsigned long long), st);
  if (e != cudaSuccess) return e;
  dp_error_kernel<<<blocks, 256, 0, st>>>(2 * n, L, y_x, y_M, y5_x, y5_M, ks, c, h_dev, rtol,
                                         atol, err_bits);
  return cudaGetLastError();
}

}  // namespace mmvm
