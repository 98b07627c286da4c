// Arithmetic peak of the device, measured: every thread of a full-occupancy
// grid runs independent fused multiply-add chains, so the FMA pipe is the only
// limit.  The all-pairs kernel is bound by that pipe, and its roofline
// fraction is reported against this number.
#include <cuda_runtime.h>

#include <string>

#include "../../include/mmvm.h"

namespace mmvm {
void set_last_error(const char* msg);
}

namespace {

constexpr int kChains = 8;   // independent accumulators per thread
constexpr int kUnroll = 16;  // FMAs per chain per loop trip
constexpr int kThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kThreads) fma_peak_kernel(T* sink, int iters, T a, T b) {
  T acc[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) acc[c] = T(threadIdx.x) * T(1e-7) + T(c);
#pragma unroll 1
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
      for (int c = 0; c < kChains; ++c) acc[c] = fma(acc[c], a, b);
    }
  }
  T s = T(0);
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += acc[c];
  // the chains converge to b / (1 - a) > 0, so this store never happens; it
  // only keeps the arithmetic alive
  if (s < T(-1) && sink) sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

int fail(int code, const std::string& m) {
  mmvm::set_last_error(m.c_str());
  return code;
}

template <typename T>
cudaError_t run(int blocks, int iters, cudaStream_t st, cudaEvent_t e0, cudaEvent_t e1,
                float* ms) {
  const T a = T(0.999999), b = T(1e-7);
  fma_peak_kernel<T><<<blocks, kThreads, 0, st>>>(nullptr, iters / 8, a, b);  // warm-up
  cudaError_t e = cudaEventRecord(e0, st);
  if (e != cudaSuccess) return e;
  fma_peak_kernel<T><<<blocks, kThreads, 0, st>>>(nullptr, iters, a, b);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = cudaEventRecord(e1, st)) != cudaSuccess) return e;
  if ((e = cudaEventSynchronize(e1)) != cudaSuccess) return e;
  return cudaEventElapsedTime(ms, e0, e1);
}

}  // namespace

extern "C" int mmvm_alu_peak(int32_t device, int32_t precision, double* flops_per_s) {
  if (!flops_per_s) return fail(MMVM_E_INVALID_ARG, "null argument");
  if (precision != MMVM_FP64 && precision != MMVM_MIXED_FP32)
    return fail(MMVM_E_INVALID_ARG, "unknown precision");
  cudaError_t e = cudaSetDevice(device);
  if (e != cudaSuccess) return fail(MMVM_E_DEVICE, cudaGetErrorString(e));
  int sms = 0, per_sm = 0;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device)) != cudaSuccess ||
      (e = cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxThreadsPerMultiProcessor, device)) !=
          cudaSuccess)
    return fail(MMVM_E_DEVICE, cudaGetErrorString(e));
  const int blocks = sms * (per_sm / kThreads);
  // about 50 ms at the expected rate of each pipe
  const int iters = precision == MMVM_MIXED_FP32 ? 40000 : 800;
  cudaStream_t st = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  float ms = 0.f;
  if ((e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking)) == cudaSuccess &&
      (e = cudaEventCreate(&e0)) == cudaSuccess && (e = cudaEventCreate(&e1)) == cudaSuccess) {
    e = precision == MMVM_MIXED_FP32 ? run<float>(blocks, iters, st, e0, e1, &ms)
                                     : run<double>(blocks, iters, st, e0, e1, &ms);
  }
  if (e1) cudaEventDestroy(e1);
  if (e0) cudaEventDestroy(e0);
  if (st) cudaStreamDestroy(st);
  if (e != cudaSuccess) return fail(MMVM_E_DEVICE, cudaGetErrorString(e));
  if (!(ms > 0.f)) return fail(MMVM_E_DEVICE, "timing failed");
  const double flops = 2.0 * kChains * kUnroll * (double)iters * blocks * kThreads;
  *flops_per_s = flops / (ms * 1e-3);
  return MMVM_OK;
}
