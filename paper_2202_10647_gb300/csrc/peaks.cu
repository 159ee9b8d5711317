// peaks.cu -- ion_measure_peaks: throughput of the arithmetic the step's
// forms are bound by, measured on the current device (the HBM and tensor
// peaks come from elsewhere): FP32 ex2 and tanh on the SFU, FP64 fused
// multiply-add, and FP64 exp2 (a software sequence on the FP64 pipe).
// Every thread runs 8 independent dependency chains so that the loop
// measures issue throughput, not latency.
#include <cstdint>

#include "ion_device.cuh"
#include "ion_step.cuh"
#include "ionize.h"

namespace {

constexpr int kThreads = 256;
constexpr int kChains = 8;

__global__ void __launch_bounds__(kThreads) sfu_ex2_loop(float* out, int iters) {
  float a[kChains];
#pragma unroll
  for (int j = 0; j < kChains; ++j) a[j] = 0.01f * (threadIdx.x + j);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < kChains; ++j) a[j] = ion::ex2_approx(a[j] * -0.5f);
  }
  float s = 0.0f;
#pragma unroll
  for (int j = 0; j < kChains; ++j) s += a[j];
  if (s == 12345.0f) out[0] = s;  // keeps the chains alive
}

__device__ __forceinline__ float tanh_sfu(float x) {
  float y;
  asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__global__ void __launch_bounds__(kThreads) sfu_tanh_loop(float* out, int iters) {
  float a[kChains];
#pragma unroll
  for (int j = 0; j < kChains; ++j) a[j] = 0.01f * (threadIdx.x + j);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < kChains; ++j) a[j] = tanh_sfu(a[j] + 0.25f);
  }
  float s = 0.0f;
#pragma unroll
  for (int j = 0; j < kChains; ++j) s += a[j];
  if (s == 12345.0f) out[0] = s;
}

__global__ void __launch_bounds__(kThreads) dfma_loop(double* out, int iters) {
  double a[kChains];
#pragma unroll
  for (int j = 0; j < kChains; ++j) a[j] = 0.001 * (threadIdx.x + j);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < kChains; ++j) a[j] = fma(a[j], 0.999999, 1e-7);
  }
  double s = 0.0;
#pragma unroll
  for (int j = 0; j < kChains; ++j) s += a[j];
  if (s == 12345.0) out[0] = s;
}

__global__ void __launch_bounds__(kThreads) dexp2_loop(double* out, int iters) {
  double a[kChains];
#pragma unroll
  for (int j = 0; j < kChains; ++j) a[j] = 0.001 * (threadIdx.x + j);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < kChains; ++j) a[j] = exp2(a[j] * -0.5);
  }
  double s = 0.0;
#pragma unroll
  for (int j = 0; j < kChains; ++j) s += a[j];
  if (s == 12345.0) out[0] = s;
}

}  // namespace

extern "C" int ion_measure_peaks(double* out) {
  if (!out) return ion::set_error(ION_EINVAL, "ion_measure_peaks: out is NULL");
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess)
    return ion::set_error(ION_ECUDA, "ion_measure_peaks: %s", cudaGetErrorString(e));
  void* scratch = nullptr;
  cudaEvent_t a = nullptr, b = nullptr;
  if ((e = cudaMalloc(&scratch, 64)) != cudaSuccess ||
      (e = cudaEventCreate(&a)) != cudaSuccess || (e = cudaEventCreate(&b)) != cudaSuccess) {
    if (scratch) cudaFree(scratch);
    if (a) cudaEventDestroy(a);
    return ion::set_error(ION_ECUDA, "ion_measure_peaks: %s", cudaGetErrorString(e));
  }
  const int blocks = sms * 8;
  const double threads = (double)blocks * kThreads;
  // iteration counts sized for a few ms per loop
  const int it_sfu = 4096, it_fma = 8192, it_dexp = 256;
  float ms[4] = {0, 0, 0, 0};
  for (int k = 0; k < 4 && e == cudaSuccess; ++k) {
    for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {  // first run warms up
      cudaEventRecord(a, 0);
      switch (k) {
        case 0:
          sfu_ex2_loop<<<blocks, kThreads>>>(static_cast<float*>(scratch), it_sfu);
          break;
        case 1:
          sfu_tanh_loop<<<blocks, kThreads>>>(static_cast<float*>(scratch), it_sfu);
          break;
        case 2:
          dfma_loop<<<blocks, kThreads>>>(static_cast<double*>(scratch), it_fma);
          break;
        default:
          dexp2_loop<<<blocks, kThreads>>>(static_cast<double*>(scratch), it_dexp);
          break;
      }
      cudaEventRecord(b, 0);
      e = cudaEventSynchronize(b);
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms[k], a, b);
    }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  cudaFree(scratch);
  if (e != cudaSuccess)
    return ion::set_error(ION_ECUDA, "ion_measure_peaks: %s", cudaGetErrorString(e));
  out[0] = threads * it_sfu * kChains / (ms[0] * 1e-3);       // ex2 / s
  out[1] = threads * it_sfu * kChains / (ms[1] * 1e-3);       // tanh / s
  out[2] = 2.0 * threads * it_fma * kChains / (ms[2] * 1e-3);  // FP64 flop / s
  out[3] = threads * it_dexp * kChains / (ms[3] * 1e-3);      // FP64 exp2 / s
  return ion::set_error(ION_OK, "%s", "");
}

extern "C" int ion_binary_version(void) {
  cudaFuncAttributes fa;
  const cudaError_t e = cudaFuncGetAttributes(&fa, sfu_ex2_loop);
  if (e != cudaSuccess)
    return ion::set_error(ION_ECUDA, "ion_binary_version: %s", cudaGetErrorString(e));
  ion::set_error(ION_OK, "%s", "");
  return fa.binaryVersion;
}
