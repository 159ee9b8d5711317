// check.cu -- ion_conservation: the largest deviation of a cell's population
// sum from its expected value, the diagnostic of multi-step runs.  The
// update of Eqs. 4-9 only moves population between the states of a window
// and the states outside it are not touched, so sum_k N_k of every cell is
// conserved by the method; this kernel measures how well the arithmetic
// keeps it.
#include <cmath>
#include <cstdint>

#include "ion_step.cuh"
#include "ionize.h"

namespace {

constexpr int kThreads = 256;
constexpr int kUnroll = 8;

// Non-negative floats (and NaN, whose bits lie above +inf) order like their
// bit patterns as unsigned integers.
__device__ __forceinline__ unsigned ordered_bits(float d) {
  return d != d ? 0x7fc00000u : __float_as_uint(d);
}

// Error-free sum of two floats: a + b = s + e exactly (Knuth's TwoSum).
__device__ __forceinline__ void two_sum_acc(float& s, float& e, float x) {
  const float t = s + x;
  const float bp = t - s;
  const float err = (s - (t - bp)) + (x - bp);
  s = t;
  e += err;
}

// FP32 populations, four cells per thread (ld % 4 == 0, N 16-byte aligned):
// each cell's planes are summed in float-float (TwoSum), whose error for a
// few dozen non-negative terms of order 1 stays below 1e-12, far under the
// FP32 rounding being measured; FP64 adds would make the kernel bound by
// GB300's FP64 rate instead of memory.
__global__ void __launch_bounds__(kThreads)
    conservation_f32x4_kernel(const float* __restrict__ N, int64_t ld, int64_t ncells,
                              int nplanes, double target, unsigned* out) {
  unsigned worst = 0;
  const int64_t stride = (int64_t)gridDim.x * kThreads * 4;
  for (int64_t c = ((int64_t)blockIdx.x * kThreads + threadIdx.x) * 4; c < ncells;
       c += stride) {
    const float4* p = reinterpret_cast<const float4*>(N + c);
    const int64_t ld4 = ld / 4;
    float s[4] = {0.f, 0.f, 0.f, 0.f}, e[4] = {0.f, 0.f, 0.f, 0.f};
    int k = 0;
    for (; k + kUnroll <= nplanes; k += kUnroll) {
      float4 x[kUnroll];
#pragma unroll
      for (int u = 0; u < kUnroll; ++u) x[u] = __ldcs(p + (int64_t)(k + u) * ld4);
#pragma unroll
      for (int u = 0; u < kUnroll; ++u) {
        two_sum_acc(s[0], e[0], x[u].x);
        two_sum_acc(s[1], e[1], x[u].y);
        two_sum_acc(s[2], e[2], x[u].z);
        two_sum_acc(s[3], e[3], x[u].w);
      }
    }
    for (; k < nplanes; ++k) {
      const float4 x = __ldcs(p + (int64_t)k * ld4);
      two_sum_acc(s[0], e[0], x.x);
      two_sum_acc(s[1], e[1], x.y);
      two_sum_acc(s[2], e[2], x.z);
      two_sum_acc(s[3], e[3], x.w);
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      if (c + j < ncells) {
        const double d = ((double)s[j] - target) + (double)e[j];
        worst = max(worst, ordered_bits((float)fabs(d)));
      }
    }
  }
  worst = __reduce_max_sync(0xffffffffu, worst);
  __shared__ unsigned red[kThreads / 32];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = worst;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned m = 0;
#pragma unroll
    for (int i = 0; i < kThreads / 32; ++i) m = max(m, red[i]);
    atomicMax(out, m);
  }
}

template <typename T>
__global__ void __launch_bounds__(kThreads)
    conservation_kernel(const T* __restrict__ N, int64_t ld, int64_t ncells, int nplanes,
                        double target, unsigned* out) {
  unsigned worst = 0;
  const int64_t stride = (int64_t)gridDim.x * kThreads;
  for (int64_t c = (int64_t)blockIdx.x * kThreads + threadIdx.x; c < ncells; c += stride) {
    const T* p = N + c;
    double s = 0.0;
    int k = 0;
    for (; k + kUnroll <= nplanes; k += kUnroll) {
      T x[kUnroll];
#pragma unroll
      for (int u = 0; u < kUnroll; ++u) x[u] = __ldcs(p + (int64_t)(k + u) * ld);
#pragma unroll
      for (int u = 0; u < kUnroll; ++u) s += (double)x[u];
    }
    for (; k < nplanes; ++k) s += (double)__ldcs(p + (int64_t)k * ld);
    worst = max(worst, ordered_bits((float)fabs(s - target)));
  }
  worst = __reduce_max_sync(0xffffffffu, worst);
  __shared__ unsigned red[kThreads / 32];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = worst;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned m = 0;
#pragma unroll
    for (int i = 0; i < kThreads / 32; ++i) m = max(m, red[i]);
    atomicMax(out, m);
  }
}

}  // namespace

extern "C" int ion_conservation(const void* N, int64_t ld, int64_t ncells, int nplanes,
                                double target, int dtype, float* out_max, void* stream) {
  if (dtype != ION_DTYPE_F32 && dtype != ION_DTYPE_F64)
    return ion::set_error(ION_EINVAL, "ion_conservation: unknown dtype %d", dtype);
  if (ncells < 0 || ncells >= (int64_t(1) << 40))
    return ion::set_error(ION_EINVAL, "ion_conservation: ncells=%lld out of range",
                          (long long)ncells);
  if (nplanes < 1 || nplanes > ION_MAX_Z + 1)
    return ion::set_error(ION_EINVAL, "ion_conservation: nplanes=%d outside [1, %d]", nplanes,
                          ION_MAX_Z + 1);
  if (!out_max || (reinterpret_cast<uintptr_t>(out_max) % 4) != 0)
    return ion::set_error(ION_EINVAL, "ion_conservation: out_max must be a 4-byte aligned "
                                      "device pointer");
  const size_t el = dtype == ION_DTYPE_F32 ? 4 : 8;
  if ((ncells > 0 && !N) || (reinterpret_cast<uintptr_t>(N) % el) != 0)
    return ion::set_error(ION_EINVAL, "ion_conservation: N must be non-NULL and aligned");
  if (ld < ncells || ld > (int64_t(1) << 40))
    return ion::set_error(ION_EINVAL, "ion_conservation: ld=%lld < ncells", (long long)ld);
  if (!std::isfinite(target))
    return ion::set_error(ION_EINVAL, "ion_conservation: target must be finite");
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess)
    return ion::set_error(ION_ECUDA, "ion_conservation: %s", cudaGetErrorString(e));
  const int64_t need = ncells > 0 ? (ncells + 4 * kThreads - 1) / (4 * kThreads) : 1;
  const int64_t cap = (int64_t)sms * (2048 / kThreads);
  const int blocks = (int)(need < cap ? need : cap);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  unsigned* out = reinterpret_cast<unsigned*>(out_max);
  if ((e = cudaMemsetAsync(out, 0, sizeof(unsigned), s)) != cudaSuccess)
    return ion::set_error(ION_ECUDA, "ion_conservation: %s", cudaGetErrorString(e));
  const bool x4 = dtype == ION_DTYPE_F32 && ld % 4 == 0 &&
                  (reinterpret_cast<uintptr_t>(N) % 16) == 0;
  if (x4)
    conservation_f32x4_kernel<<<blocks, kThreads, 0, s>>>(static_cast<const float*>(N), ld,
                                                          ncells, nplanes, target, out);
  else if (dtype == ION_DTYPE_F32)
    conservation_kernel<float><<<blocks, kThreads, 0, s>>>(static_cast<const float*>(N), ld,
                                                           ncells, nplanes, target, out);
  else
    conservation_kernel<double><<<blocks, kThreads, 0, s>>>(static_cast<const double*>(N), ld,
                                                            ncells, nplanes, target, out);
  e = cudaGetLastError();
  if (e != cudaSuccess)
    return ion::set_error(ION_ECUDA, "ion_conservation launch: %s", cudaGetErrorString(e));
  return ion::set_error(ION_OK, "%s", "");
}

extern "C" int ion_copy_cells(void* dst, int64_t ld_dst, const void* src, int64_t ld_src,
                              int nplanes, int64_t offset, int64_t ncells, int elem_bytes,
                              void* stream) {
  if (elem_bytes != 1 && elem_bytes != 2 && elem_bytes != 4 && elem_bytes != 8)
    return ion::set_error(ION_EINVAL, "ion_copy_cells: elem_bytes=%d not 1, 2, 4 or 8",
                          elem_bytes);
  if (nplanes < 1 || ncells < 0 || offset < 0)
    return ion::set_error(ION_EINVAL, "ion_copy_cells: need nplanes >= 1, ncells >= 0, "
                                      "offset >= 0");
  if (ncells == 0) return ion::set_error(ION_OK, "%s", "");
  if (!dst || !src) return ion::set_error(ION_EINVAL, "ion_copy_cells: NULL array");
  if (offset + ncells > ld_dst || offset + ncells > ld_src)
    return ion::set_error(ION_EINVAL, "ion_copy_cells: offset + ncells exceeds a row");
  const size_t eb = (size_t)elem_bytes;
  const cudaError_t e = cudaMemcpy2DAsync(
      static_cast<char*>(dst) + offset * eb, (size_t)ld_dst * eb,
      static_cast<const char*>(src) + offset * eb, (size_t)ld_src * eb, (size_t)ncells * eb,
      (size_t)nplanes, cudaMemcpyDefault, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess)
    return ion::set_error(ION_ECUDA, "ion_copy_cells: %s", cudaGetErrorString(e));
  return ion::set_error(ION_OK, "%s", "");
}
