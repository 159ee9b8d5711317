// step_f64.cu -- the plain FP64 form of ion_step (ION_F64_PLAIN): FP64 data
// and arithmetic everywhere, one cell per thread, every width and path
// inline.  It is bound by GB300's FP64 rate, not by memory.
#include <cstdint>

#include "ion_cell.cuh"
#include "ion_step.cuh"

namespace ion {

namespace {

constexpr int kThreads = 256;

__global__ void __launch_bounds__(kThreads)
    ion_step_f64_kernel(const __grid_constant__ JobIO J,
                        const __grid_constant__ Policy pol, uint32_t* hdr) {
  __shared__ StagedF64 tab;
  stage_f64(J.tab, pol.log2dt, &tab);
  __syncthreads();
  const int64_t cl = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (cl >= J.ncells) return;
  const int c = (int)cl;
  const double Ec = static_cast<const double*>(J.E)[c];
  const int lo = J.lo[c], hi = J.hi[c];
  if (!window_ok(lo, hi, J.Z)) {
    atomicAdd(&hdr[kHdrInvalid], 1u);
    return;
  }
  global_cell_any<F64Form>(J, pol, tab, c, Ec, lo, hi, false);
}

}  // namespace

cudaError_t launch_step_f64(const JobIO& job, const Policy& pol, uint32_t* hdr,
                            cudaStream_t s) {
  if (job.ncells == 0) return cudaSuccess;
  const int blocks = (int)((job.ncells + kThreads - 1) / kThreads);
  ion_step_f64_kernel<<<blocks, kThreads, 0, s>>>(job, pol, hdr);
  return cudaGetLastError();
}

}  // namespace ion
