// step_f64.cu -- the plain FP64 form of ion_step (ION_F64_PLAIN): FP64 data
// and arithmetic everywhere, one cell per thread, every path inline, the
// warp's widest window as the width bound of all its lanes.  It is bound by
// GB300's FP64 rate, not by memory.
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
  __shared__ float ecold[ION_MAX_Z + ION_MAX_WINDOW];
  __shared__ int nq;
  __shared__ int queue[kThreads];
  if (threadIdx.x == 0) nq = 0;
  stage_f64(J.tab, pol.log2dt, &tab);
  if (threadIdx.x < 32) stage_cold(J.tab, pol.log2dt, kColdLog2F64, ecold, threadIdx.x);
  __syncthreads();
  const int64_t cl = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (cl < J.ncells) {
    const int c = (int)cl;
    const double Ec = static_cast<const double*>(J.E)[c];
    const int lo = J.lo[c], hi = J.hi[c];
    if (!window_ok(lo, hi, J.Z)) {
      atomicAdd(&hdr[kHdrInvalid], 1u);
    } else if (!pol.adaptive && hi > lo && fabs(Ec) < (double)ecold[lo]) {
      // Cold cell (|E| below the field at which its largest window rate
      // reaches 2^kColdLog2F64): the series would take no term
      // (2 W dt <= kThrF64[0]), so N stays as it is and no electron is
      // freed; only the window rule runs.  (The adaptive policy goes the
      // full way.)
      static_cast<double*>(J.dne)[c] = 0.0;
      if ((pol.flags & ION_NO_WINDOW_UPDATE) == 0 && hi < J.Z) {
        const double* p = static_cast<const double*>(J.N) + (int64_t)lo * J.ld + c;
        if (p[0] < pol.eps) {
          double v[ION_MAX_WINDOW];
#pragma unroll
          for (int r = 0; r < ION_MAX_WINDOW; ++r)
            v[r] = r < hi - lo ? p[(int64_t)r * J.ld] : 0.0;
          int nl = lo, nh = hi;
          slide_window<double, ION_MAX_WINDOW>(v, hi - lo + 1, J.Z, pol.eps, nl, nh);
          J.lo[c] = (uint8_t)nl;
          J.hi[c] = (uint8_t)nh;
        }
      }
    } else {
      queue[atomicAdd(&nq, 1)] = c;
    }
  }
  __syncthreads();
  // The block's other cells, packed into its first warps so that the FP64
  // work runs in full warps (cold and invalid cells no longer idle lanes of
  // it); the warp's widest window picks one width bound for all its lanes
  // (a per-lane switch would run every width present).
  const bool act = (int)threadIdx.x < nq;
  int c = 0, lo = 0, hi = 0;
  double Ec = 0.0;
  if (act) {
    c = queue[threadIdx.x];
    Ec = static_cast<const double*>(J.E)[c];
    lo = J.lo[c];
    hi = J.hi[c];
  }
  const int Wm = __reduce_max_sync(0xffffffffu, act ? hi - lo + 1 : 0);
  if (!act) return;
  if (Wm <= 2)
    global_cell<F64Form, 2>(J, pol, tab, c, Ec, lo, hi, false);
  else if (Wm <= 4)
    global_cell<F64Form, 4>(J, pol, tab, c, Ec, lo, hi, false);
  else
    global_cell<F64Form, 6>(J, pol, tab, c, Ec, lo, hi, false);
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
