// step_f64.cu -- the plain FP64 form of ion_step (ION_F64_PLAIN): FP64 data
// and arithmetic everywhere.  It is bound by GB300's FP64 pipe, not by
// memory, so its design is about keeping that pipe's lanes busy:
//   * a persistent grid of warps draws groups of 32 cells from a counter in
//     the workspace header;
//   * cold cells (every window rate below the field at which the FP64 series
//     would take a term) are finished where they are found: N and the
//     freed electrons are left as they are, only the window rule runs;
//   * the others are sorted into per-warp queues by window width (2, 4, 6)
//     and by an FP32 estimate of their largest W dt (Taylor with few terms,
//     Taylor with many, Bateman form), and each queue is worked off 32
//     cells at a time, so that the FP64 arithmetic runs in full warps whose
//     lanes take the same path with the same width bound.
#include <cstdint>
#include <mutex>

#include "ion_cell.cuh"
#include "ion_step.cuh"

namespace ion {

namespace {

constexpr int kWarps = 8;
constexpr int kThreads = 32 * kWarps;
// width classes {<= 2, <= 4, <= 6} x forms {Taylor with at most 6 terms,
// Taylor, Bateman}
constexpr int kWidthClasses = 3;
constexpr int kClasses = 3 * kWidthClasses;
// a queue holds at most 31 cells left over plus one group's 32
constexpr int kQueueCap = 64;
// FP32 estimates of the largest W dt that pick the form class: 2 W dt below
// kThrF64[6] takes at most 6 Taylor terms; above 0.49 the FP64 cell most
// likely takes the Bateman form (its own FP64 rates decide).
constexpr float kFewTerms = 0.0139108f / 2.0f;
constexpr float kBateman = 0.49f;
constexpr int kRunF64 = 4;  // groups drawn per counter update

struct F64Smem {
  StagedF64 tab;
  StagedF32 tab32;  // for the FP32 estimate of the rates
  uint32_t queue[kWarps][kClasses][kQueueCap];
  int count[kWarps][kClasses];
};

// One batch of n <= 32 queued cells of width class wc, one per lane; returns
// the bits of |change of sum_k N_k| of the lane's cell (ION_CONSERVATION_CHECK).
__device__ __forceinline__ uint32_t f64_batch(const JobIO& J, const Policy& pol,
                                              const StagedF64& tab, const uint32_t* q, int n,
                                              int wc, int lane) {
  if (lane >= n) return 0u;
  const int c = (int)q[lane];
  const double Ec = static_cast<const double*>(J.E)[c];
  const int lo = J.lo[c], hi = J.hi[c];
  double d = 0.0;
  double* dp = (pol.flags & ION_CONSERVATION_CHECK) ? &d : nullptr;
  if (wc == 0)
    global_cell<F64Form, 2>(J, pol, tab, c, Ec, lo, hi, false, dp);
  else if (wc == 1)
    global_cell<F64Form, 4>(J, pol, tab, c, Ec, lo, hi, false, dp);
  else
    global_cell<F64Form, 6>(J, pol, tab, c, Ec, lo, hi, false, dp);
  return abs_bits(d);
}

__global__ void __launch_bounds__(kThreads)
    ion_step_f64_kernel(const __grid_constant__ JobIO J, const __grid_constant__ Policy pol,
                        uint32_t* hdr) {
  __shared__ F64Smem sm;
  __shared__ float ecold[ION_MAX_Z + ION_MAX_WINDOW];
  stage_f64(J.tab, pol.log2dt, &sm.tab);
  stage_f32(J.tab, pol.log2dt, &sm.tab32);
  if (threadIdx.x < 32) stage_cold(J.tab, pol.log2dt, kColdLog2F64, ecold, threadIdx.x);
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  if (lane < kClasses) sm.count[wib][lane] = 0;
  __syncthreads();
  uint32_t(*queue)[kQueueCap] = sm.queue[wib];
  int* count = sm.count[wib];
  const unsigned below = (1u << lane) - 1u;
  const int ngroups = (J.ncells + 31) / 32;
  int g = 0, left = 0;
  uint32_t cmax = 0;
  for (;;) {
    if (left == 0) {
      int b = 0;
      if (lane == 0) b = (int)atomicAdd(&hdr[kHdrChunk], (unsigned)kRunF64);
      g = __shfl_sync(kFull, b, 0);
      left = kRunF64;
    }
    if (g >= ngroups) break;  // groups come in increasing order: no more
    const int c = g * 32 + lane;
    ++g;
    --left;
    int cls = -1;
    if (c < J.ncells) {
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
        // class by width and by an FP32 estimate of the largest W dt
        const int w = hi - lo + 1;
        const FieldF32 f = field_f32((float)Ec);
        float lmax = 0.0f;
        if (!pol.zero_dt)
          for (int r = 0; r < w - 1; ++r) lmax = fmaxf(lmax, rate_dt_f32(sm.tab32, lo + r, f));
        const int form = lmax <= kFewTerms ? 0 : lmax <= kBateman ? 1 : 2;
        const int wc = w <= 2 ? 0 : w <= 4 ? 1 : 2;
        cls = form * kWidthClasses + wc;
      }
    }
    // append to the class queues; work off every queue holding a full warp
#pragma unroll 1
    for (int q = 0; q < kClasses; ++q) {
      const unsigned m = __ballot_sync(kFull, cls == q);
      if (!m) continue;
      const int n0 = count[q];
      if (cls == q) queue[q][n0 + __popc(m & below)] = (uint32_t)c;
      int n = n0 + __popc(m);
      __syncwarp();
      if (n >= 32) {
        n -= 32;
        cmax = max(cmax, f64_batch(J, pol, sm.tab, &queue[q][n], 32, q % kWidthClasses, lane));
        __syncwarp();
      }
      if (lane == 0) count[q] = n;
      __syncwarp();
    }
  }
  // what is left in the queues, in partial warps
#pragma unroll 1
  for (int q = 0; q < kClasses; ++q) {
    const int n = count[q];
    if (n > 0) cmax = max(cmax, f64_batch(J, pol, sm.tab, &queue[q][0], n, q % kWidthClasses, lane));
    __syncwarp();
  }
  if (pol.flags & ION_CONSERVATION_CHECK) warp_max_into(&hdr[kHdrCons], cmax);
}

std::mutex g_mu;
constexpr int kMaxDevices = 64;
int g_fit[kMaxDevices] = {};  // resident blocks per SM, per device (0: not yet)

}  // namespace

cudaError_t launch_step_f64(const JobIO& job, const Policy& pol, uint32_t* hdr,
                            cudaStream_t s) {
  if (job.ncells == 0) return cudaSuccess;
  int dev = 0, fit = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
    return e;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    const bool cache = dev >= 0 && dev < kMaxDevices;
    if (cache) fit = g_fit[dev];
    if (fit < 1) {
      if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fit, ion_step_f64_kernel,
                                                             kThreads, 0)) != cudaSuccess)
        return e;
      fit = fit < 1 ? 1 : fit;
      if (cache) g_fit[dev] = fit;
    }
  }
  // the group counter starts at 0 for every job
  if ((e = cudaMemsetAsync(hdr + kHdrChunk, 0, sizeof(uint32_t), s)) != cudaSuccess) return e;
  const int64_t groups = ((int64_t)job.ncells + 31) / 32;
  const int64_t need = (groups + kWarps - 1) / kWarps;
  const int64_t cap = (int64_t)fit * sms;
  const int blocks = (int)(need < cap ? need : cap);
  ion_step_f64_kernel<<<blocks, kThreads, 0, s>>>(job, pol, hdr);
  return cudaGetLastError();
}

}  // namespace ion
