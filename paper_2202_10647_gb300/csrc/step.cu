// step.cu -- the ion_step kernels.
//
// FP32 form (ION_F32), three kernels on the caller's stream:
//   ion_step_f32_kernel       persistent, one cell per thread per pass over
//                             all cells and every window width.  It finishes
//                             the cells whose rates all have W dt <= 0.025
//                             (at most four Taylor terms of exp(dt A)); the
//                             others ("hard" cells) are left untouched and
//                             queued, so that warps doing the long work are
//                             made of hard cells only.  In a laser field the
//                             instantaneous |E| swings from zero to its peak
//                             every few cells, so without this split almost
//                             every warp near the pulse would run the longest
//                             path of its lanes.
//   ion_step_f32_hard_kernel  the queued cells: Taylor form up to W dt <= 1,
//                             divided-difference (Bateman) form above; cells
//                             with a nearly degenerate rate pair go on to
//   ion_step_fb_kernel        FP32 rates, FP64 Bateman coefficients and
//                             propagation, rounded back.
// Plain FP64 form (ION_F64_PLAIN): ion_step_f64_kernel, one cell per thread,
// every width and path inline.
//
// One step is Eqs. 1-9 of the paper per cell; see ion_device.cuh.
#include <cstdint>

#include "ion_device.cuh"
#include "ion_step.cuh"

namespace ion {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kThreads = 256;

__device__ __forceinline__ bool window_ok(int lo, int hi, int Z) {
  return lo <= hi && hi <= Z && hi - lo + 1 <= ION_MAX_WINDOW;
}

// Per-precision hooks of the generic cell code.
struct F32Form {
  using T = float;
  using Staged = StagedF32;
  using Field = FieldF32;
  __device__ static Field field(float E) { return field_f32(E); }
  __device__ static float rate(const StagedF32& t, int k, const Field& f) {
    return rate_dt_f32(t, k, f);
  }
};

struct F64Form {
  using T = double;
  using Staged = StagedF64;
  struct Field {
    double E;
  };
  __device__ static Field field(double E) { return {E}; }
  __device__ static double rate(const StagedF64& t, int k, const Field& f) {
    return rate_dt_f64(t, k, f.E);
  }
};

// Warp-aggregated append of `value` for the lanes with `take` set: one
// atomic per warp.  Every lane of the warp calls this.
__device__ __forceinline__ void warp_append(uint32_t* counter, uint32_t* queue,
                                            bool take, uint32_t value) {
  const unsigned m = __ballot_sync(kFull, take);
  if (!m) return;
  const int lane = threadIdx.x & 31;
  unsigned base = 0;
  if (lane == 0) base = atomicAdd(counter, (unsigned)__popc(m));
  base = __shfl_sync(kFull, base, 0);
  if (take) queue[base + __popc(m & ((1u << lane) - 1u))] = value;
}

// ---------------------------------------------------------------------------
// One cell (index c, window [lo, hi] of width w <= WM, validated).
// Returns true if the cell was left to the FP64 queue.
// ---------------------------------------------------------------------------
template <class F, int WM>
__device__ __forceinline__ bool cell(const StepArgs& a,
                                     const typename F::Staged& tab, int c,
                                     typename F::T Ec, int lo, int hi,
                                     bool allow_fb) {
  using T = typename F::T;
  T* __restrict__ N = static_cast<T*>(a.N);
  const int64_t ld = a.ld;
  const int w = hi - lo + 1;
  T v[WM];
#pragma unroll
  for (int r = 0; r < WM; ++r)
    v[r] = r < w ? __ldcs(N + (int64_t)(lo + r) * ld + c) : T(0);

  T dne = T(0);
  int nlo = lo, nhi = hi;
  if constexpr (WM >= 2) {
   if (w >= 2) {
    const typename F::Field f = F::field(Ec);
    T lam[WM];
    T lmax = T(0);
#pragma unroll
    for (int r = 0; r < WM; ++r) {
      lam[r] = (r < w - 1 && !a.zero_dt) ? F::rate(tab, lo + r, f) : T(0);
      lmax = fmax(lmax, lam[r]);
    }
    if (lmax <= DDParams<T>::prop_max) {
      dne = taylor_propagate<T, WM>(v, lam, w, lmax);
    } else {
      if (allow_fb && (a.flags & ION_NO_FP64_FALLBACK) == 0 &&
          ((a.flags & ION_FORCE_FP64_COEF) != 0 ||
           (a.gap > 0.0 && near_degenerate<T, WM>(lam, w, (T)a.gap))))
        return true;
      dne = dd_update<T, WM>(v, lam, w);
    }
    if ((a.flags & ION_NO_WINDOW_UPDATE) == 0)
      slide_window<T, WM>(v, w, a.Z, (T)a.eps, nlo, nhi);
#pragma unroll
    for (int r = 0; r < WM; ++r)
      if (r < w) __stcs(N + (int64_t)(lo + r) * ld + c, v[r]);
   }
  }
  const T* __restrict__ G = static_cast<const T*>(a.n_gas);
  __stcs(static_cast<T*>(a.dne) + c, G ? dne * G[c] : dne);
  if (nlo != lo) {
    a.lo[c] = (uint8_t)nlo;
    a.hi[c] = (uint8_t)nhi;
  }
  return false;
}

// Dispatch on the warp's widest window (WMIN..WMAX instantiated).
template <class F, int WMIN, int WMAX>
__device__ __forceinline__ bool cell_bucket(int WMw, const StepArgs& a,
                                            const typename F::Staged& tab,
                                            int c, typename F::T Ec, int lo,
                                            int hi, bool ok, bool allow_fb) {
  if (!ok) return false;
  if (WMIN <= 1 && WMw <= 1) return cell<F, 1>(a, tab, c, Ec, lo, hi, allow_fb);
  if (WMIN <= 2 && WMAX >= 2 && WMw == 2) return cell<F, 2>(a, tab, c, Ec, lo, hi, allow_fb);
  if (WMIN <= 3 && WMAX >= 3 && WMw == 3) return cell<F, 3>(a, tab, c, Ec, lo, hi, allow_fb);
  if (WMIN <= 4 && WMAX >= 4 && WMw == 4) return cell<F, 4>(a, tab, c, Ec, lo, hi, allow_fb);
  if (WMIN <= 5 && WMAX >= 5 && WMw == 5) return cell<F, 5>(a, tab, c, Ec, lo, hi, allow_fb);
  if (WMAX >= 6 && WMw >= 6) return cell<F, 6>(a, tab, c, Ec, lo, hi, allow_fb);
  return false;
}

// Loads this thread's cell; returns the widest valid window of the warp.
template <class F>
__device__ __forceinline__ int load_cell(const StepArgs& a, int c, bool in,
                                         typename F::T& Ec, int& lo, int& hi,
                                         bool& ok) {
  using T = typename F::T;
  Ec = in ? __ldcs(static_cast<const T*>(a.E) + c) : T(0);
  lo = in ? __ldcs(a.lo + c) : 1;
  hi = in ? __ldcs(a.hi + c) : 0;
  ok = in && window_ok(lo, hi, a.Z);
  return __reduce_max_sync(kFull, ok ? hi - lo + 1 : 0);
}

// Kernel A's cell: finishes it if every W dt <= kLamEasy, else returns true
// (the cell is left untouched for the hard kernel).
constexpr float kLamEasy = 0.025f;  // 2 kLamEasy <= kThrF32[4]: 4 terms suffice
constexpr int kEasyTerms = 4;

template <int WM>
__device__ __forceinline__ bool easy_cell(const StepArgs& a, const StagedF32& tab,
                                          int c, float Ec, int lo, int hi) {
  float* __restrict__ N = static_cast<float*>(a.N);
  const int64_t ld = a.ld;
  const int w = hi - lo + 1;
  float v[WM];
#pragma unroll
  for (int r = 0; r < WM; ++r)
    v[r] = r < w ? __ldcs(N + (int64_t)(lo + r) * ld + c) : 0.0f;
  float dne = 0.0f;
  int nlo = lo, nhi = hi;
  if constexpr (WM >= 2) {
    if (w >= 2) {
      const FieldF32 f = field_f32(Ec);
      float lam[WM];
      float lmax = 0.0f;
#pragma unroll
      for (int r = 0; r < WM; ++r) {
        lam[r] = (r < w - 1 && !a.zero_dt) ? rate_dt_f32(tab, lo + r, f) : 0.0f;
        lmax = fmaxf(lmax, lam[r]);
      }
      if (lmax > kLamEasy) return true;
      dne = taylor_propagate<float, WM, kEasyTerms>(v, lam, w, lmax);
      if ((a.flags & ION_NO_WINDOW_UPDATE) == 0)
        slide_window<float, WM>(v, w, a.Z, (float)a.eps, nlo, nhi);
#pragma unroll
      for (int r = 0; r < WM; ++r)
        if (r < w) __stcs(N + (int64_t)(lo + r) * ld + c, v[r]);
    }
  }
  const float* __restrict__ G = static_cast<const float*>(a.n_gas);
  __stcs(static_cast<float*>(a.dne) + c, G ? dne * G[c] : dne);
  if (nlo != lo) {
    a.lo[c] = (uint8_t)nlo;
    a.hi[c] = (uint8_t)nhi;
  }
  return false;
}

__global__ void __launch_bounds__(kThreads)
    ion_step_f32_kernel(const __grid_constant__ StepArgs a) {
  __shared__ StagedF32 tab;
  stage_f32(a.tab, a.log2dt, &tab);
  __syncthreads();
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t cl = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
       cl - threadIdx.x < a.ncells; cl += stride) {
    const bool in = cl < a.ncells;
    const int c = in ? (int)cl : 0;
    float Ec;
    int lo, hi;
    bool ok;
    const int WMw = load_cell<F32Form>(a, c, in, Ec, lo, hi, ok);
    if (in && !ok) atomicAdd(&a.hdr[kHdrInvalid], 1u);
    bool hard = false;
    if (ok) {
      switch (WMw) {
        case 1:
          hard = easy_cell<1>(a, tab, c, Ec, lo, hi);
          break;
        case 2:
          hard = easy_cell<2>(a, tab, c, Ec, lo, hi);
          break;
        case 3:
          hard = easy_cell<3>(a, tab, c, Ec, lo, hi);
          break;
        case 4:
          hard = easy_cell<4>(a, tab, c, Ec, lo, hi);
          break;
        case 5:
          hard = easy_cell<5>(a, tab, c, Ec, lo, hi);
          break;
        default:
          hard = easy_cell<6>(a, tab, c, Ec, lo, hi);
          break;
      }
    }
    warp_append(&a.hdr[kHdrHard], a.hard, hard, (uint32_t)c);
  }
}

// The hard cells, one per thread, each with its own width.
__global__ void __launch_bounds__(kThreads)
    ion_step_f32_hard_kernel(const __grid_constant__ StepArgs a) {
  __shared__ StagedF32 tab;
  stage_f32(a.tab, a.log2dt, &tab);
  __syncthreads();
  const unsigned n = *((volatile unsigned*)&a.hdr[kHdrHard]);
  const unsigned stride = gridDim.x * blockDim.x;
  const unsigned n_up = (n + 31u) & ~31u;  // whole warps stay in the loop
  for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n_up; i += stride) {
    const bool in = i < n;
    const int c = in ? (int)a.hard[i] : 0;
    const int lo = in ? a.lo[c] : 0, hi = in ? a.hi[c] : 0;
    const float Ec = in ? static_cast<const float*>(a.E)[c] : 0.0f;
    bool fb = false;
    if (in) {
      switch (hi - lo + 1) {
        case 2:
          fb = cell<F32Form, 2>(a, tab, c, Ec, lo, hi, true);
          break;
        case 3:
          fb = cell<F32Form, 3>(a, tab, c, Ec, lo, hi, true);
          break;
        case 4:
          fb = cell<F32Form, 4>(a, tab, c, Ec, lo, hi, true);
          break;
        case 5:
          fb = cell<F32Form, 5>(a, tab, c, Ec, lo, hi, true);
          break;
        case 6:
          fb = cell<F32Form, 6>(a, tab, c, Ec, lo, hi, true);
          break;
        default:
          break;
      }
    }
    warp_append(&a.hdr[kHdrFallback], a.queue, fb, (uint32_t)c);
  }
}

__global__ void __launch_bounds__(kThreads)
    ion_step_f64_kernel(const __grid_constant__ StepArgs a) {
  __shared__ StagedF64 tab;
  stage_f64(a.tab, a.log2dt, &tab);
  __syncthreads();
  const int64_t cl = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool in = cl < a.ncells;
  const int c = in ? (int)cl : 0;
  double Ec;
  int lo, hi;
  bool ok;
  const int WMw = load_cell<F64Form>(a, c, in, Ec, lo, hi, ok);
  if (in && !ok) atomicAdd(&a.hdr[kHdrInvalid], 1u);
  cell_bucket<F64Form, 1, 6>(WMw, a, tab, c, Ec, lo, hi, ok, false);
}

// ---------------------------------------------------------------------------
// FP64-coefficient pass over the queued cells, one cell per thread.
// ---------------------------------------------------------------------------
template <int W>
__device__ __forceinline__ void fb_cell(const StepArgs& a, const StagedF32& tab,
                                        int c, int lo, int hi) {
  float* __restrict__ N = static_cast<float*>(a.N);
  const FieldF32 f = field_f32(static_cast<const float*>(a.E)[c]);
  double v[W], lam[W];
#pragma unroll
  for (int r = 0; r < W; ++r) {
    v[r] = (double)N[(int64_t)(lo + r) * a.ld + c];
    lam[r] = (r < W - 1 && !a.zero_dt) ? (double)rate_dt_f32(tab, lo + r, f) : 0.0;
  }
  const double dne = dd_update<double, W>(v, lam, W);
  float vf[W];
#pragma unroll
  for (int r = 0; r < W; ++r) {
    vf[r] = __double2float_rn(v[r]);
    N[(int64_t)(lo + r) * a.ld + c] = vf[r];
  }
  int nlo = lo, nhi = hi;
  if ((a.flags & ION_NO_WINDOW_UPDATE) == 0)
    slide_window<float, W>(vf, W, a.Z, (float)a.eps, nlo, nhi);
  const float* G = static_cast<const float*>(a.n_gas);
  const float d = __double2float_rn(dne);
  static_cast<float*>(a.dne)[c] = G ? d * G[c] : d;
  a.lo[c] = (uint8_t)nlo;
  a.hi[c] = (uint8_t)nhi;
}

__global__ void __launch_bounds__(128)
    ion_step_fb_kernel(const __grid_constant__ StepArgs a) {
  __shared__ StagedF32 tab;
  stage_f32(a.tab, a.log2dt, &tab);
  __syncthreads();
  const unsigned n = *((volatile unsigned*)&a.hdr[kHdrFallback]);
  for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += gridDim.x * blockDim.x) {
    const int c = (int)a.queue[i];
    const int lo = a.lo[c], hi = a.hi[c];
    switch (hi - lo + 1) {
      case 2:
        fb_cell<2>(a, tab, c, lo, hi);
        break;
      case 3:
        fb_cell<3>(a, tab, c, lo, hi);
        break;
      case 4:
        fb_cell<4>(a, tab, c, lo, hi);
        break;
      case 5:
        fb_cell<5>(a, tab, c, lo, hi);
        break;
      case 6:
        fb_cell<6>(a, tab, c, lo, hi);
        break;
      default:
        break;
    }
  }
}

}  // namespace

size_t step_workspace_bytes(int64_t ncells, bool f64) {
  if (f64) return kHdrBytes;
  const size_t q = (4 * (size_t)ncells + 255) / 256 * 256;
  return kHdrBytes + 2 * q;
}

void bind_workspace(StepArgs& a, void* ws) {
  char* p = static_cast<char*>(ws);
  a.hdr = reinterpret_cast<uint32_t*>(p);
  const size_t q = (4 * (size_t)a.ncells + 255) / 256 * 256;
  a.queue = reinterpret_cast<uint32_t*>(p + kHdrBytes);
  a.hard = reinterpret_cast<uint32_t*>(p + kHdrBytes + q);
}

namespace {
int resident_blocks_f32() {
  static int blocks = 0;
  if (!blocks) {
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, ion_step_f32_kernel, kThreads, 0) !=
            cudaSuccess ||
        b < 1)
      b = 1;
    blocks = b;
  }
  return blocks;
}
}  // namespace

cudaError_t launch_step_f32(const StepArgs& a, int num_sms, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(a.hdr, 0, kHdrWords * sizeof(uint32_t), s);
  if (e != cudaSuccess) return e;
  if (a.ncells == 0) return cudaSuccess;
  const int64_t tiles = (a.ncells + kThreads - 1) / kThreads;
  const int64_t cap = (int64_t)resident_blocks_f32() * num_sms;
  const int blocks = (int)(tiles < cap ? tiles : cap);
  ion_step_f32_kernel<<<blocks, kThreads, 0, s>>>(a);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  ion_step_f32_hard_kernel<<<4 * num_sms, kThreads, 0, s>>>(a);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const bool need_fb = (a.flags & ION_NO_FP64_FALLBACK) == 0 &&
                       ((a.flags & ION_FORCE_FP64_COEF) != 0 || a.gap > 0.0);
  if (need_fb) {
    ion_step_fb_kernel<<<2 * num_sms, 128, 0, s>>>(a);
    e = cudaGetLastError();
  }
  return e;
}

cudaError_t launch_step_f64(const StepArgs& a, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(a.hdr, 0, kHdrWords * sizeof(uint32_t), s);
  if (e != cudaSuccess) return e;
  if (a.ncells == 0) return cudaSuccess;
  const int blocks = (int)((a.ncells + kThreads - 1) / kThreads);
  ion_step_f64_kernel<<<blocks, kThreads, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace ion
