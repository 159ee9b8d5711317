// step.cu -- the ion_step kernels.
//
//   ion_step_f32_kernel   FP32 SoA, 4 cells per thread (16-byte vector
//                         loads/stores of every window plane when the 4
//                         cells share their window), one window-width bucket
//                         per warp, FP32 rates and coefficients.  Cells with
//                         a nearly degenerate rate pair are left untouched
//                         and queued in the workspace.
//   ion_step_fb_kernel    the queued cells: the same FP32 rates, FP64
//                         Bateman coefficients and propagation, rounded back.
//   ion_step_f64_kernel   the plain FP64 form, 2 cells per thread.
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

// Append the flagged cells of a warp to the FP64 queue with one atomic per
// warp.  Every lane of the warp calls this.
template <int CPT>
__device__ __forceinline__ void queue_append(const StepArgs& a,
                                             const bool (&fb)[CPT], int c0) {
  int nf = 0;
#pragma unroll
  for (int j = 0; j < CPT; ++j) nf += fb[j] ? 1 : 0;
  if (!__ballot_sync(kFull, nf > 0)) return;
  const int lane = threadIdx.x & 31;
  int x = nf;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(kFull, x, o);
    x += lane >= o ? y : 0;
  }
  const int total = __shfl_sync(kFull, x, 31);
  unsigned base = 0;
  if (lane == 31) base = atomicAdd(&a.hdr[kHdrFallback], (unsigned)total);
  base = __shfl_sync(kFull, base, 31);
  unsigned pos = base + (unsigned)(x - nf);
#pragma unroll
  for (int j = 0; j < CPT; ++j)
    if (fb[j]) a.queue[pos++] = (uint32_t)(c0 + j);
}

template <typename T>
struct Vec16;
template <>
struct Vec16<float> {
  using type = float4;
  static constexpr int n = 4;
};
template <>
struct Vec16<double> {
  using type = double2;
  static constexpr int n = 2;
};

template <typename T>
__device__ __forceinline__ void unpack(const typename Vec16<T>::type& x,
                                       T (&o)[Vec16<T>::n]);
template <>
__device__ __forceinline__ void unpack<float>(const float4& x, float (&o)[4]) {
  o[0] = x.x;
  o[1] = x.y;
  o[2] = x.z;
  o[3] = x.w;
}
template <>
__device__ __forceinline__ void unpack<double>(const double2& x,
                                               double (&o)[2]) {
  o[0] = x.x;
  o[1] = x.y;
}
__device__ __forceinline__ float4 pack(const float (&o)[4]) {
  return make_float4(o[0], o[1], o[2], o[3]);
}
__device__ __forceinline__ double2 pack(const double (&o)[2]) {
  return make_double2(o[0], o[1]);
}

// Per-precision hooks of the generic cell loop.
struct F32Form {
  using T = float;
  using Staged = StagedF32;
  struct Field {
    FieldF32 f;
  };
  __device__ static Field field(float E) { return {field_f32(E)}; }
  __device__ static float rate(const StagedF32& t, int k, const Field& f) {
    return rate_dt_f32(t, k, f.f);
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

// ---------------------------------------------------------------------------
// The CPT cells c0..c0+CPT-1 of one thread, window width bound WM.
// lo/hi are the cells' windows (in), nlo/nhi the windows after the slide
// (out).  fb[j] is set for cells left to the FP64 queue.
// ---------------------------------------------------------------------------
template <class F, int WM, int CPT>
__device__ __forceinline__ void cells(const StepArgs& a,
                                      const typename F::Staged& tab, int c0,
                                      bool full, const typename F::T (&Ev)[CPT],
                                      const int (&lo)[CPT], const int (&hi)[CPT],
                                      const bool (&ok)[CPT], int (&nlo)[CPT],
                                      int (&nhi)[CPT], bool (&fb)[CPT],
                                      typename F::T (&dne)[CPT], bool allow_fb) {
  using T = typename F::T;
  using V = Vec16<T>;
  T* __restrict__ N = static_cast<T*>(a.N);
  const int64_t ld = a.ld;
  int w[CPT];
  bool uni = full;
#pragma unroll
  for (int j = 0; j < CPT; ++j) {
    w[j] = ok[j] ? hi[j] - lo[j] + 1 : 0;
    uni = uni && ok[j] && lo[j] == lo[0] && w[j] == w[0];
  }

  T v[CPT][WM];
#pragma unroll
  for (int j = 0; j < CPT; ++j)
#pragma unroll
    for (int r = 0; r < WM; ++r) v[j][r] = T(0);
  if (uni) {
#pragma unroll
    for (int r = 0; r < WM; ++r)
      if (r < w[0]) {
        T o[CPT];
        unpack<T>(__ldcs(reinterpret_cast<const typename V::type*>(
                      N + (int64_t)(lo[0] + r) * ld + c0)),
                  o);
#pragma unroll
        for (int j = 0; j < CPT; ++j) v[j][r] = o[j];
      }
  } else {
#pragma unroll
    for (int j = 0; j < CPT; ++j)
#pragma unroll
      for (int r = 0; r < WM; ++r)
        if (r < w[j]) v[j][r] = __ldcs(N + (int64_t)(lo[j] + r) * ld + c0 + j);
  }

  const bool force64 = allow_fb && (a.flags & ION_FORCE_FP64_COEF) != 0;
  const bool no_fb = !allow_fb || (a.flags & ION_NO_FP64_FALLBACK) != 0;
  const bool upd = (a.flags & ION_NO_WINDOW_UPDATE) == 0;
  const T gap = (T)a.gap;
  const T eps = (T)a.eps;
  // One copy of the coefficient code serves the CPT cells: cell j's values
  // are selected into registers, updated, and selected back.
#pragma unroll 1
  for (int j = 0; j < CPT; ++j) {
    T vj[WM];
    T Ej = Ev[0];
    int loj = lo[0], hij = hi[0], wj = w[0];
#pragma unroll
    for (int r = 0; r < WM; ++r) vj[r] = v[0][r];
#pragma unroll
    for (int jj = 1; jj < CPT; ++jj)
      if (j == jj) {
        Ej = Ev[jj];
        loj = lo[jj];
        hij = hi[jj];
        wj = w[jj];
#pragma unroll
        for (int r = 0; r < WM; ++r) vj[r] = v[jj][r];
      }
    bool fbj = false;
    T dnej = T(0);
    int nloj = loj, nhij = hij;
    if (wj >= 2) {
      const typename F::Field f = F::field(Ej);
      T lam[WM];
#pragma unroll
      for (int r = 0; r < WM; ++r)
        lam[r] = (r < wj - 1 && !a.zero_dt) ? F::rate(tab, loj + r, f) : T(0);
      fbj = !no_fb &&
            (force64 || (gap > T(0) && near_degenerate<T, WM>(lam, wj, gap)));
      if (!fbj) {
        dnej = window_update<T, WM>(vj, lam, wj);
        if (upd) slide_window<T, WM>(vj, wj, a.Z, eps, nloj, nhij);
      }
    }
#pragma unroll
    for (int jj = 0; jj < CPT; ++jj)
      if (j == jj) {
        fb[jj] = fbj;
        dne[jj] = dnej;
        nlo[jj] = nloj;
        nhi[jj] = nhij;
#pragma unroll
        for (int r = 0; r < WM; ++r) v[jj][r] = vj[r];
      }
  }

  bool anyfb = false;
#pragma unroll
  for (int j = 0; j < CPT; ++j) anyfb = anyfb || fb[j];
  if (uni && !anyfb) {
#pragma unroll
    for (int r = 0; r < WM; ++r)
      if (r < w[0]) {
        T o[CPT];
#pragma unroll
        for (int j = 0; j < CPT; ++j) o[j] = v[j][r];
        __stcs(reinterpret_cast<typename V::type*>(N + (int64_t)(lo[0] + r) * ld + c0),
               pack(o));
      }
  } else {
#pragma unroll
    for (int j = 0; j < CPT; ++j) {
      if (!ok[j] || fb[j]) continue;
#pragma unroll
      for (int r = 0; r < WM; ++r)
        if (r < w[j]) __stcs(N + (int64_t)(lo[j] + r) * ld + c0 + j, v[j][r]);
    }
  }
}

// Loads the per-cell inputs of a thread, runs the warp's width bucket, and
// stores dne and the windows.  Shared by the FP32 and FP64 kernels.
template <class F, int CPT>
__device__ __forceinline__ void step_thread(const StepArgs& a,
                                            const typename F::Staged& tab,
                                            bool allow_fb) {
  using T = typename F::T;
  using V = Vec16<T>;
  const int64_t c0l = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * CPT;
  const int c0 = (int)(c0l < a.ncells ? c0l : a.ncells);
  const bool full = c0l + CPT <= a.ncells;
  const T* __restrict__ E = static_cast<const T*>(a.E);

  T Ev[CPT];
  int lo[CPT], hi[CPT];
  bool ok[CPT];
  if (full) {
    unpack<T>(__ldcs(reinterpret_cast<const typename V::type*>(E + c0)), Ev);
    if constexpr (CPT == 4) {
      const uint32_t l4 = __ldcs(reinterpret_cast<const unsigned int*>(a.lo + c0));
      const uint32_t h4 = __ldcs(reinterpret_cast<const unsigned int*>(a.hi + c0));
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        lo[j] = (l4 >> (8 * j)) & 0xff;
        hi[j] = (h4 >> (8 * j)) & 0xff;
      }
    } else {
      const uint32_t l2 = __ldcs(reinterpret_cast<const unsigned short*>(a.lo + c0));
      const uint32_t h2 = __ldcs(reinterpret_cast<const unsigned short*>(a.hi + c0));
#pragma unroll
      for (int j = 0; j < CPT; ++j) {
        lo[j] = (l2 >> (8 * j)) & 0xff;
        hi[j] = (h2 >> (8 * j)) & 0xff;
      }
    }
  } else {
#pragma unroll
    for (int j = 0; j < CPT; ++j) {
      const bool in = c0l + j < a.ncells;
      Ev[j] = in ? E[c0 + j] : T(0);
      lo[j] = in ? a.lo[c0 + j] : 1;
      hi[j] = in ? a.hi[c0 + j] : 0;  // lo > hi: marks "no cell"
    }
  }
  int wmax = 0, nbad = 0;
#pragma unroll
  for (int j = 0; j < CPT; ++j) {
    const bool in = c0l + j < a.ncells;
    ok[j] = in && window_ok(lo[j], hi[j], a.Z);
    nbad += (in && !ok[j]) ? 1 : 0;
    wmax = ok[j] ? max(wmax, hi[j] - lo[j] + 1) : wmax;
  }
  if (nbad) atomicAdd(&a.hdr[kHdrInvalid], (unsigned)nbad);
  const int WMw = __reduce_max_sync(kFull, wmax);

  int nlo[CPT], nhi[CPT];
  bool fb[CPT];
  T dne[CPT];
#pragma unroll
  for (int j = 0; j < CPT; ++j) {
    nlo[j] = lo[j];
    nhi[j] = hi[j];
    fb[j] = false;
    dne[j] = T(0);
  }
  switch (WMw) {
    case 0:
    case 1:
      break;  // nothing moves; dne = 0
    case 2:
      cells<F, 2, CPT>(a, tab, c0, full, Ev, lo, hi, ok, nlo, nhi, fb, dne, allow_fb);
      break;
    case 3:
      cells<F, 3, CPT>(a, tab, c0, full, Ev, lo, hi, ok, nlo, nhi, fb, dne, allow_fb);
      break;
    case 4:
      cells<F, 4, CPT>(a, tab, c0, full, Ev, lo, hi, ok, nlo, nhi, fb, dne, allow_fb);
      break;
    case 5:
      cells<F, 5, CPT>(a, tab, c0, full, Ev, lo, hi, ok, nlo, nhi, fb, dne, allow_fb);
      break;
    default:
      cells<F, 6, CPT>(a, tab, c0, full, Ev, lo, hi, ok, nlo, nhi, fb, dne, allow_fb);
      break;
  }

  // dne (x n_gas) and the windows of the cells this kernel finished
  bool all = full;
#pragma unroll
  for (int j = 0; j < CPT; ++j) all = all && ok[j] && !fb[j];
  T* __restrict__ D = static_cast<T*>(a.dne);
  const T* __restrict__ G = static_cast<const T*>(a.n_gas);
  if (all) {
    if (G) {
      T g[CPT];
      unpack<T>(__ldcs(reinterpret_cast<const typename V::type*>(G + c0)), g);
#pragma unroll
      for (int j = 0; j < CPT; ++j) dne[j] *= g[j];
    }
    __stcs(reinterpret_cast<typename V::type*>(D + c0), pack(dne));
    uint32_t l = 0, h = 0;
#pragma unroll
    for (int j = 0; j < CPT; ++j) {
      l |= (uint32_t)nlo[j] << (8 * j);
      h |= (uint32_t)nhi[j] << (8 * j);
    }
    if constexpr (CPT == 4) {
      __stcs(reinterpret_cast<unsigned int*>(a.lo + c0), l);
      __stcs(reinterpret_cast<unsigned int*>(a.hi + c0), h);
    } else {
      __stcs(reinterpret_cast<unsigned short*>(a.lo + c0), (unsigned short)l);
      __stcs(reinterpret_cast<unsigned short*>(a.hi + c0), (unsigned short)h);
    }
  } else {
#pragma unroll
    for (int j = 0; j < CPT; ++j) {
      if (!ok[j] || fb[j]) continue;
      D[c0 + j] = G ? dne[j] * G[c0 + j] : dne[j];
      a.lo[c0 + j] = (uint8_t)nlo[j];
      a.hi[c0 + j] = (uint8_t)nhi[j];
    }
  }
  if (allow_fb) queue_append<CPT>(a, fb, c0);
}

__global__ void __launch_bounds__(kThreads, 2)
    ion_step_f32_kernel(const __grid_constant__ StepArgs a) {
  __shared__ StagedF32 tab;
  stage_f32(a.tab, a.log2dt, &tab);
  __syncthreads();
  step_thread<F32Form, 4>(a, tab, true);
}

__global__ void __launch_bounds__(kThreads)
    ion_step_f64_kernel(const __grid_constant__ StepArgs a) {
  __shared__ StagedF64 tab;
  stage_f64(a.tab, a.log2dt, &tab);
  __syncthreads();
  step_thread<F64Form, 2>(a, tab, false);
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
  const double dne = window_update<double, W>(v, lam, W);
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

cudaError_t launch_step_f32(const StepArgs& a, int num_sms, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(a.hdr, 0, 2 * sizeof(uint32_t), s);
  if (e != cudaSuccess) return e;
  if (a.ncells == 0) return cudaSuccess;
  const int64_t per_block = (int64_t)kThreads * 4;
  const int blocks = (int)((a.ncells + per_block - 1) / per_block);
  ion_step_f32_kernel<<<blocks, kThreads, 0, s>>>(a);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const bool need_fb = (a.flags & ION_NO_FP64_FALLBACK) == 0 &&
                       ((a.flags & ION_FORCE_FP64_COEF) != 0 || a.gap > 0.0);
  if (need_fb) {
    ion_step_fb_kernel<<<2 * num_sms, 128, 0, s>>>(a);
    e = cudaGetLastError();
  }
  return e;
}

cudaError_t launch_step_f64(const StepArgs& a, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(a.hdr, 0, 2 * sizeof(uint32_t), s);
  if (e != cudaSuccess) return e;
  if (a.ncells == 0) return cudaSuccess;
  const int64_t per_block = (int64_t)kThreads * 2;
  const int blocks = (int)((a.ncells + per_block - 1) / per_block);
  ion_step_f64_kernel<<<blocks, kThreads, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace ion
