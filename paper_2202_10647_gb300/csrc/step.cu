// step.cu -- the ion_step kernels.
//
// FP32 form (ION_F32), three kernels on the caller's stream:
//   ion_step_f32_kernel  persistent; every warp walks its own sequence of
//       32-cell chunks through a 4-stage ring in shared memory.  cp.async
//       brings |E|, k_lo and k_hi in two chunks ahead and each lane's own
//       window planes one chunk ahead, so the loads in flight cost no
//       registers and the traffic is exactly the cells' windows.  A cell
//       whose rates all have W dt <= 0.025 is finished here (at most four
//       Taylor terms of exp(dt A)).  The others ("stiff" cells) write the
//       inputs already loaded into a record queue (coalesced, warp by warp):
//       in a laser field |E| swings from zero to its peak every few cells, so
//       most warps near the pulse hold a few stiff cells, and finishing them
//       in place would make every such warp run the longest path of its
//       lanes and would size this kernel's registers for it.
//   ion_step_f32_stiff_kernel  the records, one per thread in full warps:
//       Taylor form up to W dt <= 1, divided-difference (Bateman) form above.
//       Cells with a nearly degenerate rate pair are left untouched and
//       queued for
//   ion_step_fb_kernel   FP32 rates, FP64 Bateman coefficients and
//       propagation, rounded back to FP32.
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
constexpr int kThreads = 256;       // FP64 kernel
constexpr int kWarps = 4;           // warps per block of the FP32 kernel
constexpr int kStages = 4;          // chunks in the per-warp ring
constexpr float kLamEasy = 0.025f;  // 2 kLamEasy <= kThrF32[4]: 4 terms
constexpr int kEasyTerms = 4;

__device__ __forceinline__ bool window_ok(int lo, int hi, int Z) {
  return lo <= hi && hi <= Z && hi - lo + 1 <= ION_MAX_WINDOW;
}

// ---------------------------------------------------------------------------
// cp.async (global -> shared, 4 bytes, completion tracked per thread in
// commit groups; no spin loop is involved).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
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
// Full update of one cell whose window populations v[0..w-1] are loaded
// (w <= WM): rates, Taylor or Bateman form, window slide, stores.  Returns
// true (and stores nothing) if the cell goes to the FP64 queue.
// ---------------------------------------------------------------------------
template <class F, int WM>
__device__ __forceinline__ bool finish_cell(const StepArgs& a,
                                            const typename F::Staged& tab, int c,
                                            typename F::T Ec, int lo, int hi,
                                            typename F::T (&v)[WM],
                                            bool allow_fb) {
  using T = typename F::T;
  T* __restrict__ N = static_cast<T*>(a.N);
  const int64_t ld = a.ld;
  const int w = hi - lo + 1;
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

// The same, loading the window from global memory; W bounds the width.
template <class F, int W>
__device__ __forceinline__ bool global_cell(const StepArgs& a,
                                            const typename F::Staged& tab, int c,
                                            typename F::T Ec, int lo, int hi,
                                            bool allow_fb) {
  using T = typename F::T;
  const T* __restrict__ N = static_cast<const T*>(a.N);
  T v[W];
#pragma unroll
  for (int r = 0; r < W; ++r)
    v[r] = r < hi - lo + 1 ? __ldcs(N + (int64_t)(lo + r) * a.ld + c) : T(0);
  return finish_cell<F, W>(a, tab, c, Ec, lo, hi, v, allow_fb);
}

// Dispatch on a width known to be 1..6 (per-lane switch).
template <class F>
__device__ __forceinline__ bool global_cell_any(const StepArgs& a,
                                                const typename F::Staged& tab,
                                                int c, typename F::T Ec, int lo,
                                                int hi, bool allow_fb) {
  switch (hi - lo + 1) {
    case 1:
      return global_cell<F, 1>(a, tab, c, Ec, lo, hi, allow_fb);
    case 2:
      return global_cell<F, 2>(a, tab, c, Ec, lo, hi, allow_fb);
    case 3:
      return global_cell<F, 3>(a, tab, c, Ec, lo, hi, allow_fb);
    case 4:
      return global_cell<F, 4>(a, tab, c, Ec, lo, hi, allow_fb);
    case 5:
      return global_cell<F, 5>(a, tab, c, Ec, lo, hi, allow_fb);
    default:
      return global_cell<F, 6>(a, tab, c, Ec, lo, hi, allow_fb);
  }
}

// ---------------------------------------------------------------------------
// FP32 streaming kernel.
// ---------------------------------------------------------------------------
struct ChunkStage {
  float E[32];
  uint8_t lo[32];
  uint8_t hi[32];
  float P[ION_MAX_WINDOW][32];  // P[r][lane] = N[lo + r] of the lane's cell
};

// Appends the record of a stiff cell (one atomic per warp).  Every lane of
// the warp calls this; `take` lanes pass their cell's inputs.
__device__ __forceinline__ void append_record(const StepArgs& a, bool take, int c,
                                              float Ec, int lo, int hi,
                                              const float* v, int vstride) {
  const unsigned m = __ballot_sync(kFull, take);
  if (!m) return;
  const int lane = threadIdx.x & 31;
  unsigned base = 0;
  if (lane == 0) base = atomicAdd(&a.hdr[kHdrStiff], (unsigned)__popc(m));
  base = __shfl_sync(kFull, base, 0);
  if (take) {
    const unsigned i = base + __popc(m & ((1u << lane) - 1u));
    a.rec_c[i] = (uint32_t)c;
    a.rec_E[i] = Ec;
    a.rec_lohi[i] = (uint16_t)(lo | (hi << 8));
    const int w = hi - lo + 1;
    for (int r = 0; r < w; ++r) a.rec_V[(int64_t)r * a.rec_cap + i] = v[r * vstride];
  }
}

// Easy path of a lane's cell in a staged chunk: finishes it if every
// W dt <= kLamEasy and returns false, else returns true untouched.  Written
// for lanes that mostly agree: every window rate takes the plain FP32
// exponent, the float-float refinement runs only for rates above 2^-12, and
// the Taylor series runs the warp's largest term count (extra terms only add
// accuracy).
template <int WM>
__device__ __forceinline__ bool easy_cell(const StepArgs& a, const StagedF32& tab,
                                          const ChunkStage& st, int lane, int c,
                                          float Ec, int lo, int hi, bool ok) {
  // every lane of the warp calls this; lanes with !ok only take part in the
  // warp reduction
  const int w = ok ? hi - lo + 1 : 0;
  lo = ok ? lo : 0;
  float v[WM];
#pragma unroll
  for (int r = 0; r < WM; ++r) v[r] = st.P[r][lane];  // r >= w: ignored
  float dne = 0.0f;
  int nlo = lo, nhi = hi;
  bool stiff = false;
  if constexpr (WM >= 2) {
    const FieldF32 f = field_f32(Ec);
    const bool live = w >= 2 && !f.zero && !a.zero_dt;
    float lam[WM];
    float y0[WM];
    bool need_precise = false;
#pragma unroll
    for (int r = 0; r < WM - 1; ++r) {
      const float4 h = tab.hi[min(lo + r, ION_MAX_Z)];
      const float q = h.z * f.rE;
      y0[r] = fmaf(-h.y, f.lg, h.x) - q;
      const bool on = live && r < w - 1 && q <= (float)kCutoffLog2;
      lam[r] = on ? ex2_approx(y0[r]) : 0.0f;
      need_precise |= on && y0[r] >= -12.0f;
    }
    lam[WM - 1] = 0.0f;
    if (need_precise) {
#pragma unroll
      for (int r = 0; r < WM - 1; ++r)
        if (lam[r] != 0.0f && y0[r] >= -12.0f) lam[r] = rate_dt_f32(tab, lo + r, f);
    }
    float lmax = 0.0f;
#pragma unroll
    for (int r = 0; r < WM - 1; ++r) lmax = fmaxf(lmax, lam[r]);
    stiff = lmax > kLamEasy;
    // terms of exp(dt A) v: R = number of thresholds below 2 lmax (<= 4)
    const float x = stiff ? 0.0f : 2.0f * lmax;
    int R = 0;
#pragma unroll
    for (int i = 0; i < kEasyTerms; ++i) R += x > kThrF32[i] ? 1 : 0;
    const int Rw = __reduce_max_sync(kFull, R);
    if (!stiff && w >= 2) {
      float t[WM], inc[WM];
#pragma unroll
      for (int i = 0; i < WM; ++i) {
        t[i] = i < w ? v[i] : 0.0f;
        inc[i] = 0.0f;
      }
#pragma unroll
      for (int k = 1; k <= kEasyTerms; ++k) {
        if (k > Rw) break;
        const float rk = 1.0f / k;
#pragma unroll
        for (int i = WM - 1; i >= 0; --i) {
          const float gain = i > 0 ? lam[i - 1] * t[i - 1] : 0.0f;
          t[i] = (gain - lam[i] * t[i]) * rk;
          inc[i] += t[i];
        }
      }
      float cum = 0.0f;
#pragma unroll
      for (int r = 0; r < WM - 1; ++r) {
        if (r < w - 1) {
          cum -= inc[r];  // population that left states <= r
          dne += cum;
        }
      }
#pragma unroll
      for (int r = 0; r < WM; ++r) v[r] += inc[r];
      if ((a.flags & ION_NO_WINDOW_UPDATE) == 0 && v[0] < (float)a.eps && hi < a.Z)
        slide_window<float, WM>(v, w, a.Z, (float)a.eps, nlo, nhi);
      float* p = static_cast<float*>(a.N) + (int64_t)lo * a.ld + c;
#pragma unroll
      for (int r = 0; r < WM; ++r) {
        if (r < w) __stcs(p, v[r]);
        p += a.ld;
      }
    }
  }
  if (stiff || !ok) return stiff;
  const float* __restrict__ G = static_cast<const float*>(a.n_gas);
  __stcs(static_cast<float*>(a.dne) + c, G ? dne * G[c] : dne);
  if (nlo != lo) {
    a.lo[c] = (uint8_t)nlo;
    a.hi[c] = (uint8_t)nhi;
  }
  return false;
}

__global__ void __launch_bounds__(kWarps * 32, 8)
    ion_step_f32_kernel(const __grid_constant__ StepArgs a) {
  __shared__ StagedF32 tab;
  __shared__ ChunkStage ring[kWarps][kStages];
  stage_f32(a.tab, a.log2dt, &tab);
  {
    // plane slots past a cell's window are read (and ignored) by the easy
    // path; keep them finite
    float* z = reinterpret_cast<float*>(&ring[0][0]);
    for (int i = threadIdx.x; i < (int)(sizeof(ring) / sizeof(float)); i += blockDim.x)
      z[i] = 0.0f;
  }
  __syncthreads();

  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  ChunkStage* S = ring[wib];
  const int gw = blockIdx.x * kWarps + wib;
  const int TW = gridDim.x * kWarps;
  const int nfull = a.ncells >> 5;
  const int K = gw < nfull ? (nfull - 1 - gw) / TW + 1 : 0;
  const float* __restrict__ E = static_cast<const float*>(a.E);
  const float* __restrict__ N = static_cast<const float*>(a.N);
  const int64_t ld = a.ld;

  // |E|, k_lo, k_hi of the warp's chunk k into its stage (one commit group).
  auto issue_front = [&](int k) {
    if (k < K) {
      const int c0 = (gw + k * TW) << 5;
      ChunkStage& st = S[k % kStages];
      cp_async4(&st.E[lane], E + c0 + lane);
      if (lane < 8)
        cp_async4(&st.lo[4 * lane], a.lo + c0 + 4 * lane);
      else if (lane < 16)
        cp_async4(&st.hi[4 * (lane - 8)], a.hi + c0 + 4 * (lane - 8));
    }
    cp_async_commit();
  };
  // the window planes of the lane's cell of chunk k (one commit group).
  auto issue_planes = [&](int k) {
    if (k < K) {
      const int c = ((gw + k * TW) << 5) + lane;
      ChunkStage& st = S[k % kStages];
      const int lo = st.lo[lane], hi = st.hi[lane];
      const int w = window_ok(lo, hi, a.Z) ? hi - lo + 1 : 0;
      const float* p = N + (int64_t)lo * ld + c;
      for (int r = 0; r < w; ++r) {
        cp_async4(&st.P[r][lane], p);
        p += ld;
      }
    }
    cp_async_commit();
  };

  issue_front(0);
  issue_front(1);
  cp_async_wait<1>();  // front(0)
  __syncwarp();
  issue_planes(0);
  for (int k = 0; k < K; ++k) {
    issue_front(k + 2);
    cp_async_wait<2>();  // front(k+1): pending are planes(k), front(k+2)
    __syncwarp();
    issue_planes(k + 1);
    cp_async_wait<2>();  // planes(k): pending are front(k+2), planes(k+1)
    __syncwarp();

    const ChunkStage& st = S[k % kStages];
    const int c = ((gw + k * TW) << 5) + lane;
    const float Ec = st.E[lane];
    const int lo = st.lo[lane], hi = st.hi[lane];
    const bool ok = window_ok(lo, hi, a.Z);
    if (!ok) atomicAdd(&a.hdr[kHdrInvalid], 1u);
    const int WMw = __reduce_max_sync(kFull, ok ? hi - lo + 1 : 0);
    bool stiff;
    if (WMw <= 1)
      stiff = easy_cell<1>(a, tab, st, lane, c, Ec, lo, hi, ok);
    else if (WMw == 2)
      stiff = easy_cell<2>(a, tab, st, lane, c, Ec, lo, hi, ok);
    else if (WMw <= 4)
      stiff = easy_cell<4>(a, tab, st, lane, c, Ec, lo, hi, ok);
    else
      stiff = easy_cell<6>(a, tab, st, lane, c, Ec, lo, hi, ok);
    append_record(a, stiff, c, Ec, lo, hi, &st.P[0][lane], 32);
    __syncwarp();
  }
  cp_async_wait<0>();

  // the last, partial chunk (ncells % 32 cells): every valid cell becomes a
  // record for the stiff kernel, which runs the full path
  const int tail = a.ncells & 31;
  if (tail && gw == TW - 1) {
    const int c = (nfull << 5) + lane;
    bool take = false;
    float Ec = 0.0f, v[ION_MAX_WINDOW];
    int lo = 0, hi = 0;
    if (lane < tail) {
      Ec = E[c];
      lo = a.lo[c];
      hi = a.hi[c];
      take = window_ok(lo, hi, a.Z);
      if (!take) atomicAdd(&a.hdr[kHdrInvalid], 1u);
      const float* p = N + (int64_t)lo * ld + c;
#pragma unroll
      for (int r = 0; r < ION_MAX_WINDOW; ++r) {
        v[r] = (take && r < hi - lo + 1) ? p[0] : 0.0f;
        p += ld;
      }
    }
    append_record(a, take, c, Ec, lo, hi, v, 1);
  }
}

// The stiff-cell records, one per thread.
template <int W>
__device__ __forceinline__ bool record_cell(const StepArgs& a, const StagedF32& tab,
                                            unsigned i, int c, float Ec, int lo,
                                            int hi) {
  float v[W];
#pragma unroll
  for (int r = 0; r < W; ++r) v[r] = __ldcs(a.rec_V + (int64_t)r * a.rec_cap + i);
  return finish_cell<F32Form, W>(a, tab, c, Ec, lo, hi, v, true);
}

__global__ void __launch_bounds__(256)
    ion_step_f32_stiff_kernel(const __grid_constant__ StepArgs a) {
  __shared__ StagedF32 tab;
  stage_f32(a.tab, a.log2dt, &tab);
  __syncthreads();
  const unsigned n = *((volatile unsigned*)&a.hdr[kHdrStiff]);
  const unsigned stride = gridDim.x * blockDim.x;
  const unsigned n_up = (n + 31u) & ~31u;  // whole warps stay in the loop
  for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n_up; i += stride) {
    bool fb = false;
    int c = 0;
    if (i < n) {
      c = (int)__ldcs(a.rec_c + i);
      const float Ec = __ldcs(a.rec_E + i);
      const unsigned lh = __ldcs(a.rec_lohi + i);
      const int lo = lh & 0xff, hi = lh >> 8;
      switch (hi - lo + 1) {
        case 1:
          fb = record_cell<1>(a, tab, i, c, Ec, lo, hi);
          break;
        case 2:
          fb = record_cell<2>(a, tab, i, c, Ec, lo, hi);
          break;
        case 3:
          fb = record_cell<3>(a, tab, i, c, Ec, lo, hi);
          break;
        case 4:
          fb = record_cell<4>(a, tab, i, c, Ec, lo, hi);
          break;
        case 5:
          fb = record_cell<5>(a, tab, i, c, Ec, lo, hi);
          break;
        default:
          fb = record_cell<6>(a, tab, i, c, Ec, lo, hi);
          break;
      }
    }
    warp_append(&a.hdr[kHdrFallback], a.queue, fb, (uint32_t)c);
  }
}

// ---------------------------------------------------------------------------
// Plain FP64 form: one cell per thread, all paths inline.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads)
    ion_step_f64_kernel(const __grid_constant__ StepArgs a) {
  __shared__ StagedF64 tab;
  stage_f64(a.tab, a.log2dt, &tab);
  __syncthreads();
  const int64_t cl = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (cl >= a.ncells) return;
  const int c = (int)cl;
  const double Ec = static_cast<const double*>(a.E)[c];
  const int lo = a.lo[c], hi = a.hi[c];
  if (!window_ok(lo, hi, a.Z)) {
    atomicAdd(&a.hdr[kHdrInvalid], 1u);
    return;
  }
  global_cell_any<F64Form>(a, tab, c, Ec, lo, hi, false);
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

int resident_blocks_f32() {
  static int blocks = 0;
  if (!blocks) {
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, ion_step_f32_kernel, kWarps * 32,
                                                      0) != cudaSuccess ||
        b < 1)
      b = 1;
    blocks = b;
  }
  return blocks;
}

}  // namespace

// Workspace: header | FP64 queue (4 B/cell) | stiff records: cell index
// (4 B), |E| (4 B), lo|hi (2 B), window (6 x 4 B) per cell.
namespace {
size_t round256(size_t x) { return (x + 255) / 256 * 256; }
}  // namespace

size_t step_workspace_bytes(int64_t ncells, bool f64) {
  if (f64) return kHdrBytes;
  const size_t n = (size_t)ncells;
  return kHdrBytes + round256(4 * n) + round256(4 * n) + round256(4 * n) +
         round256(2 * n) + round256(4 * n * ION_MAX_WINDOW);
}

void bind_workspace(StepArgs& a, void* ws) {
  char* p = static_cast<char*>(ws);
  const size_t n = (size_t)a.ncells;
  a.hdr = reinterpret_cast<uint32_t*>(p);
  p += kHdrBytes;
  a.queue = reinterpret_cast<uint32_t*>(p);
  p += round256(4 * n);
  a.rec_c = reinterpret_cast<uint32_t*>(p);
  p += round256(4 * n);
  a.rec_E = reinterpret_cast<float*>(p);
  p += round256(4 * n);
  a.rec_lohi = reinterpret_cast<uint16_t*>(p);
  p += round256(2 * n);
  a.rec_V = reinterpret_cast<float*>(p);
  a.rec_cap = (int64_t)n;
}

cudaError_t launch_step_f32(const StepArgs& a, int num_sms, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(a.hdr, 0, kHdrWords * sizeof(uint32_t), s);
  if (e != cudaSuccess) return e;
  if (a.ncells == 0) return cudaSuccess;
  const int64_t chunks = ((int64_t)a.ncells + 31) / 32;
  const int64_t need = (chunks + kWarps - 1) / kWarps;
  const int64_t cap = (int64_t)resident_blocks_f32() * num_sms;
  const int blocks = (int)(need < cap ? need : cap);
  ion_step_f32_kernel<<<blocks, kWarps * 32, 0, s>>>(a);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  ion_step_f32_stiff_kernel<<<4 * num_sms, 256, 0, s>>>(a);
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
