// ion_cell.cuh -- per-cell device code shared by the FP32 and FP64 step
// kernels: the full update of one cell (rates, Taylor or Bateman form, window
// slide, stores), queue appends and cp.async helpers.
#pragma once

#include <cstdint>

#include "ion_device.cuh"
#include "ion_step.cuh"

namespace ion {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ bool window_ok(int lo, int hi, int Z) {
  return lo <= hi && hi <= Z && hi - lo + 1 <= ION_MAX_WINDOW;
}

// ---------------------------------------------------------------------------
// cp.async (global -> shared; completion tracked per thread in commit
// groups, no spin loop involved).
// ---------------------------------------------------------------------------
template <int BYTES>
__device__ __forceinline__ void cp_async(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  if constexpr (BYTES == 16)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem)
                 : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(s), "l"(gmem),
                 "n"(BYTES)
                 : "memory");
}
// The same with the shared-memory destination as a 32-bit shared address.
template <int BYTES>
__device__ __forceinline__ void cp_async_s(uint32_t s, const void* gmem) {
  if constexpr (BYTES == 16)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem)
                 : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(s), "l"(gmem),
                 "n"(BYTES)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// A running sum in twice the working precision (Knuth's TwoSum): the value
// is s + e.  Used for the change of a window's total population, whose size
// is that of the rounding of the stored populations.
template <typename T>
struct ExactSum {
  T s = T(0), e = T(0);
  __device__ __forceinline__ void add(T x) {
    const T t = s + x;
    const T z = t - s;
    e += (s - (t - z)) + (x - z);
    s = t;
  }
  __device__ __forceinline__ T value() const { return s + e; }
};

// The bits of |x| as a float, for a running maximum over non-negative
// floats (which order like their bits; a NaN is larger than every number).
template <typename T>
__device__ __forceinline__ uint32_t abs_bits(T x) {
  return __float_as_uint(fabsf((float)x));
}

// The largest of the warp's bits into *word (every lane calls this).
__device__ __forceinline__ void warp_max_into(uint32_t* word, uint32_t bits) {
  const unsigned m = __reduce_max_sync(0xffffffffu, bits);
  if ((threadIdx.x & 31) == 0 && m) atomicMax(word, m);
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
  using Field = FieldF64;
  __device__ static Field field(double E) { return field_f64(E); }
  __device__ static double rate(const StagedF64& t, int k, const Field& f) {
    return rate_dt_f64(t, k, f);
  }
};

// Warp-aggregated append of (value, tag) for the lanes with `take` set: one
// atomic per warp.  Every lane of the warp calls this.
__device__ __forceinline__ void warp_append(uint32_t* counter, uint32_t* queue,
                                            uint8_t* tags, bool take, uint32_t value,
                                            uint8_t tag) {
  const unsigned m = __ballot_sync(kFull, take);
  if (!m) return;
  const int lane = threadIdx.x & 31;
  unsigned base = 0;
  if (lane == 0) base = atomicAdd(counter, (unsigned)__popc(m));
  base = __shfl_sync(kFull, base, 0);
  if (take) {
    const unsigned i = base + __popc(m & ((1u << lane) - 1u));
    queue[i] = value;
    if (tags) tags[i] = tag;
  }
}

// Appends the record of a stiff cell (one atomic per warp and width class).
// Every lane of the warp calls this; `take` lanes pass their cell's inputs.
// Records of windows of at most kRecNarrow states fill the record arrays
// from the front, wider ones from the back, so that the stiff kernel's
// warps see one class each and run the shorter divided-difference table
// wherever they can.
__device__ __forceinline__ void append_record(const Scratch& S, bool take, int job,
                                              int c, float Ec, int lo, int hi,
                                              const float* v) {
  const bool wide = hi - lo + 1 > kRecNarrow;
  const unsigned mn = __ballot_sync(kFull, take && !wide);
  const unsigned mw = __ballot_sync(kFull, take && wide);
  if (!(mn | mw)) return;
  const int lane = threadIdx.x & 31;
  unsigned bn = 0, bw = 0;
  if (lane == 0) {
    if (mn) bn = atomicAdd(&S.hdr[kHdrRecNarrow], (unsigned)__popc(mn));
    if (mw) bw = atomicAdd(&S.hdr[kHdrRecWide], (unsigned)__popc(mw));
  }
  bn = __shfl_sync(kFull, bn, 0);
  bw = __shfl_sync(kFull, bw, 0);
  if (take) {
    const unsigned below = (1u << lane) - 1u;
    const unsigned i = wide ? (unsigned)S.rec_cap - 1u - (bw + __popc(mw & below))
                            : bn + __popc(mn & below);
    S.rec_c[i] = (uint32_t)c;
    S.rec_job[i] = (uint8_t)job;
    S.rec_E[i] = Ec;
    S.rec_lohi[i] = (uint16_t)(lo | (hi << 8));
    const int w = hi - lo + 1;
#pragma unroll
    for (int r = 0; r < ION_MAX_WINDOW; ++r)
      if (r < w) S.rec_V[(int64_t)r * S.rec_cap + i] = v[r];
  }
}

// The window rule after a step (unless ION_NO_WINDOW_UPDATE): the paper's
// slide, or the adaptive width.  v holds the window after the step.
template <typename T, int WM>
__device__ __forceinline__ void window_after_step(const JobIO& J, const Policy& pol,
                                                  const T (&v)[WM], int w, int& lo, int& hi) {
  if (pol.flags & ION_NO_WINDOW_UPDATE) return;
  if (pol.adaptive)
    adapt_window<T, WM>(v, w, J.Z, pol_eps<T>(pol), pol.wmin, pol.wmax, pol_grow<T>(pol), lo,
                        hi);
  else if (v[0] < pol_eps<T>(pol) && hi < J.Z)
    slide_window<T, WM>(v, w, J.Z, pol_eps<T>(pol), lo, hi);
}

// ---------------------------------------------------------------------------
// Update of one cell whose window populations v[0..w-1] and rates
// lam[r] = W_{lo+r} dt (r < w-1; 0 beyond) are known (2 <= w <= WM): Taylor
// or Bateman form, window slide, stores.  Returns true (and stores nothing)
// if the cell goes to the FP64 queue.
// ---------------------------------------------------------------------------
// With `change` set (ION_CONSERVATION_CHECK), *change receives
// |sum_r v'_r - sum_r v_r| over the window, 0 if the cell is queued.
template <typename T, int WM>
__device__ __forceinline__ bool update_cell(const JobIO& J, const Policy& pol, int c, int lo,
                                            int hi, T (&v)[WM], const T (&lam)[WM],
                                            bool allow_fb, T* change = nullptr) {
  T* __restrict__ N = static_cast<T*>(J.N);
  const int w = hi - lo + 1;
  T dne = T(0);
  int nlo = lo, nhi = hi;
  if (change) *change = T(0);
  if constexpr (WM >= 2) {
    if (w >= 2) {
      T lmax = T(0);
#pragma unroll
      for (int r = 0; r < WM; ++r) lmax = fmax(lmax, lam[r]);
      ExactSum<T> acc;
      if (change) {
#pragma unroll
        for (int r = 0; r < WM; ++r)
          if (r < w) acc.add(-v[r]);
      }
      if (lmax <= DDParams<T>::prop_max) {
        dne = taylor_propagate<T, WM>(v, lam, w, lmax);
      } else {
        if (allow_fb && (pol.flags & ION_NO_FP64_FALLBACK) == 0 &&
            ((pol.flags & ION_FORCE_FP64_COEF) != 0 ||
             (pol_gap<T>(pol) > T(0) && near_degenerate<T, WM>(lam, w, pol_gap<T>(pol)))))
          return true;
        dne = dd_update<T, WM>(v, lam, w);
      }
      if (change) {
#pragma unroll
        for (int r = 0; r < WM; ++r)
          if (r < w) acc.add(v[r]);
        *change = fabs(acc.value());
      }
      window_after_step<T, WM>(J, pol, v, w, nlo, nhi);
      T* p = N + (int64_t)lo * J.ld + c;
#pragma unroll
      for (int r = 0; r < WM; ++r) {
        if (r < w) __stcs(p, v[r]);
        p += J.ld;
      }
    }
  }
  const T* __restrict__ G = static_cast<const T*>(J.n_gas);
  __stcs(static_cast<T*>(J.dne) + c, G ? dne * G[c] : dne);
  if (nlo != lo || nhi != hi) {
    J.lo[c] = (uint8_t)nlo;
    J.hi[c] = (uint8_t)nhi;
  }
  return false;
}

// Full update of one cell whose window populations are loaded: the rates of
// Eq. 1, then update_cell.
template <class F, int WM>
__device__ __forceinline__ bool finish_cell(const JobIO& J, const Policy& pol,
                                            const typename F::Staged& tab, int c,
                                            typename F::T Ec, int lo, int hi,
                                            typename F::T (&v)[WM], bool allow_fb,
                                            typename F::T* change = nullptr) {
  using T = typename F::T;
  const int w = hi - lo + 1;
  T lam[WM];
#pragma unroll
  for (int r = 0; r < WM; ++r) lam[r] = T(0);
  if (w >= 2 && !pol.zero_dt) {
    const typename F::Field f = F::field(Ec);
#pragma unroll
    for (int r = 0; r < WM; ++r)
      if (r < w - 1) lam[r] = F::rate(tab, lo + r, f);
  }
  return update_cell<T, WM>(J, pol, c, lo, hi, v, lam, allow_fb, change);
}

// The same, loading the window from global memory; W bounds the width.
template <class F, int W>
__device__ __forceinline__ bool global_cell(const JobIO& J, const Policy& pol,
                                            const typename F::Staged& tab, int c,
                                            typename F::T Ec, int lo, int hi,
                                            bool allow_fb, typename F::T* change = nullptr) {
  using T = typename F::T;
  const T* __restrict__ N = static_cast<const T*>(J.N);
  T v[W];
  const T* p = N + (int64_t)lo * J.ld + c;
#pragma unroll
  for (int r = 0; r < W; ++r) {
    v[r] = r < hi - lo + 1 ? __ldcs(p) : T(0);
    p += J.ld;
  }
  return finish_cell<F, W>(J, pol, tab, c, Ec, lo, hi, v, allow_fb, change);
}

}  // namespace ion
