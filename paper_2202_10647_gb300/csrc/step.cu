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
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem)
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
// Each lane owns a quad of 4 consecutive cells; a warp's chunk is 128 cells.
constexpr int kQ = 4;
constexpr int kChunk = 32 * kQ;

struct QuadStage {
  float4 E[32];                   // |E| of the lane's quad
  uint32_t lo[32];                // k_lo of the quad, 4 x u8
  uint32_t hi[32];                // k_hi of the quad, 4 x u8
  float4 P[ION_MAX_WINDOW][32];   // P[r][lane].j = N[lo_j + r] of cell j
};

// Appends the record of a stiff cell (one atomic per warp).  Every lane of
// the warp calls this; `take` lanes pass their cell's inputs.
__device__ __forceinline__ void append_record(const StepArgs& a, bool take, int c,
                                              float Ec, int lo, int hi,
                                              const float* v) {
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
#pragma unroll
    for (int r = 0; r < ION_MAX_WINDOW; ++r)
      if (r < w) a.rec_V[(int64_t)r * a.rec_cap + i] = v[r];
  }
}

__device__ __forceinline__ float f4get(const float4& x, int j) {
  return j == 0 ? x.x : j == 1 ? x.y : j == 2 ? x.z : x.w;
}

// Easy path of the lane's quad (cells c0..c0+3, window bound WM).  Every
// lane of the warp calls this.  Cells whose rates all have W dt <= kLamEasy
// are finished; stiff[j] marks the others, which are left untouched.
// Written for lanes that mostly agree: every window rate takes the plain
// FP32 exponent (the stiff path recomputes its rates in float-float), and
// the Taylor series runs the warp's largest term count (extra terms only add
// accuracy).
template <int WM>
__device__ __forceinline__ void easy_quad(const StepArgs& a, const StagedF32& tab,
                                          const QuadStage& st, int lane, int c0,
                                          const float (&Ev)[kQ], const int (&lo)[kQ],
                                          const int (&hi)[kQ], const bool (&ok)[kQ],
                                          bool uni, bool (&stiff)[kQ],
                                          float (&v)[kQ][WM]) {
  int w[kQ];
#pragma unroll
  for (int j = 0; j < kQ; ++j) w[j] = ok[j] ? hi[j] - lo[j] + 1 : 0;
#pragma unroll
  for (int r = 0; r < WM; ++r) {
    const float4 p = st.P[r][lane];
    v[0][r] = p.x;
    v[1][r] = p.y;
    v[2][r] = p.z;
    v[3][r] = p.w;
  }
  float lam[kQ][WM];
  int Rl = 0;
#pragma unroll
  for (int j = 0; j < kQ; ++j) {
    stiff[j] = false;
#pragma unroll
    for (int r = 0; r < WM; ++r) lam[j][r] = 0.0f;
    if constexpr (WM >= 2) {
      // Plain FP32 exponent y = (a_hi + a_lo) - b log2|E| - C/|E|: its
      // error is below ~6e-5 in log2 units even for terms of 10^3, i.e. a
      // relative error of W dt below 4e-5, which moves populations by at most
      // 0.025 * 4e-5 = 1e-6 in the cells this path finishes (W dt <= 0.025).
      const FieldF32 f = field_f32(Ev[j]);
      const bool live = w[j] >= 2 && !f.zero && !a.zero_dt;
      const int base = ok[j] ? lo[j] : 0;
#pragma unroll
      for (int r = 0; r < WM - 1; ++r) {
        const float4 h = tab.hi[min(base + r, ION_MAX_Z)];
        const float q = h.z * f.rE;
        const float y = (fmaf(-h.y, f.lg, h.x) - q) + h.w;
        const bool on = live && r < w[j] - 1 && q <= (float)kCutoffLog2;
        lam[j][r] = on ? ex2_approx(fminf(y, 99.0f)) : 0.0f;
      }
      float lmax = 0.0f;
#pragma unroll
      for (int r = 0; r < WM - 1; ++r) lmax = fmaxf(lmax, lam[j][r]);
      stiff[j] = lmax > kLamEasy;
      const float x = stiff[j] ? 0.0f : 2.0f * lmax;
      int R = 0;
#pragma unroll
      for (int i = 0; i < kEasyTerms; ++i) R += x > kThrF32[i] ? 1 : 0;
      Rl = max(Rl, R);
    }
  }
  if constexpr (WM < 2) return;
  const int Rw = __reduce_max_sync(kFull, Rl);
  float dne[kQ];
  int nlo[kQ], nhi[kQ];
#pragma unroll
  for (int j = 0; j < kQ; ++j) {
    dne[j] = 0.0f;
    nlo[j] = lo[j];
    nhi[j] = hi[j];
    if (stiff[j] || w[j] < 2) continue;
    float t[WM], inc[WM];
#pragma unroll
    for (int i = 0; i < WM; ++i) {
      t[i] = i < w[j] ? v[j][i] : 0.0f;
      inc[i] = 0.0f;
    }
#pragma unroll
    for (int k = 1; k <= kEasyTerms; ++k) {
      if (k > Rw) break;
      const float rk = 1.0f / k;
#pragma unroll
      for (int i = WM - 1; i >= 0; --i) {
        const float gain = i > 0 ? lam[j][i - 1] * t[i - 1] : 0.0f;
        t[i] = (gain - lam[j][i] * t[i]) * rk;
        inc[i] += t[i];
      }
    }
    float cum = 0.0f;
#pragma unroll
    for (int r = 0; r < WM - 1; ++r) {
      if (r < w[j] - 1) {
        cum -= inc[r];  // population that left states <= r
        dne[j] += cum;
      }
    }
#pragma unroll
    for (int r = 0; r < WM; ++r) v[j][r] += inc[r];
    if ((a.flags & ION_NO_WINDOW_UPDATE) == 0 && v[j][0] < (float)a.eps && hi[j] < a.Z)
      slide_window<float, WM>(v[j], w[j], a.Z, (float)a.eps, nlo[j], nhi[j]);
  }
  // stores
  const float* __restrict__ G = static_cast<const float*>(a.n_gas);
  if (G) {
#pragma unroll
    for (int j = 0; j < kQ; ++j)
      if (ok[j] && !stiff[j]) dne[j] *= G[c0 + j];
  }
  const bool whole = uni && !stiff[0] && !stiff[1] && !stiff[2] && !stiff[3];
  float* __restrict__ N = static_cast<float*>(a.N);
  float* __restrict__ D = static_cast<float*>(a.dne);
  if (whole && a.vec) {
    float* p = N + (int64_t)lo[0] * a.ld + c0;
#pragma unroll
    for (int r = 0; r < WM; ++r) {
      if (r < w[0])
        __stcs(reinterpret_cast<float4*>(p), make_float4(v[0][r], v[1][r], v[2][r], v[3][r]));
      p += a.ld;
    }
    __stcs(reinterpret_cast<float4*>(D + c0), make_float4(dne[0], dne[1], dne[2], dne[3]));
  } else {
#pragma unroll
    for (int j = 0; j < kQ; ++j) {
      if (!ok[j] || stiff[j]) continue;
      float* p = N + (int64_t)lo[j] * a.ld + c0 + j;
#pragma unroll
      for (int r = 0; r < WM; ++r) {
        if (r < w[j]) __stcs(p, v[j][r]);
        p += a.ld;
      }
      __stcs(D + c0 + j, dne[j]);
    }
  }
#pragma unroll
  for (int j = 0; j < kQ; ++j) {
    if (ok[j] && !stiff[j] && nlo[j] != lo[j]) {
      a.lo[c0 + j] = (uint8_t)nlo[j];
      a.hi[c0 + j] = (uint8_t)nhi[j];
    }
  }
}

// Width-1 quads: nothing moves; only dne = 0 is written.
__device__ __forceinline__ void trivial_quad(const StepArgs& a, int c0,
                                             const bool (&ok)[kQ]) {
  float* D = static_cast<float*>(a.dne);
#pragma unroll
  for (int j = 0; j < kQ; ++j)
    if (ok[j]) __stcs(D + c0 + j, 0.0f);
}

__global__ void __launch_bounds__(kWarps * 32, 4)
    ion_step_f32_kernel(const __grid_constant__ StepArgs a) {
  constexpr int kStagesQ = 3;
  __shared__ StagedF32 tab;
  __shared__ QuadStage ring[kWarps][kStagesQ];
  stage_f32(a.tab, a.log2dt, &tab);
  {
    // plane slots past a cell's window are read (and ignored); keep them
    // finite
    float* z = reinterpret_cast<float*>(&ring[0][0]);
    for (int i = threadIdx.x; i < (int)(sizeof(ring) / sizeof(float)); i += blockDim.x)
      z[i] = 0.0f;
  }
  __syncthreads();

  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  QuadStage* S = ring[wib];
  const int gw = blockIdx.x * kWarps + wib;
  const int TW = gridDim.x * kWarps;
  const int nfull = a.ncells / kChunk;
  const int K = gw < nfull ? (nfull - 1 - gw) / TW + 1 : 0;
  const float* __restrict__ E = static_cast<const float*>(a.E);
  const float* __restrict__ N = static_cast<const float*>(a.N);
  const int64_t ld = a.ld;

  // |E|, k_lo, k_hi of the lane's quad of chunk k into stage `sg` (one
  // commit group)
  auto issue_front = [&](int k, int sg) {
    if (k < K) {
      const int c0 = (gw + k * TW) * kChunk + kQ * lane;
      QuadStage& st = S[sg];
      if (a.vec) {
        cp_async16(&st.E[lane], E + c0);
      } else {
        float* e = reinterpret_cast<float*>(&st.E[lane]);
#pragma unroll
        for (int j = 0; j < kQ; ++j) cp_async4(e + j, E + c0 + j);
      }
      cp_async4(&st.lo[lane], a.lo + c0);
      cp_async4(&st.hi[lane], a.hi + c0);
    }
    cp_async_commit();
  };
  // the window planes of the lane's quad of chunk k in stage `sg` (one
  // commit group)
  auto issue_planes = [&](int k, int sg) {
    if (k < K) {
      const int c0 = (gw + k * TW) * kChunk + kQ * lane;
      QuadStage& st = S[sg];
      const uint32_t l4 = st.lo[lane], h4 = st.hi[lane];
      const int lo0 = l4 & 0xff, hi0 = h4 & 0xff;
      if (a.vec && l4 == lo0 * 0x01010101u && h4 == hi0 * 0x01010101u) {
        // the quad shares its window: one 16-byte copy per plane
        const int w = window_ok(lo0, hi0, a.Z) ? hi0 - lo0 + 1 : 0;
        const float* p = N + (int64_t)lo0 * ld + c0;
        float4* d = &st.P[0][lane];
        for (int r = 0; r < w; ++r) {
          cp_async16(d, p);
          p += ld;
          d += 32;
        }
      } else {
        float* P0 = reinterpret_cast<float*>(&st.P[0][lane]);
#pragma unroll
        for (int j = 0; j < kQ; ++j) {
          const int lj = (l4 >> (8 * j)) & 0xff, hj = (h4 >> (8 * j)) & 0xff;
          const int w = window_ok(lj, hj, a.Z) ? hj - lj + 1 : 0;
          const float* p = N + (int64_t)lj * ld + c0 + j;
          for (int r = 0; r < w; ++r) {
            cp_async4(P0 + r * 128 + j, p);
            p += ld;
          }
        }
      }
    }
    cp_async_commit();
  };

  // stages: chunk k lives in s0, k+1 in s1, k+2 in s2 (a rotation of 0,1,2)
  int s0 = 0, s1 = 1, s2 = 2;
  issue_front(0, s0);
  issue_front(1, s1);
  cp_async_wait<1>();  // front(0)
  __syncwarp();
  issue_planes(0, s0);
  for (int k = 0; k < K; ++k) {
    issue_front(k + 2, s2);
    cp_async_wait<2>();  // front(k+1): pending are planes(k), front(k+2)
    __syncwarp();
    issue_planes(k + 1, s1);
    cp_async_wait<2>();  // planes(k): pending are front(k+2), planes(k+1)
    __syncwarp();

    const QuadStage& st = S[s0];
    const int c0 = (gw + k * TW) * kChunk + kQ * lane;
    const float4 e4 = st.E[lane];
    const float Ev[kQ] = {e4.x, e4.y, e4.z, e4.w};
    const uint32_t l4 = st.lo[lane], h4 = st.hi[lane];
    int lo[kQ], hi[kQ], wl = 0;
    bool ok[kQ];
    const bool same = l4 == (l4 & 0xff) * 0x01010101u && h4 == (h4 & 0xff) * 0x01010101u;
    bool uni;
    if (same) {
      const int l0 = l4 & 0xff, h0 = h4 & 0xff;
      const bool o = window_ok(l0, h0, a.Z);
#pragma unroll
      for (int j = 0; j < kQ; ++j) {
        lo[j] = l0;
        hi[j] = h0;
        ok[j] = o;
      }
      wl = o ? h0 - l0 + 1 : 0;
      if (!o) atomicAdd(&a.hdr[kHdrInvalid], (unsigned)kQ);
      uni = o;
    } else {
      int nbad = 0;
#pragma unroll
      for (int j = 0; j < kQ; ++j) {
        lo[j] = (l4 >> (8 * j)) & 0xff;
        hi[j] = (h4 >> (8 * j)) & 0xff;
        ok[j] = window_ok(lo[j], hi[j], a.Z);
        nbad += ok[j] ? 0 : 1;
        wl = ok[j] ? max(wl, hi[j] - lo[j] + 1) : wl;
      }
      if (nbad) atomicAdd(&a.hdr[kHdrInvalid], (unsigned)nbad);
      uni = false;
    }
    const int WMw = __reduce_max_sync(kFull, wl);
    bool stiff[kQ] = {false, false, false, false};
    if (WMw <= 1) {
      trivial_quad(a, c0, ok);
    } else if (WMw == 2) {
      float v[kQ][2];
      easy_quad<2>(a, tab, st, lane, c0, Ev, lo, hi, ok, uni, stiff, v);
    } else if (WMw <= 4) {
      float v[kQ][4];
      easy_quad<4>(a, tab, st, lane, c0, Ev, lo, hi, ok, uni, stiff, v);
    } else {
      float v[kQ][6];
      easy_quad<6>(a, tab, st, lane, c0, Ev, lo, hi, ok, uni, stiff, v);
    }
    // stiff cells: their inputs (as loaded) go to the record queue
    if (__ballot_sync(kFull, stiff[0] || stiff[1] || stiff[2] || stiff[3])) {
#pragma unroll
      for (int j = 0; j < kQ; ++j) {
        float vin[ION_MAX_WINDOW];
#pragma unroll
        for (int r = 0; r < ION_MAX_WINDOW; ++r) vin[r] = f4get(st.P[r][lane], j);
        append_record(a, stiff[j], c0 + j, Ev[j], lo[j], hi[j], vin);
      }
    }
    __syncwarp();
    const int t = s0;
    s0 = s1;
    s1 = s2;
    s2 = t;
  }
  cp_async_wait<0>();

  // the last, partial chunk (ncells % 128 cells): every valid cell becomes a
  // record for the stiff kernel, which runs the full path
  const int tail0 = nfull * kChunk;
  if (tail0 < a.ncells && gw == TW - 1) {
    for (int cb = tail0; cb < a.ncells; cb += 32) {
      const int c = cb + lane;
      bool take = false;
      float Ec = 0.0f, v[ION_MAX_WINDOW];
      int lo = 0, hi = 0;
#pragma unroll
      for (int r = 0; r < ION_MAX_WINDOW; ++r) v[r] = 0.0f;
      if (c < a.ncells) {
        Ec = E[c];
        lo = a.lo[c];
        hi = a.hi[c];
        take = window_ok(lo, hi, a.Z);
        if (!take) atomicAdd(&a.hdr[kHdrInvalid], 1u);
        const float* p = N + (int64_t)lo * ld + c;
#pragma unroll
        for (int r = 0; r < ION_MAX_WINDOW; ++r) {
          if (take && r < hi - lo + 1) v[r] = p[0];
          p += ld;
        }
      }
      append_record(a, take, c, Ec, lo, hi, v);
    }
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
  const int64_t chunks = ((int64_t)a.ncells + kChunk - 1) / kChunk;
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
