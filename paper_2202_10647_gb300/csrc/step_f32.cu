// step_f32.cu -- the FP32 form of ion_step / ion_step_batched (ION_F32):
// one persistent launch over the cells of up to kMaxJobs species, then two
// small kernels over the cells it left behind.
//
//   ion_stream_kernel<Q, W>  every warp draws chunks of 32*Q cells (Q
//       consecutive cells per lane) in runs of four from a counter in the
//       workspace header and moves them through a 4-stage ring in
//       shared memory.  cp.async brings |E|, k_lo and k_hi in three chunks
//       ahead and each lane's own window planes two chunks ahead (one copy of
//       4*Q bytes per plane when the lane's cells share their window), so the
//       loads in flight cost no registers and the traffic is exactly the
//       cells' windows.  A chunk whose cells all lie below their species'
//       cold field (no rate reaches the first Taylor term) only writes dne.
//       A cell whose rates all have W dt <= 1 (1.5 with one cell per
//       lane) is finished here with the Taylor series of exp(dt A).  The others ("stiff" cells,
//       the Bateman form) write the inputs already loaded into a record queue:
//       in a laser field |E| swings from zero to its peak every few cells, so
//       most warps near the pulse hold a few stiff cells, and finishing them
//       in place would make every such warp run the longest path of its
//       lanes.  The window-width bucket (the loops' bound) is taken per warp
//       and chunk.  Q and W (warps per block) are the launch shape that
//       ion_autotune picks.
//   ion_stiff_kernel   the records, one per thread in full warps: Taylor form
//       up to W dt <= 1, divided-difference (Bateman) form above.  Cells with
//       a nearly degenerate rate pair are left untouched and queued for
//   ion_fb_kernel      FP32 rates, FP64 Bateman coefficients and propagation,
//       rounded back to FP32.
//
// One step is Eqs. 1-9 of the paper per cell; see ion_device.cuh.
#include <cstdint>
#include <mutex>

#include "ion_cell.cuh"
#include "ion_step.cuh"

namespace ion {

namespace {

constexpr int kStages = 4;
// The streaming kernel finishes every cell whose rates all have
// W dt <= lam_easy<Q>() with the Taylor form, in at most kEasyTerms terms:
// 2 lam_easy <= kThrF32[kEasyTerms] (3 <= 3.19).  The warp runs the term
// count of its largest rate, so the bound trades a longer series for every
// cell of a warp against the records that a lower bound makes: with 32 cells
// per warp (Q = 1) the series up to W dt = 1.5 measured faster than records
// (2-3 % on the Ar-like and mixed batches, the FP32 rounding of the series
// about 2.7e-7 there against 2.0e-7 at 1); with 64 (Q = 2) records above 1.
template <int Q>
constexpr float lam_easy() {
  return Q == 1 ? 1.5f : 1.0f;
}
constexpr int kEasyTerms = 18;
// 1/k! for the Taylor terms of the streaming kernel (constant memory: the
// term loop reads one entry per term at a warp-uniform index)
__constant__ const float kInvFactF32[kEasyTerms + 1] = {
    1.0f,
    1.0f,
    1.0f / 2,
    1.0f / 6,
    1.0f / 24,
    1.0f / 120,
    1.0f / 720,
    1.0f / 5040,
    1.0f / 40320,
    1.0f / 362880,
    1.0f / 3628800,
    1.0f / 39916800,
    1.0f / 479001600,
    1.0f / 6227020800.0f,
    1.0f / 87178291200.0f,
    1.0f / 1307674368000.0f,
    1.0f / 20922789888000.0f,
    1.0f / 355687428096000.0f,
    1.0f / 6402373705728000.0f};
// Rates with W dt above this are recomputed in float-float arithmetic.
constexpr float kLamPrecise = 1.0f / 64.0f;

template <int Q>
struct VecOf;
template <>
struct VecOf<1> {
  using T = float;
};
template <>
struct VecOf<2> {
  using T = float2;
};
template <>
struct VecOf<4> {
  using T = float4;
};

__device__ __forceinline__ float vget(const float& x, int) { return x; }
__device__ __forceinline__ float vget(const float2& x, int j) { return j == 0 ? x.x : x.y; }
__device__ __forceinline__ float vget(const float4& x, int j) {
  return j == 0 ? x.x : j == 1 ? x.y : j == 2 ? x.z : x.w;
}
__device__ __forceinline__ void vstore(float* p, const float (&v)[1]) { __stcs(p, v[0]); }
__device__ __forceinline__ void vstore(float* p, const float (&v)[2]) {
  __stcs(reinterpret_cast<float2*>(p), make_float2(v[0], v[1]));
}
__device__ __forceinline__ void vstore(float* p, const float (&v)[4]) {
  __stcs(reinterpret_cast<float4*>(p), make_float4(v[0], v[1], v[2], v[3]));
}

template <int Q>
struct QStage {
  using V = typename VecOf<Q>::T;
  V E[32];                      // |E| of the lane's Q cells
  uint32_t lo[8 * Q];           // k_lo of the chunk's 32*Q cells
  uint32_t hi[8 * Q];           // k_hi
  V P[ION_MAX_WINDOW][32];      // P[r][lane] component j = N[lo_j + r] of cell j
  int g;                        // the chunk (>= nchunks: none)
};

// Chunks are handed out in runs of this many consecutive ones.
constexpr int kRun = 4;
static_assert((kRun & (kRun - 1)) == 0, "kRun is a power of two");

// The Q bytes of a lane in a packed byte array (one load of Q bytes), and
// whether they are equal.
template <int Q>
__device__ __forceinline__ uint32_t lane_bytes(const uint32_t* arr, int lane) {
  if constexpr (Q == 4) return arr[lane];
  if constexpr (Q == 2) return reinterpret_cast<const uint16_t*>(arr)[lane];
  return reinterpret_cast<const uint8_t*>(arr)[lane];
}
template <int Q>
__device__ __forceinline__ bool bytes_equal(uint32_t x) {
  if constexpr (Q == 4) return x == (x & 0xff) * 0x01010101u;
  if constexpr (Q == 2) return x == (x & 0xff) * 0x0101u;
  return true;
}

// Job of a chunk (jobs are few; chunks are numbered job after job).
__device__ __forceinline__ int job_of(const BatchArgs& a, int g) {
  if (a.njobs == 1) return 0;  // uniform: the single-species call
  int j = 0;
#pragma unroll
  for (int i = 1; i < kMaxJobs; ++i)
    if (i < a.njobs && g >= a.job[i].chunk0) j = i;
  return j;
}

// Easy path of the lane's Q cells (c0..c0+Q-1 of job J, window bound WM).
// Every lane of the warp calls this.  Cells whose rates all have
// W dt <= lam_easy<Q>() are finished; stiff[j] marks the others, left untouched.
// Every window rate first takes the plain FP32 exponent y = a_hi - b log2|E|
// - C/|E| (a_lo, the low part of a, left out: half an ulp of a, below 1e-5 in
// log2 units for |a| < 256): its error is below ~7e-5 in log2 units even for
// terms of 10^3, i.e. a relative error of W dt below 5e-5, which moves
// populations by at most 5e-5 W dt; rates above kLamPrecise = 2^-6 (where
// that could reach 8e-7) are recomputed in float-float.  Past the cutoff
// (C/|E| > kCutoffLog2, where Eq. 1 is 0) y lies far below -126, so the
// SFU's ex2, which flushes results below 2^-126 to 0, needs no test for it.  The Taylor series runs the warp's
// largest term count (extra terms only add accuracy), counted by one ballot:
// lane i holds thr_lane = kThrF32[i] (infinity from lane kEasyTerms on).
template <int Q>
using PlaneRows = typename VecOf<Q>::T[ION_MAX_WINDOW][32];

// The records of a warp's chunk: the stiff cells of all its lanes, one
// atomic per class (narrow from the front of the arrays, wide from the
// back) for the whole warp, cell j of every lane after cell j-1 of every
// lane; the inputs as loaded (the stage's planes).
template <int Q>
__device__ __forceinline__ void append_records(const Scratch& S, int job, int c0,
                                               const float (&Ec)[Q], const int (&lo)[Q],
                                               const int (&hi)[Q], const bool (&take)[Q],
                                               const PlaneRows<Q>& P, int lane) {
  bool any = false;
#pragma unroll
  for (int j = 0; j < Q; ++j) any = any || take[j];
  if (!__ballot_sync(kFull, any)) return;
  unsigned mn[Q], mw[Q], nn = 0, nw = 0;
#pragma unroll
  for (int j = 0; j < Q; ++j) {
    const bool wide = hi[j] - lo[j] + 1 > kRecNarrow;
    mn[j] = __ballot_sync(kFull, take[j] && !wide);
    mw[j] = __ballot_sync(kFull, take[j] && wide);
    nn += __popc(mn[j]);
    nw += __popc(mw[j]);
  }
  unsigned bn = 0, bw = 0;
  if (lane == 0) {
    if (nn) bn = atomicAdd(&S.hdr[kHdrRecNarrow], nn);
    if (nw) bw = atomicAdd(&S.hdr[kHdrRecWide], nw);
  }
  bn = __shfl_sync(kFull, bn, 0);
  bw = __shfl_sync(kFull, bw, 0);
  const unsigned below = (1u << lane) - 1u;
#pragma unroll
  for (int j = 0; j < Q; ++j) {
    if (take[j]) {
      const bool wide = hi[j] - lo[j] + 1 > kRecNarrow;
      const unsigned i = wide ? (unsigned)S.rec_cap - 1u - (bw + __popc(mw[j] & below))
                              : bn + __popc(mn[j] & below);
      S.rec_c[i] = (uint32_t)(c0 + j);
      S.rec_job[i] = (uint8_t)job;
      S.rec_E[i] = Ec[j];
      S.rec_lohi[i] = (uint16_t)(lo[j] | (hi[j] << 8));
      const int w = hi[j] - lo[j] + 1;
#pragma unroll
      for (int r = 0; r < ION_MAX_WINDOW; ++r)
        if (r < w) S.rec_V[(int64_t)r * S.rec_cap + i] = vget(P[r][lane], j);
    }
    bn += __popc(mn[j]);
    bw += __popc(mw[j]);
  }
}

// CONS (the call has ION_CONSERVATION_CHECK; a separate instantiation, so
// that the other calls carry none of it): cmax becomes the larger of itself
// and the bits of |sum_r v'_r - sum_r v_r| of each cell finished here.
template <int Q, int WM, bool AD, bool CONS>
__device__ __forceinline__ void easy_cells(const JobIO& J, const Policy& pol,
                                           const StagedF32& tab, const PlaneRows<Q>& P,
                                           int lane, int c0, const float (&Ev)[Q],
                                           const int (&lo)[Q], const int (&hi)[Q],
                                           const bool (&ok)[Q], bool uni, bool (&stiff)[Q],
                                           float thr_lane, uint32_t& cmax) {
  int w[Q];
  float v[Q][WM];
#pragma unroll
  for (int j = 0; j < Q; ++j) w[j] = ok[j] ? hi[j] - lo[j] + 1 : 0;
#pragma unroll
  for (int r = 0; r < WM; ++r) {
    const typename VecOf<Q>::T p = P[r][lane];
#pragma unroll
    for (int j = 0; j < Q; ++j) v[j][r] = vget(p, j);  // r >= w: ignored
  }
  float lam[Q][WM];
  float xl = 0.0f;
#pragma unroll
  for (int j = 0; j < Q; ++j) {
    stiff[j] = false;
#pragma unroll
    for (int r = 0; r < WM; ++r) lam[j][r] = 0.0f;
    const FieldF32 f = field_f32(Ev[j]);
    const bool live = w[j] >= 2 && !f.zero && !pol.zero_dt;
    const int base = ok[j] ? lo[j] : 0;
#pragma unroll
    for (int r = 0; r < WM - 1; ++r) {
      const float4 h = tab.hi[base + r];  // < ION_MAX_Z + ION_MAX_WINDOW
      const float y = fmaf(-h.z, f.rE, fmaf(-h.y, f.lg, h.x));
      const bool on = live && r < w[j] - 1;
      lam[j][r] = on ? ex2_approx(fminf(y, 99.0f)) : 0.0f;
    }
#pragma unroll
    for (int r = 0; r < WM - 1; ++r)
      if (lam[j][r] > kLamPrecise) lam[j][r] = rate_ff_f32(tab, base + r, f);
    float lmax = 0.0f;
#pragma unroll
    for (int r = 0; r < WM - 1; ++r) lmax = fmaxf(lmax, lam[j][r]);
    stiff[j] = lmax > lam_easy<Q>();
    xl = fmaxf(xl, stiff[j] ? 0.0f : 2.0f * lmax);
  }
  // the warp's largest 2 max(W dt) (non-negative floats order like their
  // bits), then its term count once
  const float xw = __uint_as_float(__reduce_max_sync(kFull, __float_as_uint(xl)));
  const int Rw = __popc(__ballot_sync(kFull, xw > thr_lane));
  float dne[Q];
  int nlo[Q], nhi[Q];
  // u = (dt A)^k v unnormalized (|dt A| <= 2 lam_easy keeps it small);
  // inc = sum_k u / k!.  The term loop is outermost so that the Q cells'
  // recurrences interleave.  Slots past a cell's window start from whatever
  // the stage holds there: their rates and the rate into them are zero, so
  // their u is zero after one term and their inc stays zero.  Stiff cells
  // run with rates above lam_easy; their inc is never read.
  float u[Q][WM], inc[Q][WM];
#pragma unroll
  for (int j = 0; j < Q; ++j) {
#pragma unroll
    for (int i = 0; i < WM; ++i) {
      u[j][i] = v[j][i];
      inc[j][i] = 0.0f;
    }
  }
#pragma unroll 1
  for (int k = 1; k <= Rw; ++k) {
    const float ck = kInvFactF32[k];
#pragma unroll
    for (int j = 0; j < Q; ++j) {
#pragma unroll
      for (int i = WM - 2; i >= 0; --i) {
        u[j][i] = fmaf(-lam[j][i], u[j][i], i > 0 ? lam[j][i - 1] * u[j][i - 1] : 0.0f);
        inc[j][i] = fmaf(u[j][i], ck, inc[j][i]);
      }
    }
  }
  // the last slot by conservation: the top state of a window of width WM
  // gains what the others lost (narrower windows reach their top inside the
  // series, whose rate there is zero, and never read this slot)
#pragma unroll
  for (int j = 0; j < Q; ++j) {
    float t = 0.0f;
#pragma unroll
    for (int i = 0; i < WM - 1; ++i) t -= inc[j][i];
    inc[j][WM - 1] = t;
  }
#pragma unroll
  for (int j = 0; j < Q; ++j) {
    dne[j] = 0.0f;
    nlo[j] = lo[j];
    nhi[j] = hi[j];
    if (stiff[j] || w[j] < 2) continue;
    float cum = 0.0f;
#pragma unroll
    for (int r = 0; r < WM - 1; ++r) {
      if (r < w[j] - 1) {
        cum -= inc[j][r];  // population that left states <= r
        dne[j] += cum;
      }
    }
#pragma unroll
    for (int r = 0; r < WM; ++r) v[j][r] += inc[j][r];
    if constexpr (CONS) {
      ExactSum<float> acc;
#pragma unroll
      for (int r = 0; r < WM; ++r) {
        if (r < w[j]) {
          acc.add(-vget(P[r][lane], j));
          acc.add(v[j][r]);
        }
      }
      cmax = max(cmax, abs_bits(acc.value()));
    }
    if ((pol.flags & ION_NO_WINDOW_UPDATE) == 0) {
      if constexpr (AD)
        adapt_window<float, WM>(v[j], w[j], J.Z, pol.eps_f, pol.wmin, pol.wmax,
                                pol.eps_grow_f, nlo[j], nhi[j]);
      else if (v[j][0] < pol.eps_f && hi[j] < J.Z)
        slide_window<float, WM>(v[j], w[j], J.Z, pol.eps_f, nlo[j], nhi[j]);
    }
  }
  // stores
  const float* __restrict__ G = static_cast<const float*>(J.n_gas);
  if (G) {
#pragma unroll
    for (int j = 0; j < Q; ++j)
      if (ok[j] && !stiff[j]) dne[j] *= G[c0 + j];
  }
  bool whole = uni;
#pragma unroll
  for (int j = 0; j < Q; ++j) whole = whole && !stiff[j];
  float* __restrict__ N = static_cast<float*>(J.N);
  float* __restrict__ D = static_cast<float*>(J.dne);
  if (whole && J.vec) {
    float* p = N + (int64_t)lo[0] * J.ld + c0;
#pragma unroll
    for (int r = 0; r < WM; ++r) {
      if (r < w[0]) {
        float o[Q];
#pragma unroll
        for (int j = 0; j < Q; ++j) o[j] = v[j][r];
        vstore(p, o);
      }
      p += J.ld;
    }
    vstore(D + c0, dne);
  } else {
#pragma unroll
    for (int j = 0; j < Q; ++j) {
      if (!ok[j] || stiff[j]) continue;
      float* p = N + (int64_t)lo[j] * J.ld + c0 + j;
#pragma unroll
      for (int r = 0; r < WM; ++r) {
        if (r < w[j]) __stcs(p, v[j][r]);
        p += J.ld;
      }
      __stcs(D + c0 + j, dne[j]);
    }
  }
#pragma unroll
  for (int j = 0; j < Q; ++j) {
    if (ok[j] && !stiff[j] && (nlo[j] != lo[j] || nhi[j] != hi[j])) {
      J.lo[c0 + j] = (uint8_t)nlo[j];
      J.hi[c0 + j] = (uint8_t)nhi[j];
    }
  }
}

template <int Q>
constexpr size_t stage_bytes() {
  return sizeof(QStage<Q>);
}

template <int Q, int W>
constexpr size_t stream_smem(int njobs) {
  return (size_t)njobs * sizeof(StagedF32) + (size_t)W * kStages * sizeof(QStage<Q>);
}

// Registers per thread of the streaming kernel, by cells per lane: 80 lets
// three blocks of 8 warps (24 warps) share an SM's 64K registers with no
// spill at Q = 2; left to itself the compiler takes about 90, and two blocks.
template <int Q>
constexpr int stream_regs() {
  return Q == 1 ? 64 : Q == 2 ? 80 : 128;
}

// Each job's last, partial chunk (ncells % kChunk cells), taken by one warp
// per job (gw of TW): every valid cell becomes a record for the stiff
// kernel, which runs the full path.
__device__ __forceinline__ void tail_records(const BatchArgs& a, int kChunk, int gw, int TW,
                                             int lane) {
  for (int jid = 0; jid < a.njobs; ++jid) {
    if (gw != (TW - 1 - jid % TW)) continue;
    const JobIO& J = a.job[jid];
    const int tail0 = (J.ncells / kChunk) * kChunk;
    for (int cb = tail0; cb < J.ncells; cb += 32) {
      const int c = cb + lane;
      bool take = false;
      float Ec = 0.0f, v[ION_MAX_WINDOW];
      int lo = 0, hi = 0;
#pragma unroll
      for (int r = 0; r < ION_MAX_WINDOW; ++r) v[r] = 0.0f;
      if (c < J.ncells) {
        Ec = static_cast<const float*>(J.E)[c];
        lo = J.lo[c];
        hi = J.hi[c];
        take = window_ok(lo, hi, J.Z);
        if (!take) atomicAdd(&a.ws.hdr[kHdrInvalid], 1u);
        const float* p = static_cast<const float*>(J.N) + (int64_t)lo * J.ld + c;
#pragma unroll
        for (int r = 0; r < ION_MAX_WINDOW; ++r) {
          if (take && r < hi - lo + 1) v[r] = p[0];
          p += J.ld;
        }
      }
      append_record(a.ws, take, jid, c, Ec, lo, hi, v);
    }
  }
}

// AD: the adaptive window policy (a separate instantiation, so that the
// fixed rule's kernels carry none of it).
template <int Q, int W, bool AD, bool CONS>
__global__ void __maxnreg__(stream_regs<Q>())
    ion_stream_kernel(const __grid_constant__ BatchArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  StagedF32* tabs = reinterpret_cast<StagedF32*>(smem);
  QStage<Q>* ring = reinterpret_cast<QStage<Q>*>(smem + (size_t)a.njobs * sizeof(StagedF32));
  for (int j = 0; j < a.njobs; ++j) stage_f32(a.job[j].tab, a.pol.log2dt, &tabs[j]);
  for (int j = threadIdx.x >> 5; j < a.njobs; j += W)
    stage_cold(a.job[j].tab, a.pol.log2dt, kColdLog2, tabs[j].ecold, threadIdx.x & 31);
  {
    // plane slots past a cell's window are read (and ignored); keep them
    // finite
    float* z = reinterpret_cast<float*>(ring);
    const int nz = (int)(W * kStages * sizeof(QStage<Q>) / sizeof(float));
    for (int i = threadIdx.x; i < nz; i += blockDim.x) z[i] = 0.0f;
  }
  __syncthreads();

  constexpr int kChunk = 32 * Q;
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  QStage<Q>* S = ring + wib * kStages;
  const int gw = blockIdx.x * W + wib;
  const int TW = gridDim.x * W;
  using V = typename VecOf<Q>::T;

  // Each warp draws its chunks in runs of kRun consecutive ones from a
  // counter in the workspace header, so that warps whose chunks are cheap
  // (cold) take more of them and all warps run out of work together.
  uint32_t* const next = &a.ws.hdr[kHdrChunk];
  int gnext = 0;
  if (lane == 0) gnext = (int)atomicAdd(next, (unsigned)kRun);
  gnext = __shfl_sync(kFull, gnext, 0);
  auto take_chunk = [&]() -> int {
    const int g = gnext;
    if (g >= a.nchunks) return g;
    if ((++gnext & (kRun - 1)) == 0) {  // kRun is a power of two
      int b = 0;
      if (lane == 0) b = (int)atomicAdd(next, (unsigned)kRun);
      gnext = __shfl_sync(kFull, b, 0);
    }
    return g;
  };

  // |E|, k_lo, k_hi of the next chunk into stage sg (one commit group)
  auto issue_front = [&](int sg) {
    const int g = take_chunk();
    if (lane == 0) S[sg].g = g;
    if (g < a.nchunks) {
      const JobIO& J = a.job[job_of(a, g)];
      const int cb = (g - J.chunk0) * kChunk;
      QStage<Q>& st = S[sg];
      const float* E = static_cast<const float*>(J.E) + cb + Q * lane;
      if (J.vec) {
        cp_async<4 * Q>(&st.E[lane], E);
      } else {
        float* e = reinterpret_cast<float*>(&st.E[lane]);
#pragma unroll
        for (int j = 0; j < Q; ++j) cp_async<4>(e + j, E + j);
      }
      if constexpr (Q == 4) {
        cp_async<4>(&st.lo[lane], J.lo + cb + 4 * lane);
        cp_async<4>(&st.hi[lane], J.hi + cb + 4 * lane);
      } else {
        constexpr int nw = 8 * Q;
        if (lane < nw)
          cp_async<4>(&st.lo[lane], J.lo + cb + 4 * lane);
        else if (lane < 2 * nw)
          cp_async<4>(&st.hi[lane - nw], J.hi + cb + 4 * (lane - nw));
      }
    }
    cp_async_commit();
  };
  // the window planes of the lane's cells of the chunk in stage sg
  auto issue_planes = [&](int sg) {
    const int g = S[sg].g;
    if (g < a.nchunks) {
      const JobIO& J = a.job[job_of(a, g)];
      const int c0 = (g - J.chunk0) * kChunk + Q * lane;
      QStage<Q>& st = S[sg];
      const uint32_t l = lane_bytes<Q>(st.lo, lane), h = lane_bytes<Q>(st.hi, lane);
      const int lo0 = l & 0xff, hi0 = h & 0xff;
      const float* N = static_cast<const float*>(J.N);
      if (J.vec && bytes_equal<Q>(l) && bytes_equal<Q>(h)) {
        // the lane's cells share their window: one copy per plane
        const int w = window_ok(lo0, hi0, J.Z) ? hi0 - lo0 + 1 : 0;
        const float* p = N + (int64_t)lo0 * J.ld + c0;
        V* d = &st.P[0][lane];
#pragma unroll
        for (int r = 0; r < ION_MAX_WINDOW; ++r) {
          if (r < w) cp_async<4 * Q>(d + 32 * r, p + (int64_t)r * J.ld);
        }
      } else {
        float* P0 = reinterpret_cast<float*>(&st.P[0][lane]);
#pragma unroll
        for (int j = 0; j < Q; ++j) {
          const int lj = (l >> (8 * j)) & 0xff, hj = (h >> (8 * j)) & 0xff;
          const int w = window_ok(lj, hj, J.Z) ? hj - lj + 1 : 0;
          const float* p = N + (int64_t)lj * J.ld + c0 + j;
          for (int r = 0; r < w; ++r) {
            cp_async<4>(P0 + r * 32 * Q + j, p);
            p += J.ld;
          }
        }
      }
    }
    cp_async_commit();
  };

  const float thr_lane = lane < kEasyTerms ? kThrF32[lane] : __int_as_float(0x7f800000);
  uint32_t cmax = 0;  // largest |change of sum_k N_k| (bits), ION_CONSERVATION_CHECK
  // Chunk k lives in stage k mod 4.  Commit groups go out in the order
  // front(k+3), planes(k+2) in iteration k, so one wait that leaves the two
  // newest pending (planes(k+1), front(k+3)) completes front(k+2) and
  // planes(k): the planes arrive two iterations after they are requested,
  // which hides the memory latency behind chunks that take little
  // arithmetic.
  static_assert(kStages == 4, "stage k mod 4");
  issue_front(0);
  issue_front(1);
  issue_front(2);
  cp_async_wait<2>();  // front(0)
  __syncwarp();
  issue_planes(0);
  cp_async_wait<2>();  // front(1)
  __syncwarp();
  issue_planes(1);
  for (int k = 0;; ++k) {
    issue_front((k + 3) & 3);
    cp_async_wait<2>();  // front(k+2) and planes(k)
    __syncwarp();
    issue_planes((k + 2) & 3);

    const QStage<Q>& st = S[k & 3];
    const int g = st.g;
    if (g >= a.nchunks) break;  // chunks come in increasing order: no more
    const int jid = job_of(a, g);
    const JobIO& J = a.job[jid];
    const int c0 = (g - J.chunk0) * kChunk + Q * lane;
    const V e = st.E[lane];
    float Ev[Q];
#pragma unroll
    for (int j = 0; j < Q; ++j) Ev[j] = vget(e, j);
    const uint32_t l = lane_bytes<Q>(st.lo, lane), h = lane_bytes<Q>(st.hi, lane);
    int lo[Q], hi[Q], wl = 0;
    bool ok[Q];
    bool uni;
    if (bytes_equal<Q>(l) && bytes_equal<Q>(h)) {
      const int l0 = l & 0xff, h0 = h & 0xff;
      const bool o = window_ok(l0, h0, J.Z);
#pragma unroll
      for (int j = 0; j < Q; ++j) {
        lo[j] = l0;
        hi[j] = h0;
        ok[j] = o;
      }
      wl = o ? h0 - l0 + 1 : 0;
      if (!o) atomicAdd(&a.ws.hdr[kHdrInvalid], (unsigned)Q);
      uni = o;
    } else {
      int nbad = 0;
#pragma unroll
      for (int j = 0; j < Q; ++j) {
        lo[j] = (l >> (8 * j)) & 0xff;
        hi[j] = (h >> (8 * j)) & 0xff;
        ok[j] = window_ok(lo[j], hi[j], J.Z);
        nbad += ok[j] ? 0 : 1;
        wl = ok[j] ? max(wl, hi[j] - lo[j] + 1) : wl;
      }
      if (nbad) atomicAdd(&a.ws.hdr[kHdrInvalid], (unsigned)nbad);
      uni = false;
    }
    const int WMw = __reduce_max_sync(kFull, wl);
    bool stiff[Q];
#pragma unroll
    for (int j = 0; j < Q; ++j) stiff[j] = false;
    const StagedF32& tab = tabs[jid];
    // Cold chunks: every cell has w < 2 or |E| below the field at which its
    // largest window rate reaches 2^kColdLog2.  The series would take no
    // term (2 W dt <= kThrF32[0]), so the step leaves N as it is and frees
    // no electron: dne is written, and k_lo/k_hi where the window rule
    // (the paper's slide, or the adaptive rule on the loaded planes) moves
    // the window.
    bool cold = WMw <= 1;
    if (!cold) {
      bool c = true;
#pragma unroll
      for (int j = 0; j < Q; ++j)
        c = c && (!ok[j] || hi[j] == lo[j] ||
                  fabsf(Ev[j]) < tab.ecold[min(lo[j], ION_MAX_Z)]);
      cold = __all_sync(kFull, c);
    }
    if (cold) {
      float* D = static_cast<float*>(J.dne);
      if (uni && J.vec) {
        float z[Q];
#pragma unroll
        for (int j = 0; j < Q; ++j) z[j] = 0.0f;
        vstore(D + c0, z);
      }
#pragma unroll
      for (int j = 0; j < Q; ++j) {
        if (!ok[j]) continue;
        if (!(uni && J.vec)) __stcs(D + c0 + j, 0.0f);
        if constexpr (AD) {
          if ((a.pol.flags & ION_NO_WINDOW_UPDATE) == 0 && hi[j] > lo[j]) {
            float v[ION_MAX_WINDOW];
#pragma unroll
            for (int r = 0; r < ION_MAX_WINDOW; ++r) v[r] = vget(st.P[r][lane], j);
            int nl = lo[j], nh = hi[j];
            adapt_window<float, ION_MAX_WINDOW>(v, hi[j] - lo[j] + 1, J.Z, a.pol.eps_f,
                                                a.pol.wmin, a.pol.wmax, a.pol.eps_grow_f, nl, nh);
            if (nl != lo[j] || nh != hi[j]) {
              J.lo[c0 + j] = (uint8_t)nl;
              J.hi[c0 + j] = (uint8_t)nh;
            }
          }
        } else if ((a.pol.flags & ION_NO_WINDOW_UPDATE) == 0 && hi[j] > lo[j] &&
                   hi[j] < J.Z && vget(st.P[0][lane], j) < a.pol.eps_f) {
          float v[ION_MAX_WINDOW];
#pragma unroll
          for (int r = 0; r < ION_MAX_WINDOW; ++r) v[r] = vget(st.P[r][lane], j);
          int nl = lo[j], nh = hi[j];
          slide_window<float, ION_MAX_WINDOW>(v, hi[j] - lo[j] + 1, J.Z, a.pol.eps_f, nl, nh);
          J.lo[c0 + j] = (uint8_t)nl;
          J.hi[c0 + j] = (uint8_t)nh;
        }
      }
    } else if (WMw == 2) {
      easy_cells<Q, 2, AD, CONS>(J, a.pol, tab, st.P, lane, c0, Ev, lo, hi, ok, uni, stiff,
                                     thr_lane, cmax);
    } else if (WMw <= 4) {
      easy_cells<Q, 4, AD, CONS>(J, a.pol, tab, st.P, lane, c0, Ev, lo, hi, ok, uni, stiff,
                                     thr_lane, cmax);
    } else {
      easy_cells<Q, 6, AD, CONS>(J, a.pol, tab, st.P, lane, c0, Ev, lo, hi, ok, uni, stiff,
                                     thr_lane, cmax);
    }
    // stiff cells: their inputs (as loaded) go to the record queue
    append_records<Q>(a.ws, jid, c0, Ev, lo, hi, stiff, st.P, lane);
    __syncwarp();
  }
  cp_async_wait<0>();
  if constexpr (CONS) warp_max_into(&a.ws.hdr[kHdrCons], cmax);

  tail_records(a, kChunk, gw, TW, lane);
}

// ---------------------------------------------------------------------------
// ion_lean_kernel<Q, W>: the streaming kernel for one species under the
// paper's window rule (ion_step's common case) with less bookkeeping per
// chunk than ion_stream_kernel.  The cell arithmetic is the same
// (easy_cells, records for stiff cells, the cold-chunk rule).
//   * A warp's runs of four chunks fill its four stages in order, so the
//     chunk of a stage follows from three run bases kept in registers: the
//     run being computed, the one whose planes are requested and the one
//     whose |E| and windows are requested.  Nothing is stored per stage.
//   * |E|, k_lo and k_hi of a chunk arrive as 16-byte copies, one per lane
//     (lanes [0, 8Q) |E|, then k_lo, then k_hi), each lane's source moving
//     by a fixed stride from chunk to chunk.
//   * Whether a chunk is cold is decided when its planes are requested (its
//     |E| and windows are then in shared memory).  A cold chunk brings in
//     only the lowest window plane of each cell, which is what the slide
//     test reads; where that state holds less than eps_shift the planes
//     above it are read directly.
//   * Element offsets into the planes are 32-bit ((Z+1) ld < 2^32).
// ---------------------------------------------------------------------------
template <int Q>
struct LStage {
  using V = typename VecOf<Q>::T;
  V E[32];                  // |E| of the chunk's 32 Q cells, Q per lane
  uint8_t lo[32 * Q];       // k_lo
  uint8_t hi[32 * Q];       // k_hi
  V P[ION_MAX_WINDOW][32];  // P[r][lane] component j = N[lo_j + r] of cell j
};
static_assert(sizeof(LStage<1>) % 16 == 0 && sizeof(LStage<2>) % 16 == 0,
              "stages keep the 16-byte alignment of the front copies");

template <int Q, int W>
constexpr size_t lean_smem() {
  return sizeof(StagedF32) + (size_t)W * kStages * sizeof(LStage<Q>);
}

template <int Q, int W, bool CONS>
__global__ void __maxnreg__(stream_regs<Q>())
    ion_lean_kernel(const __grid_constant__ BatchArgs a) {
  static_assert(Q == 1 || Q == 2, "one 16-byte front copy per lane at most");
  static_assert(kRun == kStages, "a run of chunks fills the stages in order");
  using V = typename VecOf<Q>::T;
  extern __shared__ __align__(16) unsigned char smem[];
  StagedF32& tab = *reinterpret_cast<StagedF32*>(smem);
  LStage<Q>* ring = reinterpret_cast<LStage<Q>*>(smem + sizeof(StagedF32));
  const JobIO& J = a.job[0];
  stage_f32(J.tab, a.pol.log2dt, &tab);
  if (threadIdx.x < 32) stage_cold(J.tab, a.pol.log2dt, kColdLog2, tab.ecold, threadIdx.x);
  {
    // plane slots past a cell's window are read (and ignored); keep them
    // finite
    float* z = reinterpret_cast<float*>(ring);
    const int nz = (int)(W * kStages * sizeof(LStage<Q>) / sizeof(float));
    for (int i = threadIdx.x; i < nz; i += blockDim.x) z[i] = 0.0f;
  }
  __syncthreads();

  constexpr int kChunk = 32 * Q;
  constexpr uint32_t kStageBytes = sizeof(LStage<Q>);
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  LStage<Q>* S = ring + wib * kStages;
  const uint32_t s_base = (uint32_t)__cvta_generic_to_shared(S);
  const int gw = blockIdx.x * W + wib;
  const int TW = gridDim.x * W;
  const uint32_t nchunks = (uint32_t)a.nchunks;
  const float* __restrict__ Nf = static_cast<const float*>(J.N);
  const uint32_t ld = (uint32_t)J.ld;
  const int Z = J.Z;

  // this lane's front copy: its source at chunk 0, the source's stride per
  // chunk and its offset in a stage
  const bool f_on = lane < 12 * Q;
  const char* f_src;
  uint32_t f_stride, f_dst;
  if (lane < 8 * Q) {
    f_src = static_cast<const char*>(J.E) + 16 * lane;
    f_stride = 4 * kChunk;
    f_dst = (uint32_t)offsetof(LStage<Q>, E) + 16 * lane;
  } else if (lane < 10 * Q) {
    f_src = reinterpret_cast<const char*>(J.lo) + 16 * (lane - 8 * Q);
    f_stride = kChunk;
    f_dst = (uint32_t)offsetof(LStage<Q>, lo) + 16 * (lane - 8 * Q);
  } else {
    f_src = reinterpret_cast<const char*>(J.hi) + 16 * (lane - 10 * Q);
    f_stride = kChunk;
    f_dst = (uint32_t)offsetof(LStage<Q>, hi) + 16 * (lane - 10 * Q);
  }
  const uint32_t p_dst = (uint32_t)offsetof(LStage<Q>, P) + (uint32_t)sizeof(V) * lane;

  uint32_t* const next = &a.ws.hdr[kHdrChunk];
  auto fetch_run = [&]() -> uint32_t {
    uint32_t b = 0;
    if (lane == 0) b = atomicAdd(next, (unsigned)kRun);
    return __shfl_sync(kFull, b, 0);
  };
  auto issue_front = [&](int s, uint32_t g) {
    if (g < nchunks && f_on)
      cp_async_s<16>(s_base + s * kStageBytes + f_dst, f_src + (size_t)g * f_stride);
    cp_async_commit();
  };
  // bit s: the chunk in stage s is cold (every cell below its cold field)
  uint32_t coldm = 0;
  auto issue_planes = [&](int s, uint32_t g) {
    if (g < nchunks) {
      const LStage<Q>& st = S[s];
      const uint32_t l = lane_bytes<Q>(reinterpret_cast<const uint32_t*>(st.lo), lane);
      const uint32_t h = lane_bytes<Q>(reinterpret_cast<const uint32_t*>(st.hi), lane);
      const V e = st.E[lane];
      int lo[Q], w[Q];
      bool c = true;
#pragma unroll
      for (int j = 0; j < Q; ++j) {
        lo[j] = (l >> (8 * j)) & 0xff;
        const int hj = (h >> (8 * j)) & 0xff;
        w[j] = window_ok(lo[j], hj, Z) ? hj - lo[j] + 1 : 0;
        c = c && (w[j] <= 1 || fabsf(vget(e, j)) < tab.ecold[min(lo[j], ION_MAX_Z)]);
      }
      const bool cold = __all_sync(kFull, c);
      coldm = cold ? (coldm | (1u << s)) : (coldm & ~(1u << s));
      const uint32_t c0 = g * (uint32_t)kChunk + (uint32_t)(Q * lane);
      const uint32_t pd = s_base + s * kStageBytes + p_dst;
      if (bytes_equal<Q>(l) && bytes_equal<Q>(h)) {
        uint32_t off = (uint32_t)lo[0] * ld + c0;
        if (cold) {
          // the lowest plane alone (the window rule's)
          if (w[0] >= 1) cp_async_s<4 * Q>(pd, Nf + off);
        } else {
#pragma unroll
          for (int r = 0; r < ION_MAX_WINDOW; ++r) {
            if (r < w[0]) cp_async_s<4 * Q>(pd + r * 32 * (uint32_t)sizeof(V), Nf + off);
            off += ld;
          }
        }
      } else {
#pragma unroll
        for (int j = 0; j < Q; ++j) {
          const int rows = cold ? min(w[j], 1) : w[j];
          uint32_t off = (uint32_t)lo[j] * ld + c0 + j;
          for (int r = 0; r < rows; ++r) {
            cp_async_s<4>(pd + r * 32 * (uint32_t)sizeof(V) + 4 * j, Nf + off);
            off += ld;
          }
        }
      }
    }
    cp_async_commit();
  };

  const float thr_lane = lane < kEasyTerms ? kThrF32[lane] : __int_as_float(0x7f800000);
  uint32_t cmax = 0;  // largest |change of sum_k N_k| (bits), ION_CONSERVATION_CHECK
  // Chunk k lives in stage k mod 4, and the wait discipline is that of
  // ion_stream_kernel: fronts three chunks ahead, planes two.
  uint32_t run_next = fetch_run();
  uint32_t run_mid = run_next, run_cur = run_next;
  issue_front(0, run_next);
  issue_front(1, run_next + 1);
  issue_front(2, run_next + 2);
  cp_async_wait<2>();
  __syncwarp();
  issue_planes(0, run_mid);
  cp_async_wait<2>();
  __syncwarp();
  issue_planes(1, run_mid + 1);
  for (int k = 0;; ++k) {
    const int s3 = (k + 3) & 3, s2 = (k + 2) & 3, s0 = k & 3;
    if (s3 == 0) run_next = fetch_run();
    issue_front(s3, run_next + s3);
    cp_async_wait<2>();  // front(k+2) and planes(k)
    __syncwarp();
    if (s2 == 0) run_mid = run_next;
    issue_planes(s2, run_mid + s2);
    if (s0 == 0) run_cur = run_mid;
    const uint32_t g = run_cur + s0;
    if (g >= nchunks) break;  // runs come in increasing order: no more

    const LStage<Q>& st = S[s0];
    const int c0 = (int)(g * (uint32_t)kChunk) + Q * lane;
    const V e = st.E[lane];
    float Ev[Q];
#pragma unroll
    for (int j = 0; j < Q; ++j) Ev[j] = vget(e, j);
    const uint32_t l = lane_bytes<Q>(reinterpret_cast<const uint32_t*>(st.lo), lane);
    const uint32_t h = lane_bytes<Q>(reinterpret_cast<const uint32_t*>(st.hi), lane);
    int lo[Q], hi[Q], wl = 0;
    bool ok[Q];
    bool uni;
    if (bytes_equal<Q>(l) && bytes_equal<Q>(h)) {
      const int l0 = l & 0xff, h0 = h & 0xff;
      const bool o = window_ok(l0, h0, Z);
#pragma unroll
      for (int j = 0; j < Q; ++j) {
        lo[j] = l0;
        hi[j] = h0;
        ok[j] = o;
      }
      wl = o ? h0 - l0 + 1 : 0;
      if (!o) atomicAdd(&a.ws.hdr[kHdrInvalid], (unsigned)Q);
      uni = o;
    } else {
      int nbad = 0;
#pragma unroll
      for (int j = 0; j < Q; ++j) {
        lo[j] = (l >> (8 * j)) & 0xff;
        hi[j] = (h >> (8 * j)) & 0xff;
        ok[j] = window_ok(lo[j], hi[j], Z);
        nbad += ok[j] ? 0 : 1;
        wl = ok[j] ? max(wl, hi[j] - lo[j] + 1) : wl;
      }
      if (nbad) atomicAdd(&a.ws.hdr[kHdrInvalid], (unsigned)nbad);
      uni = false;
    }
    bool stiff[Q];
#pragma unroll
    for (int j = 0; j < Q; ++j) stiff[j] = false;
    if ((coldm >> s0) & 1u) {
      // Cold chunk: N stays as it is and no electron is freed (the series
      // would take no term); dne is written, and k_lo/k_hi where the window
      // slides.
      float* D = static_cast<float*>(J.dne);
      if (uni) {
        float z[Q];
#pragma unroll
        for (int j = 0; j < Q; ++j) z[j] = 0.0f;
        vstore(D + c0, z);
      }
#pragma unroll
      for (int j = 0; j < Q; ++j) {
        if (!ok[j]) continue;
        if (!uni) __stcs(D + c0 + j, 0.0f);
        const float p0 = vget(st.P[0][lane], j);
        if ((a.pol.flags & ION_NO_WINDOW_UPDATE) == 0 && hi[j] > lo[j] && hi[j] < Z &&
            p0 < a.pol.eps_f) {
          // the planes above the lowest were not brought in: read them
          float v[ION_MAX_WINDOW];
          v[0] = p0;
          const float* p = Nf + (uint32_t)lo[j] * ld + (uint32_t)(c0 + j);
#pragma unroll
          for (int r = 1; r < ION_MAX_WINDOW; ++r)
            v[r] = r < hi[j] - lo[j] ? p[(uint32_t)r * ld] : 0.0f;
          int nl = lo[j], nh = hi[j];
          slide_window<float, ION_MAX_WINDOW>(v, hi[j] - lo[j] + 1, Z, a.pol.eps_f, nl, nh);
          J.lo[c0 + j] = (uint8_t)nl;
          J.hi[c0 + j] = (uint8_t)nh;
        }
      }
    } else {
      const int WMw = __reduce_max_sync(kFull, wl);
      if (WMw <= 2)
        easy_cells<Q, 2, false, CONS>(J, a.pol, tab, st.P, lane, c0, Ev, lo, hi, ok, uni,
                                       stiff, thr_lane, cmax);
      else if (WMw <= 4)
        easy_cells<Q, 4, false, CONS>(J, a.pol, tab, st.P, lane, c0, Ev, lo, hi, ok, uni,
                                       stiff, thr_lane, cmax);
      else
        easy_cells<Q, 6, false, CONS>(J, a.pol, tab, st.P, lane, c0, Ev, lo, hi, ok, uni,
                                       stiff, thr_lane, cmax);
      // stiff cells: their inputs (as loaded) go to the record queue
      append_records<Q>(a.ws, 0, c0, Ev, lo, hi, stiff, st.P, lane);
    }
    __syncwarp();
  }
  cp_async_wait<0>();
  if constexpr (CONS) warp_max_into(&a.ws.hdr[kHdrCons], cmax);

  tail_records(a, kChunk, gw, TW, lane);
}

// The stiff-cell records, one per thread.  W bounds the width; the window
// planes past the cell's own width are zero.
template <int W>
__device__ __forceinline__ bool record_cell(const BatchArgs& a, const StagedF32& tab,
                                            const JobIO& J, int64_t i, int c, float Ec,
                                            int lo, int hi, float* change) {
  float v[W];
  const int w = hi - lo + 1;
#pragma unroll
  for (int r = 0; r < W; ++r)
    v[r] = r < w ? __ldcs(a.ws.rec_V + (int64_t)r * a.ws.rec_cap + i) : 0.0f;
  return finish_cell<F32Form, W>(J, a.pol, tab, c, Ec, lo, hi, v, true, change);
}

__global__ void __launch_bounds__(256, 3)
    ion_stiff_kernel(const __grid_constant__ BatchArgs a) {
  __shared__ StagedF32 tabs[kMaxJobs];
  // narrow records at [0, nn), wide ones at [cap - nw, cap); thread t < nn_up
  // takes narrow record t, t >= nn_up wide record cap - 1 - (t - nn_up)
  // (both counts rounded up to whole warps, so each warp sees one class)
  const unsigned nn = *((volatile unsigned*)&a.ws.hdr[kHdrRecNarrow]);
  const unsigned nw = *((volatile unsigned*)&a.ws.hdr[kHdrRecWide]);
  if (blockIdx.x == 0 && threadIdx.x == 0) a.ws.hdr[kHdrStiff] = nn + nw;
  const unsigned stride = gridDim.x * blockDim.x;
  const unsigned nn_up = (nn + 31u) & ~31u;
  const unsigned n_up = nn_up + ((nw + 31u) & ~31u);
  if (blockIdx.x * blockDim.x >= n_up) return;  // no record for this block
  for (int j = 0; j < a.njobs; ++j) stage_f32(a.job[j].tab, a.pol.log2dt, &tabs[j]);
  __syncthreads();
  const bool check = (a.pol.flags & ION_CONSERVATION_CHECK) != 0;
  uint32_t cmax = 0;  // largest |change of sum_k N_k| (bits)
  for (unsigned t = blockIdx.x * blockDim.x + threadIdx.x; t < n_up; t += stride) {
    const bool wide = t >= nn_up;  // warp-uniform
    const unsigned i = wide ? (unsigned)a.ws.rec_cap - 1u - (t - nn_up) : t;
    const bool have = wide ? t - nn_up < nw : t < nn;
    bool fb = false;
    int c = 0, jid = 0, lo = 0, hi = -1;
    float Ec = 0.0f;
    if (have) {
      c = (int)__ldcs(a.ws.rec_c + i);
      jid = a.ws.rec_job[i];
      Ec = __ldcs(a.ws.rec_E + i);
      const unsigned lh = __ldcs(a.ws.rec_lohi + i);
      lo = lh & 0xff;
      hi = lh >> 8;
    }
    // the warp's widest window picks the width bound for all its lanes
    // (fewer code paths, no divergence by width)
    const int wl = hi - lo + 1;
    const int Wm = __reduce_max_sync(kFull, wl);
    if (wl >= 1) {
      const JobIO& J = a.job[jid];
      const StagedF32& tab = tabs[jid];
      // (a bound of 5 for warps of 5-state windows measured slower: the
      // extra instantiation costs more than its shorter table saves)
      static_assert(kRecNarrow == 4, "width bounds of the two record classes");
      float d = 0.0f;
      float* dp = check ? &d : nullptr;
      if (wide) {
        fb = record_cell<6>(a, tab, J, i, c, Ec, lo, hi, dp);
      } else if (wl == 1) {
        fb = record_cell<1>(a, tab, J, i, c, Ec, lo, hi, dp);
      } else if (Wm <= 2) {
        fb = record_cell<2>(a, tab, J, i, c, Ec, lo, hi, dp);
      } else {
        fb = record_cell<4>(a, tab, J, i, c, Ec, lo, hi, dp);
      }
      cmax = max(cmax, abs_bits(d));
    }
    warp_append(&a.ws.hdr[kHdrFallback], a.ws.queue, a.ws.queue_job, fb, (uint32_t)c,
                (uint8_t)jid);
  }
  if (check) warp_max_into(&a.ws.hdr[kHdrCons], cmax);
}

// ---------------------------------------------------------------------------
// FP64-coefficient pass over the queued cells, one cell per thread.
// ---------------------------------------------------------------------------
// WM bounds the window width w = hi - lo + 1 (the planes past w are zero).
// Returns, with ION_CONSERVATION_CHECK, |sum_r v'_r - sum_r v_r| of the
// window as stored (the inputs summed in FP64 exactly enough: w <= 6 floats).
template <int WM>
__device__ __forceinline__ float fb_cell(const JobIO& J, const Policy& pol,
                                         const StagedF32& tab, int c, int lo, int hi) {
  float* __restrict__ N = static_cast<float*>(J.N);
  const FieldF32 f = field_f32(static_cast<const float*>(J.E)[c]);
  const int w = hi - lo + 1;
  double v[WM], lam[WM];
#pragma unroll
  for (int r = 0; r < WM; ++r) {
    v[r] = r < w ? (double)N[(int64_t)(lo + r) * J.ld + c] : 0.0;
    lam[r] = (r < w - 1 && !pol.zero_dt) ? (double)rate_dt_f32(tab, lo + r, f) : 0.0;
  }
  double s0 = 0.0;
#pragma unroll
  for (int r = 0; r < WM; ++r) s0 += v[r];
  const double dne = dd_update<double, WM>(v, lam, w);
  float vf[WM];
  double s1 = 0.0;
#pragma unroll
  for (int r = 0; r < WM; ++r) {
    vf[r] = __double2float_rn(v[r]);
    if (r < w) N[(int64_t)(lo + r) * J.ld + c] = vf[r];
    s1 += (double)vf[r];
  }
  int nlo = lo, nhi = hi;
  window_after_step<float, WM>(J, pol, vf, w, nlo, nhi);
  const float* G = static_cast<const float*>(J.n_gas);
  const float d = __double2float_rn(dne);
  static_cast<float*>(J.dne)[c] = G ? d * G[c] : d;
  J.lo[c] = (uint8_t)nlo;
  J.hi[c] = (uint8_t)nhi;
  return (float)fabs(s1 - s0);
}

// The queue is dealt out a warp at a time across the blocks (warp k of the
// grid takes entries 32k..32k+31, and warp k sits in block k mod grid), so
// that a short queue spreads over as many SMs as it has warps: the FP64 pipe
// is the bound here, and each SM has its own.  Each warp runs the
// instantiation of its widest window, so its lanes do not diverge by width.
__global__ void __launch_bounds__(128) ion_fb_kernel(const __grid_constant__ BatchArgs a) {
  __shared__ StagedF32 tabs[kMaxJobs];
  const unsigned n = *((volatile unsigned*)&a.ws.hdr[kHdrFallback]);
  const unsigned warps = gridDim.x * (blockDim.x / 32u);
  const unsigned wid = (threadIdx.x / 32u) * gridDim.x + blockIdx.x;  // warp of the grid
  const unsigned lane = threadIdx.x & 31u;
  if (blockIdx.x * 32u >= n) return;  // no queued cell for this block
  for (int j = 0; j < a.njobs; ++j) stage_f32(a.job[j].tab, a.pol.log2dt, &tabs[j]);
  __syncthreads();
  uint32_t cmax = 0;  // largest |change of sum_k N_k| (bits), ION_CONSERVATION_CHECK
  for (unsigned base = wid * 32u; base < n; base += warps * 32u) {  // warp-uniform
    const unsigned i = base + lane;
    int c = 0, jid = 0, lo = 0, hi = -1;
    if (i < n) {
      c = (int)a.ws.queue[i];
      jid = a.ws.queue_job[i];
      lo = a.job[jid].lo[c];
      hi = a.job[jid].hi[c];
    }
    const int Wm = __reduce_max_sync(kFull, hi - lo + 1);
    float d = 0.0f;
    if (hi >= lo) {
      const JobIO& J = a.job[jid];
      const StagedF32& tab = tabs[jid];
      if (Wm <= 2)
        d = fb_cell<2>(J, a.pol, tab, c, lo, hi);
      else if (Wm == 3)
        d = fb_cell<3>(J, a.pol, tab, c, lo, hi);
      else if (Wm == 4)
        d = fb_cell<4>(J, a.pol, tab, c, lo, hi);
      else if (Wm == 5)
        d = fb_cell<5>(J, a.pol, tab, c, lo, hi);
      else
        d = fb_cell<6>(J, a.pol, tab, c, lo, hi);
    }
    cmax = max(cmax, abs_bits(d));
  }
  if (a.pol.flags & ION_CONSERVATION_CHECK) warp_max_into(&a.ws.hdr[kHdrCons], cmax);
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
// One instantiation of the streaming kernel: its function and smem needs.
struct StreamVariant {
  const void* fn;
  int Q, W;
  bool adaptive;
  bool lean;  // ion_lean_kernel (one species, the paper's window rule)
  bool cons;  // ION_CONSERVATION_CHECK
  size_t (*smem)(int);
};

template <int Q, int W>
size_t smem_of(int njobs) {
  return stream_smem<Q, W>(njobs);
}

template <int Q, int W>
size_t lean_smem_of(int) {
  return lean_smem<Q, W>();
}

#define ION_VARIANT(Q, W, AD, C)                                                     \
  {                                                                                  \
    reinterpret_cast<const void*>(&ion_stream_kernel<Q, W, AD, C>), Q, W, AD, false, C, \
        &smem_of<Q, W>                                                               \
  }
#define ION_VARIANTS(AD, C)                                                       \
  ION_VARIANT(1, 2, AD, C), ION_VARIANT(1, 4, AD, C), ION_VARIANT(1, 8, AD, C),    \
      ION_VARIANT(2, 2, AD, C), ION_VARIANT(2, 4, AD, C), ION_VARIANT(2, 8, AD, C), \
      ION_VARIANT(4, 2, AD, C), ION_VARIANT(4, 4, AD, C), ION_VARIANT(4, 8, AD, C)
#define ION_LEAN(Q, W, C)                                                              \
  {                                                                                    \
    reinterpret_cast<const void*>(&ion_lean_kernel<Q, W, C>), Q, W, false, true, C,      \
        &lean_smem_of<Q, W>                                                            \
  }
#define ION_LEANS(C)                                                              \
  ION_LEAN(1, 2, C), ION_LEAN(1, 4, C), ION_LEAN(1, 8, C), ION_LEAN(2, 2, C),      \
      ION_LEAN(2, 4, C), ION_LEAN(2, 8, C)
const StreamVariant kVariants[] = {ION_VARIANTS(false, false), ION_VARIANTS(true, false),
                                   ION_VARIANTS(false, true),  ION_VARIANTS(true, true),
                                   ION_LEANS(false),           ION_LEANS(true)};
#undef ION_LEANS
#undef ION_LEAN
#undef ION_VARIANTS
#undef ION_VARIANT

const StreamVariant* find_variant(int Q, int W, bool adaptive = false, bool lean = false,
                                  bool cons = false) {
  for (const auto& v : kVariants)
    if (v.Q == Q && v.W == W && v.adaptive == adaptive && v.lean == lean && v.cons == cons)
      return &v;
  return nullptr;
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// The lean kernel serves a launch of one species under the paper's window
// rule whose arrays allow its copies: 16-byte aligned |E|, k_lo and k_hi,
// vector-aligned planes, and plane offsets that fit 32 bits.
bool lean_fits(const BatchArgs& a, int Q) {
  if (a.njobs != 1 || a.pol.adaptive || (Q != 1 && Q != 2)) return false;
  const JobIO& J = a.job[0];
  return J.vec && aligned16(J.E) && aligned16(J.lo) && aligned16(J.hi) &&
         (uint64_t)(J.Z + 1) * (uint64_t)J.ld < (uint64_t(1) << 32);
}

// Resident blocks per SM of a variant with `njobs` staged tables, set up and
// measured once per (device, variant, njobs): later calls (and calls made
// while a stream is being captured) only read the cache.
constexpr int kMaxDevices = 64;
constexpr int kNumVariants = sizeof(kVariants) / sizeof(kVariants[0]);
std::mutex g_fit_mu;
int g_fit[kMaxDevices][kNumVariants][kMaxJobs + 1];  // 0: not measured yet

cudaError_t resident_blocks(const StreamVariant& v, int njobs, size_t smem, int* fit) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const int vi = (int)(&v - kVariants);
  const bool cache = dev >= 0 && dev < kMaxDevices;
  std::lock_guard<std::mutex> lock(g_fit_mu);
  if (cache && g_fit[dev][vi][njobs] > 0) {
    *fit = g_fit[dev][vi][njobs];
    return cudaSuccess;
  }
  // the opt-in limit covers every job count, so no later call lowers it
  // under a launch that needs more
  if ((e = cudaFuncSetAttribute(v.fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)v.smem(kMaxJobs))) != cudaSuccess)
    return e;
  if ((e = cudaFuncSetAttribute(v.fn, cudaFuncAttributePreferredSharedMemoryCarveout,
                                cudaSharedmemCarveoutMaxShared)) != cudaSuccess)
    return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(fit, v.fn, v.W * 32, smem)) !=
      cudaSuccess)
    return e;
  if (cache && *fit > 0) g_fit[dev][vi][njobs] = *fit;
  return cudaSuccess;
}

}  // namespace

LaunchShape default_shape() { return {2, 8, 0}; }

bool valid_shape(const LaunchShape& s) {
  return find_variant(s.cells_per_lane, s.warps_per_block) != nullptr &&
         s.blocks_per_sm >= 0 && s.blocks_per_sm <= 32;
}

size_t step_workspace_bytes(int64_t ncells, bool f64) {
  return f64 ? kHdrBytes : f32_workspace_bytes((size_t)ncells);
}

void bind_workspace(Scratch& s, void* ws, int64_t ncells) {
  char* p = static_cast<char*>(ws);
  const size_t n = (size_t)ncells;
  s.hdr = reinterpret_cast<uint32_t*>(p);
  p += kHdrBytes;
  s.queue = reinterpret_cast<uint32_t*>(p);
  p += round256(4 * n);
  s.queue_job = reinterpret_cast<uint8_t*>(p);
  p += round256(n);
  s.rec_c = reinterpret_cast<uint32_t*>(p);
  p += round256(4 * n);
  s.rec_job = reinterpret_cast<uint8_t*>(p);
  p += round256(n);
  s.rec_E = reinterpret_cast<float*>(p);
  p += round256(4 * n);
  s.rec_lohi = reinterpret_cast<uint16_t*>(p);
  p += round256(2 * n);
  s.rec_V = reinterpret_cast<float*>(p);
  s.rec_cap = (int64_t)n;
}

cudaError_t launch_batch_f32(BatchArgs& a, const LaunchShape& shape, int num_sms,
                             cudaStream_t s) {
  const StreamVariant* v =
      find_variant(shape.cells_per_lane, shape.warps_per_block, a.pol.adaptive != 0,
                   lean_fits(a, shape.cells_per_lane),
                   (a.pol.flags & ION_CONSERVATION_CHECK) != 0);
  if (!v) return cudaErrorInvalidValue;
  cudaError_t e = cudaMemsetAsync(a.ws.hdr, 0, kHdrWords * sizeof(uint32_t), s);
  if (e != cudaSuccess) return e;
  const int chunk = 32 * v->Q;
  int total = 0, cells = 0;
  for (int j = 0; j < a.njobs; ++j) {
    a.job[j].chunk0 = total;
    total += a.job[j].ncells / chunk;
    cells += a.job[j].ncells;
  }
  a.nchunks = total;
  if (cells == 0) return cudaSuccess;
  const size_t smem = v->smem(a.njobs);
  int fit = 0;
  if ((e = resident_blocks(*v, a.njobs, smem, &fit)) != cudaSuccess) return e;
  if (fit < 1) return cudaErrorInvalidConfiguration;
  const int per_sm = shape.blocks_per_sm > 0 && shape.blocks_per_sm < fit ? shape.blocks_per_sm
                                                                          : fit;
  const int64_t need = ((int64_t)total + v->W - 1) / v->W;
  int blocks = (int)(need < (int64_t)per_sm * num_sms ? need : (int64_t)per_sm * num_sms);
  if (blocks < 1) blocks = 1;  // the tails still need a warp
  void* args[] = {&a};
  if ((e = cudaLaunchKernel(v->fn, blocks, v->W * 32, args, smem, s)) != cudaSuccess) return e;
  if ((e = launch_stiff_f32(a, num_sms, s)) != cudaSuccess) return e;
  return launch_fb_f32(a, num_sms, s);
}

// The record kernel's grid is one wave of resident blocks: a second, partial
// wave would start its share of the records only after the first finished.
int g_stiff_fit[kMaxDevices] = {};

cudaError_t launch_stiff_f32(const BatchArgs& a, int num_sms, cudaStream_t s) {
  int dev = 0, fit = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const bool cache = dev >= 0 && dev < kMaxDevices;
  {
    std::lock_guard<std::mutex> lock(g_fit_mu);
    if (cache) fit = g_stiff_fit[dev];
    if (fit < 1) {
      if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fit, ion_stiff_kernel, 256, 0)) !=
          cudaSuccess)
        return e;
      fit = fit < 1 ? 1 : fit;
      if (cache) g_stiff_fit[dev] = fit;
    }
  }
  ion_stiff_kernel<<<fit * num_sms, 256, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_fb_f32(const BatchArgs& a, int num_sms, cudaStream_t s) {
  const bool need_fb = (a.pol.flags & ION_NO_FP64_FALLBACK) == 0 &&
                       ((a.pol.flags & ION_FORCE_FP64_COEF) != 0 || a.pol.gap > 0.0);
  if (!need_fb) return cudaSuccess;
  ion_fb_kernel<<<2 * num_sms, 128, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace ion
