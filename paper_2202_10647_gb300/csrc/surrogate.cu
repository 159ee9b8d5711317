// surrogate.cu -- the rate surrogate at inference on the tensor cores.
//
// One CTA of 128 threads owns a tile of 128 cells at a time (thread t <->
// cell t of the tile <-> row t of the MMAs <-> lane t of tensor memory):
//   1. each thread evaluates layer 1 of its cell (one input, 64 GELUs),
//      splits h1 into bf16 pairs, hi = bf16(h1) and lo = bf16(h1 - hi) (the
//      weights are split the same way), and stores both parts in its lane
//      of tensor memory (tcgen05.st), where the MMAs read the A operand;
//   2. one thread issues layer 2 as 12 128x64x16 tcgen05.mma (per 16-wide
//      slice of K: A_hi W_hi + A_hi W_lo + A_lo W_hi; A from tensor memory,
//      the weights from shared memory, FP32 accumulators in tensor memory)
//      and commits them to an mbarrier.  The products carry 16 significant
//      bits of every operand instead of bf16's 8, so the network's error is
//      its training error rather than bf16 rounding (a 1-64-64-18 network
//      on Ar-like rates: median rate error 0.5 % against 2 % with single
//      bf16 operands);
//   3. every thread reads its row of the accumulators (tcgen05.ld), adds b2,
//      applies the GELU and stores h2 (hi and lo) over h1;
//   4. layer 3 likewise (N = the output count padded to 16, 32, 48 or 64),
//      reusing the same accumulator columns;
//   5. the outputs, scaled to log2 W, are staged column-major in shared
//      memory (conflict-free for any window position), and each thread
//      finishes its cell: ion_surrogate_rates writes all Z rates;
//      ion_step_surrogate picks the window's rates (network or Eq. 1, by the
//      validation bound) and finishes cells whose rates all have W dt <= 1
//      with the Taylor form.  Cells with a larger rate become records for
//      ion_step's record kernel (Bateman form, rates of Eq. 1), followed by
//      its FP64-coefficient pass.
// Waits on the mbarrier are bounded; a wait that gives up marks the call as
// failed (header word / NaN rates), frees the tensor memory and returns.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <vector>

#include "ion_cell.cuh"
#include "ion_step.cuh"
#include "ionize.h"
#include "mlp_device.cuh"

namespace ion {
namespace sg {

using mlp::H;

constexpr int kM = 128;            // cells per tile = MMA M = threads per CTA
// Tensor memory per CTA: columns [0, 64) the accumulators (layer 3 reuses
// them), [64, 96) the hi parts of the A operand (two bf16 per 32-bit column,
// the lower K index in the low half), [96, 128) its lo parts.
constexpr uint32_t kTmemCols = 128;
constexpr uint32_t kColAhi = 64, kColAlo = 96;
constexpr uint32_t kSpinLimit = 1u << 22;

// Scalars and short vectors of the network and its scaling.
struct Consts {
  float W1h[H], b1h[H], b2h[H];  // W1, b1, b2 halved (the W2 image is halved too)
  float yoff[64], yscale[64];    // log2 W_k = yscale_k acc_k + yoff_k
  float xa, xb;        // x = xa log2|E| + xb
  float l2lo, l2hi;    // trusted log2|E| range
  float yfloor;        // log2 W below this: W = 0
  float bin_a, bin_b;  // bin = floor(bin_a log2|E| + bin_b)
  int nbins;
  int Z, KP;
  int dead_wait;  // test hook (ion_surrogate_test_timeout): see mbar_wait below
};

// Device image of a surrogate (one allocation).  Each weight is a pair of
// bf16 numbers (mlp::split_round): [0] the rounded value, [1] the rounded
// remainder.
struct Dev {
  uint8_t W2img[2][64 * 128];  // layer-2 B operands: 64 rows (units) x 64 bf16 (K)
  uint8_t W3img[2][64 * 128];  // layer-3 B operands: KP rows, zero-padded
  Consts k;
  SpeciesTable tab;
};

// Byte offset of element (row r, k) of a K-major bf16 tile with 64 elements
// (128 bytes) per row in the 128-byte swizzle: 8-row groups of 1024 bytes,
// the 16-byte chunk index XORed with the row within the group.
__host__ __device__ constexpr uint32_t sw128_offset(int r, int k) {
  return (uint32_t)((r >> 3) * 1024 + (r & 7) * 128 + ((((k >> 3) ^ (r & 7)) & 7) << 4) +
                    ((k & 7) << 1));
}

// ---- PTX wrappers ---------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor: start address, leading byte offset 16
// (unused by the swizzled K-major layout), stride byte offset 1024 (one
// 8-row group), descriptor version 1 (bit 46), 128-byte swizzle (2 << 61).
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)(16 >> 4) << 16) |
         ((uint64_t)(1024 >> 4) << 32) | ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// Instruction descriptor of kind::f16: FP32 accumulators (bit 4), bf16 A
// (bit 7) and B (bit 10), both K-major, N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
      : "memory");
}

// Bounded wait for the mbarrier phase with the given parity: false if the
// phase has not completed after `limit` polls.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity,
                                          uint32_t limit = kSpinLimit) {
  for (uint32_t i = 0; i < limit; ++i) {
    uint32_t done;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        "selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

// 16 accumulator columns of this thread's lane.  The wait takes the
// registers as operands so that no use is scheduled before it.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
      "%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
        "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]),
                 "+r"(r[6]), "+r"(r[7]), "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]),
                 "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15])
               :
               : "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);  // a in the low half
  return *reinterpret_cast<const uint32_t*>(&h);
}

// A pair of activations as bf16 pairs (mlp::split_round): hi holds
// bf16(a), bf16(b); lo holds the rounded remainders.
__device__ __forceinline__ void split2(float a, float b, uint32_t& hi, uint32_t& lo) {
  hi = pack_bf16(a, b);
  lo = pack_bf16(a - __uint_as_float(hi << 16), b - __uint_as_float(hi & 0xffff0000u));
}

// 8 columns of this thread's lane from 8 registers.
__device__ __forceinline__ void tmem_st8(uint32_t taddr, const uint32_t (&r)[8]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(taddr),
      "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7])
      : "memory");
}

__device__ __forceinline__ void tmem_wait_st() {
  asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

// D += A B with A (128 x 16 bf16) read from tensor memory at column a_tmem
// and B from shared memory.
__device__ __forceinline__ void mma_bf16_ta(uint32_t d_tmem, uint32_t a_tmem, uint64_t bdesc,
                                            uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}\n" ::"r"(d_tmem),
      "r"(a_tmem), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

// One layer's products for the 128-row tile once every thread has stored its
// row of the A operand (hi and lo parts) in tensor memory: per 16-wide slice
// kk of K, A_hi W_hi + A_hi W_lo + A_lo W_hi into the accumulators.  Every
// thread calls this; thread 0 issues.  Returns false if the bounded wait
// gave up (the tile is then skipped, and the CTA's drain waits for the
// commit in flight).  dead_first: the wait polls `sdead` instead (the test
// hook of ion_surrogate_test_timeout).
__device__ __forceinline__ bool layer_products(uint32_t tmem, uint32_t sBhi, uint32_t sBlo,
                                               uint32_t idesc, int t, uint32_t sbar,
                                               uint32_t& phase, bool dead_first,
                                               uint32_t sdead) {
  tmem_wait_st();
  tc_fence_before();
  __syncthreads();
  if (t == 0) {
    tc_fence_after();
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
      const uint32_t ahi = tmem + kColAhi + kk * 8, alo = tmem + kColAlo + kk * 8;
      mma_bf16_ta(tmem, ahi, sw128_desc(sBhi + kk * 32), idesc, kk > 0 ? 1u : 0u);
      mma_bf16_ta(tmem, ahi, sw128_desc(sBlo + kk * 32), idesc, 1u);
      mma_bf16_ta(tmem, alo, sw128_desc(sBhi + kk * 32), idesc, 1u);
    }
    mma_commit(sbar);
  }
  const bool ok = dead_first ? mbar_wait(sdead, 0u, 64u) : mbar_wait(sbar, phase);
  phase ^= 1u;
  if (__syncthreads_or(!ok)) return false;
  tc_fence_after();
  return true;
}

// ---- shared-memory plan ---------------------------------------------------
struct Plan {
  uint32_t y_bytes;  // output staging (KP x 128 floats)
  uint32_t w2, w3, consts, tab, bar, slot, total;
};

__host__ __device__ constexpr Plan plan_of(int KP) {
  Plan p{};
  p.y_bytes = (uint32_t)(KP * 512);
  p.w2 = p.y_bytes;            // W2 hi, then lo (8 KB each)
  p.w3 = p.w2 + 2 * 8192;      // W3 hi, then lo (KP x 128 bytes each)
  p.consts = p.w3 + 2 * (uint32_t)KP * 128;
  p.tab = p.consts + (uint32_t)((sizeof(Consts) + 15) / 16 * 16);
  p.bar = p.tab + (uint32_t)((sizeof(StagedF32) + 15) / 16 * 16);
  p.slot = p.bar + 16;  // two barriers: the MMA commits', and one never arrived at
  p.total = p.slot + 8 + 1024;  // + slack for aligning the base to 1024
  return p;
}

struct StepArgs {
  JobIO J;
  Policy pol;
  Scratch ws;
  float pop_tol;
  const float* bound;  // [nbins][Z] of 2^bound - 1, or nullptr
  float* W_out;        // rates mode
  int64_t ldw;
  int64_t ncells;
  const float* E;
};

// Taylor-form update of one cell whose rates all have W dt <= 1 (w <= WM,
// v its window's populations, zero past w): the same series, window slide
// and stores as ion_step's streaming kernel.  WM: the warp's width bound.
template <int WM>
__device__ __forceinline__ void taylor_cell(const StepArgs& a, int c, int lo, int hi,
                                            const float (&v6)[ION_MAX_WINDOW],
                                            const float (&lam6)[ION_MAX_WINDOW], float lmax) {
  const JobIO& J = a.J;
  float* __restrict__ N = static_cast<float*>(J.N);
  const int w = hi - lo + 1;
  float dne = 0.0f;
  int nlo = lo, nhi = hi;
  if (w >= 2) {
    float v[WM], lam[WM];
#pragma unroll
    for (int r = 0; r < WM; ++r) {
      v[r] = v6[r];
      lam[r] = lam6[r];
    }
    dne = taylor_propagate<float, WM>(v, lam, w, lmax);
    window_after_step<float, WM>(J, a.pol, v, w, nlo, nhi);
    float* q = N + (int64_t)lo * J.ld + c;
#pragma unroll
    for (int r = 0; r < WM; ++r) {
      if (r < w) __stcs(q, v[r]);
      q += J.ld;
    }
  }
  const float* __restrict__ G = static_cast<const float*>(J.n_gas);
  __stcs(static_cast<float*>(J.dne) + c, G ? dne * G[c] : dne);
  if (nlo != lo || nhi != hi) {
    J.lo[c] = (uint8_t)nlo;
    J.hi[c] = (uint8_t)nhi;
  }
}

// The rates of Eq. 1 for the window's w-1 transitions as ion_step's
// streaming kernel takes them: the plain FP32 exponent for every rate, the
// float-float recompute for those above 2^-6 (W dt).
__device__ __forceinline__ void eq1_rates(const StagedF32& tab, int lo, int w, float E,
                                          float (&lam)[ION_MAX_WINDOW]) {
  const FieldF32 f = field_f32(E);
#pragma unroll
  for (int r = 0; r < ION_MAX_WINDOW - 1; ++r) {
    if (r < w - 1 && !f.zero) {
      const float4 h = tab.hi[lo + r];
      const float q = h.z * f.rE;
      const float y = (fmaf(-h.y, f.lg, h.x) - q) + h.w;
      lam[r] = q <= (float)kCutoffLog2 ? ex2_approx(fminf(y, 99.0f)) : 0.0f;
    }
  }
#pragma unroll
  for (int r = 0; r < ION_MAX_WINDOW - 1; ++r)
    if (lam[r] > 1.0f / 64.0f) lam[r] = rate_ff_f32(tab, lo + r, f);
}

// Counts the lanes with `take` set into *counter (one atomic per warp).
__device__ __forceinline__ void warp_count(uint32_t* counter, bool take) {
  const unsigned m = __ballot_sync(kFull, take);
  if ((threadIdx.x & 31) == 0 && m) atomicAdd(counter, (unsigned)__popc(m));
}

template <bool Step, int KP>
__global__ void __launch_bounds__(kM) surrogate_kernel(const Dev* __restrict__ dev,
                                                       const __grid_constant__ StepArgs a) {
  extern __shared__ unsigned char smem_raw[];
  constexpr Plan P = plan_of(KP);
  // align the base to 1024 bytes (the swizzle atoms)
  const uint32_t raw = smem_u32(smem_raw);
  unsigned char* base = smem_raw + ((1024u - (raw & 1023u)) & 1023u);
  float* Y = reinterpret_cast<float*>(base);  // output staging Y[k][128]
  Consts& K = *reinterpret_cast<Consts*>(base + P.consts);
  StagedF32& tab = *reinterpret_cast<StagedF32*>(base + P.tab);
  uint64_t* bar = reinterpret_cast<uint64_t*>(base + P.bar);
  uint32_t* slot = reinterpret_cast<uint32_t*>(base + P.slot);
  const int t = threadIdx.x;
  const int warp = t >> 5;

  // stage the operands and constants
  {
    for (int h = 0; h < 2; ++h) {
      const uint4* s2 = reinterpret_cast<const uint4*>(dev->W2img[h]);
      uint4* d2 = reinterpret_cast<uint4*>(base + P.w2 + h * 8192);
      for (int i = t; i < 8192 / 16; i += kM) d2[i] = s2[i];
      const uint4* s3 = reinterpret_cast<const uint4*>(dev->W3img[h]);
      uint4* d3 = reinterpret_cast<uint4*>(base + P.w3 + h * KP * 128);
      for (int i = t; i < KP * 128 / 16; i += kM) d3[i] = s3[i];
    }
    const uint32_t* sc = reinterpret_cast<const uint32_t*>(&dev->k);
    uint32_t* dc = reinterpret_cast<uint32_t*>(&K);
    for (int i = t; i < (int)(sizeof(Consts) / 4); i += kM) dc[i] = sc[i];
    stage_f32(&dev->tab, a.pol.log2dt, &tab);
  }
  if (t == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(1)
                 : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar + 1)), "r"(1)
                 : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(slot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_proxy_async();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *slot;
  const uint32_t tlane = tmem + ((uint32_t)(warp * 32) << 16);
  const uint32_t sW2 = smem_u32(base + P.w2), sW3 = smem_u32(base + P.w3);
  const uint32_t sbar = smem_u32(bar);
  // Test hook: the first wait of a tile polls, 64 times, a second barrier
  // that nothing arrives at, so that it gives up while the layer-2 MMAs are
  // in flight and the timeout path below runs (the drain at the end then
  // waits, with the full limit, for the commit it skipped).
  const uint32_t sdead = smem_u32(bar + 1);
  const bool dead_wait = K.dead_wait != 0;
  const int Z = K.Z;
  const float log2dt = (float)a.pol.log2dt;

  uint32_t phase = 0;
  bool failed = false;
  const int64_t ntiles = (a.ncells + kM - 1) / kM;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t c = tile * kM + t;
    const bool on = c < a.ncells;
    if (failed) {  // after a timeout: no tensor-core work, mark the outputs
      if (!Step && on)
        for (int k = 0; k < Z; ++k) a.W_out[(int64_t)k * a.ldw + c] = __int_as_float(0x7fc00000);
      continue;
    }
    __syncthreads();  // every thread is done with the previous tile's Y
    const float Eabs = on ? fabsf(a.E[c]) : 1.0f;
    // the step's window populations, loaded now so that the loads are in
    // flight while the network is evaluated
    int clo = 0, chi = 0;
    bool valid = false;
    float v[ION_MAX_WINDOW];
#pragma unroll
    for (int r = 0; r < ION_MAX_WINDOW; ++r) v[r] = 0.0f;
    if constexpr (Step) {
      if (on) {
        clo = a.J.lo[c];
        chi = a.J.hi[c];
        valid = window_ok(clo, chi, a.J.Z);
        if (valid) {
          const float* p = static_cast<const float*>(a.J.N) + (int64_t)clo * a.J.ld + c;
#pragma unroll
          for (int r = 0; r < ION_MAX_WINDOW; ++r) {
            if (r < chi - clo + 1) v[r] = __ldcs(p);
            p += a.J.ld;
          }
        }
      }
    }
    const bool pos = Eabs > (float)kEmin && Eabs < INFINITY;
    const float l2 = log2f(pos ? Eabs : 1.0f);
    const float x = fminf(fmaxf(fmaf(K.xa, l2, K.xb), -1.0f), 1.0f);
    // the step skips the network for a tile none of whose cells could use
    // it (field outside the trained range, no rate in the window, or the
    // network never trusted); the decision is uniform over the CTA
    bool use_net = true;
    // the validation bounds of the window's states, loaded now (like the
    // populations) so that the loads are in flight during the network
    float beta[ION_MAX_WINDOW - 1];
#pragma unroll
    for (int r = 0; r < ION_MAX_WINDOW - 1; ++r) beta[r] = 0.0f;
    if constexpr (Step) {
      const bool mine = valid && chi > clo && pos && l2 >= K.l2lo && l2 <= K.l2hi &&
                        !a.pol.zero_dt && a.pop_tol > 0.0f;
      use_net = __syncthreads_or(mine) != 0;
      if (mine && a.bound) {
        int bin = (int)floorf(fmaf(K.bin_a, l2, K.bin_b));
        bin = min(max(bin, 0), K.nbins - 1);
        const float* bb = a.bound + bin * Z + clo;
#pragma unroll
        for (int r = 0; r < ION_MAX_WINDOW - 1; ++r)
          if (r < chi - clo) beta[r] = __ldg(bb + r);
      }
    }
    if (use_net) {
    // layer 1 -> this thread's row of the A operand in tensor memory, as
    // bf16 pairs (hi parts from column kColAhi, lo parts from kColAlo), 8
    // columns (16 activations) at a time
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      uint32_t hi[8], lo[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int u = 16 * q + 2 * j;
        split2(mlp::gelu_half(fmaf(K.W1h[u], x, K.b1h[u])),
               mlp::gelu_half(fmaf(K.W1h[u + 1], x, K.b1h[u + 1])), hi[j], lo[j]);
      }
      tmem_st8(tlane + kColAhi + 8 * q, hi);
      tmem_st8(tlane + kColAlo + 8 * q, lo);
    }
    if (!layer_products(tmem, sW2, sW2 + 8192, idesc_bf16(kM, H), t, sbar, phase, dead_wait,
                        sdead)) {
      failed = true;
      if (!Step && on)
        for (int k = 0; k < Z; ++k) a.W_out[(int64_t)k * a.ldw + c] = __int_as_float(0x7fc00000);
      continue;
    }
    // layer 2 epilogue: h2 = g(acc + b2) -> the A operand (layer 2 has read
    // it), 16 accumulator columns at a time
#pragma unroll
    for (int ch = 0; ch < 4; ++ch) {
      float v[16];
      tmem_ld16(tlane + ch * 16, v);
      uint32_t hi[8], lo[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int u = ch * 16 + 2 * j;
        split2(mlp::gelu_half(v[2 * j] + K.b2h[u]), mlp::gelu_half(v[2 * j + 1] + K.b2h[u + 1]),
               hi[j], lo[j]);
      }
      tmem_st8(tlane + kColAhi + 8 * ch, hi);
      tmem_st8(tlane + kColAlo + 8 * ch, lo);
    }
    if (!layer_products(tmem, sW3, sW3 + KP * 128, idesc_bf16(kM, KP), t, sbar, phase, false,
                        sdead)) {
      failed = true;
      if (!Step && on)
        for (int k = 0; k < Z; ++k) a.W_out[(int64_t)k * a.ldw + c] = __int_as_float(0x7fc00000);
      continue;
    }
    // layer 3 epilogue: log2 W_k = ymean + yscale (acc + b3) -> Y[k][t]
#pragma unroll
    for (int ch = 0; ch < KP / 16; ++ch) {
      float v[16];
      tmem_ld16(tlane + ch * 16, v);
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const int k = ch * 16 + j;
        if (k < Z) Y[k * kM + t] = fmaf(K.yscale[k], v[j], K.yoff[k]);
      }
    }
    tc_fence_before();
    }  // use_net
    if constexpr (!Step) {
      if (on)
        for (int k = 0; k < Z; ++k) {
          const float s = Y[k * kM + t];
          a.W_out[(int64_t)k * a.ldw + c] = s < K.yfloor ? 0.0f : exp2f(s);
        }
    } else {
      const int lo = clo, hi = chi;
      if (on && !valid) atomicAdd(&a.ws.hdr[kHdrInvalid], 1u);
      const int w = hi - lo + 1;
      float lam[ION_MAX_WINDOW];
#pragma unroll
      for (int r = 0; r < ION_MAX_WINDOW; ++r) lam[r] = 0.0f;
      bool net = false, plain = false;
      if (valid && w >= 2 && !a.pol.zero_dt) {
        const bool in_range = use_net && pos && l2 >= K.l2lo && l2 <= K.l2hi;
        const float wfloor = exp2f(K.yfloor + log2dt);
        float err = 0.0f;
#pragma unroll
        for (int r = 0; r < ION_MAX_WINDOW - 1; ++r) {
          if (in_range && r < w - 1) {
            const int k = lo + r;
            const float s = Y[k * kM + t];
            lam[r] = s < K.yfloor ? 0.0f : ex2_approx(s + log2dt);
            err += 2.0f * fmaf(fmaxf(lam[r], wfloor), beta[r], wfloor);
          }
        }
        net = in_range && err < a.pop_tol;  // pop_tol 0: never the network
        if (!net) {
          plain = true;
#pragma unroll
          for (int r = 0; r < ION_MAX_WINDOW; ++r) lam[r] = 0.0f;
          eq1_rates(tab, lo, w, a.E[c], lam);
        }
      }
      // cells with some W dt > 1 take the Bateman form in the record kernel,
      // with the rates of Eq. 1 (their error bound is far above any useful
      // tolerance, so the network could not serve them)
      float lmax = 0.0f;
#pragma unroll
      for (int r = 0; r < ION_MAX_WINDOW; ++r) lmax = fmaxf(lmax, lam[r]);
      const bool stiff = valid && lmax > DDParams<float>::prop_max;
      net = net && !stiff;
      plain = plain || stiff;
      warp_count(&a.ws.hdr[kHdrSurrogate], net);
      warp_count(&a.ws.hdr[kHdrPlain], plain);
      if (__ballot_sync(kFull, stiff))
        append_record(a.ws, stiff, 0, (int)c, on ? a.E[c] : 0.0f, lo, hi, v);
      // the warp's widest window bounds the series for all its lanes
      const int wt = (valid && !stiff) ? w : 0;
      const int Wm = __reduce_max_sync(kFull, wt);
      if (wt > 0) {
        if (Wm <= 2)
          taylor_cell<2>(a, (int)c, lo, hi, v, lam, lmax);
        else if (Wm <= 4)
          taylor_cell<4>(a, (int)c, lo, hi, v, lam, lmax);
        else
          taylor_cell<ION_MAX_WINDOW>(a, (int)c, lo, hi, v, lam, lmax);
      }
    }
  }
  // leave: tensor memory is freed by the warp that allocated it once every
  // read of it (and, after a timeout, the pending MMAs) are done
  tc_fence_before();
  __syncthreads();
  if (failed && t == 0) {
    if (a.ws.hdr) atomicAdd(&a.ws.hdr[kHdrTimeout], 1u);
    mbar_wait(sbar, phase ^ 1u);  // the commit still pending, if it ever lands
  }
  __syncthreads();
  tc_fence_after();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(kTmemCols)
                 : "memory");
}

// ---- validation error bound (ion_surrogate_validate) ----------------------
// Sample points: bin b, point i at log2|E| = l2lo + (l2hi - l2lo)
// (b + i/(per_bin - 1))/nbins, rounded to float.
__global__ void bound_points_kernel(int nbins, int per_bin, double l2lo, double l2hi, float* E) {
  const int64_t n = (int64_t)nbins * per_bin;
  const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= n) return;
  const int64_t b = j / per_bin;
  const int i = (int)(j - b * per_bin);
  const double l2 = l2lo + (l2hi - l2lo) * ((double)b + (double)i / (per_bin - 1)) / nbins;
  E[j] = (float)exp2(l2);
}

// One thread per (bin, state): margin * max over the bin's points of
// |max(log2 W_net, floor) - max(log2 W, floor)| + floor_add, W from Eq. 1 in
// FP64.  A NaN network rate (a tensor-core wait that gave up) sets *bad.
__global__ void bound_kernel(const SpeciesTable* t, const float* E, const float* Wn, int64_t ld,
                             int nbins, int per_bin, int Z, double floor, double margin,
                             double floor_add, float* bound, unsigned* bad) {
  __shared__ StagedF64 tab;
  stage_f64(t, 0.0, &tab);
  __syncthreads();
  const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (q >= (int64_t)nbins * Z) return;
  const int64_t b = q / Z;
  const int k = (int)(q - b * Z);
  double d = 0.0;
  bool nan = false;
  for (int i = 0; i < per_bin; ++i) {
    const int64_t j = b * per_bin + i;
    const double yt = log2_rate_f64(tab, k, field_f64((double)E[j]), floor);
    const float w = Wn[(int64_t)k * ld + j];
    nan = nan || isnan(w);
    const double yn = w > 0.0f ? fmax(log2((double)w), floor) : floor;
    d = fmax(d, fabs(yn - yt));
  }
  if (nan) atomicOr(bad, 1u);
  bound[q] = (float)(d * margin + floor_add);
}

}  // namespace sg
}  // namespace ion

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
struct ion_surrogate {
  int device, num_sms, Z, KP, nbins;
  int fit_rates, fit_step;  // resident CTAs per SM of the two kernels
  ion::sg::Dev* dev;
  float* bound;  // device [nbins][Z] of 2^bound - 1, or nullptr
  ion_surrogate_norm norm;
};

namespace {

using ion::sg::Dev;
using ion::sg::StepArgs;

// Round to nearest even, as __float2bfloat16_rn does.
uint16_t to_bf16(float f) {
  uint32_t u;
  std::memcpy(&u, &f, 4);
  if ((u & 0x7fffffffu) > 0x7f800000u) return 0x7fc0;
  u += 0x7fffu + ((u >> 16) & 1u);
  return (uint16_t)(u >> 16);
}

template <bool Step>
const void* kernel_of(int KP) {
  switch (KP) {
    case 16:
      return reinterpret_cast<const void*>(&ion::sg::surrogate_kernel<Step, 16>);
    case 32:
      return reinterpret_cast<const void*>(&ion::sg::surrogate_kernel<Step, 32>);
    case 48:
      return reinterpret_cast<const void*>(&ion::sg::surrogate_kernel<Step, 48>);
    default:
      return reinterpret_cast<const void*>(&ion::sg::surrogate_kernel<Step, 64>);
  }
}

// Sets the shared-memory limit and measures residency; refuses shapes whose
// resident CTAs could ask for more tensor memory than an SM has (512
// columns), so no allocation ever has to wait.
cudaError_t prepare(const void* fn, int KP, int* fit) {
  const size_t smem = ion::sg::plan_of(KP).total;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  // all of the unified L1/shared array as shared memory, so that the
  // occupancy below (and at launch) is limited by registers and smem alone
  e = cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout,
                           cudaSharedmemCarveoutMaxShared);
  if (e != cudaSuccess) return e;
  // residency from the kernel's registers and shared memory and the SM's
  // limits (the occupancy query reports one CTA per SM for these kernels,
  // below what the SM holds)
  cudaFuncAttributes fa;
  if ((e = cudaFuncGetAttributes(&fa, fn)) != cudaSuccess) return e;
  int dev = 0, regs_sm = 0, smem_sm = 0, smem_rsv = 0, thr_sm = 0, blk_sm = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev)) ||
      (e = cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev)) ||
      (e = cudaDeviceGetAttribute(&smem_rsv, cudaDevAttrReservedSharedMemoryPerBlock, dev)) ||
      (e = cudaDeviceGetAttribute(&thr_sm, cudaDevAttrMaxThreadsPerMultiProcessor, dev)) ||
      (e = cudaDeviceGetAttribute(&blk_sm, cudaDevAttrMaxBlocksPerMultiprocessor, dev)))
    return e;
  const int warps = ion::sg::kM / 32;
  const int regs_warp = ((fa.numRegs + 7) / 8 * 8 * 32 + 255) / 256 * 256;
  int f = regs_sm / (regs_warp * warps);
  const int per_block_smem = (int)smem + (int)fa.sharedSizeBytes + smem_rsv;
  f = std::min(f, smem_sm / per_block_smem);
  f = std::min(f, thr_sm / ion::sg::kM);
  f = std::min(f, blk_sm);
  // tensor memory: the resident CTAs' columns must fit the SM's 512, so that
  // no allocation ever waits
  f = std::min(f, 512 / (int)ion::sg::kTmemCols);
  *fit = f;
  if (*fit < 1) return cudaErrorInvalidConfiguration;
  return cudaSuccess;
}

cudaError_t launch(const ion_surrogate* s, bool step, const StepArgs& a, cudaStream_t st) {
  const int64_t ntiles = (a.ncells + ion::sg::kM - 1) / ion::sg::kM;
  if (ntiles == 0) return cudaSuccess;
  const int fit = step ? s->fit_step : s->fit_rates;
  const int64_t cap = (int64_t)fit * s->num_sms;
  const int blocks = (int)(ntiles < cap ? ntiles : cap);
  const void* fn = step ? kernel_of<true>(s->KP) : kernel_of<false>(s->KP);
  const Dev* dev = s->dev;
  void* args[] = {(void*)&dev, (void*)&a};
  return cudaLaunchKernel(fn, blocks, ion::sg::kM, args, ion::sg::plan_of(s->KP).total, st);
}

int check_surrogate(const ion_surrogate* s) {
  if (!s || !s->dev) return ion::set_error(ION_EINVAL, "surrogate is NULL or destroyed");
  int d = -1;
  if (cudaGetDevice(&d) != cudaSuccess || d != s->device)
    return ion::set_error(ION_EINVAL, "the surrogate lives on device %d; make it current",
                          s->device);
  return ION_OK;
}

bool al4(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 3u) == 0; }

// Replaces the surrogate's bound by the host array b [nbins*Z] (log2 units):
// the device copy holds 2^b - 1, and the bin mapping of the kernels' Consts
// follows nbins.  Synchronous.
int install_bound(ion_surrogate* s, const float* b, int nbins) {
  const size_t m = (size_t)nbins * s->Z;
  std::vector<float> beta(m);
  for (size_t i = 0; i < m; ++i) {
    if (!(b[i] >= 0.0f) || !std::isfinite(b[i]))
      return ion::set_error(ION_EINVAL, "bound[%zu] must be finite and >= 0", i);
    beta[i] = (float)(std::exp2((double)b[i]) - 1.0);
  }
  float* dst = nullptr;
  cudaError_t e = cudaMalloc(&dst, sizeof(float) * m);
  if (e == cudaSuccess) e = cudaMemcpy(dst, beta.data(), sizeof(float) * m, cudaMemcpyHostToDevice);
  const double span = s->norm.log2E_max - s->norm.log2E_min;
  const float bin_a = (float)(nbins / span);
  const float bin_b = (float)(-s->norm.log2E_min * nbins / span);
  char* k = reinterpret_cast<char*>(s->dev) + offsetof(Dev, k);
  if (e == cudaSuccess)
    e = cudaMemcpy(k + offsetof(ion::sg::Consts, bin_a), &bin_a, sizeof bin_a,
                   cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(k + offsetof(ion::sg::Consts, bin_b), &bin_b, sizeof bin_b,
                   cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(k + offsetof(ion::sg::Consts, nbins), &nbins, sizeof nbins,
                   cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    if (dst) cudaFree(dst);
    return ion::set_error(e == cudaErrorMemoryAllocation ? ION_ENOMEM : ION_ECUDA,
                          "installing the bound: %s", cudaGetErrorString(e));
  }
  if (s->bound) cudaFree(s->bound);
  s->bound = dst;
  s->nbins = nbins;
  return ION_OK;
}

}  // namespace

extern "C" {

int ion_surrogate_create(const ion_species* sp, const float* P, const ion_surrogate_norm* norm,
                         const float* bound, int nbins, ion_surrogate** out) {
  using namespace ion;
  if (!out) return set_error(ION_EINVAL, "out is NULL");
  *out = nullptr;
  SpeciesInfo si;
  int rc = species_info(sp, &si);
  if (rc) return rc;
  if (!P || !norm) return set_error(ION_EINVAL, "P and norm must be non-NULL");
  if (!(norm->log2E_min < norm->log2E_max) || !std::isfinite(norm->log2E_min) ||
      !std::isfinite(norm->log2E_max) || !std::isfinite(norm->y_floor))
    return set_error(ION_EINVAL, "norm: need finite log2E_min < log2E_max and y_floor");
  if (bound && (nbins < 1 || nbins > 65536))
    return set_error(ION_EINVAL, "nbins=%d outside [1, 65536]", nbins);
  if (!bound) nbins = 1;
  int cur = -1;
  if (cudaGetDevice(&cur) != cudaSuccess || cur != si.device)
    return set_error(ION_EINVAL, "the species lives on device %d; make it current", si.device);
  const int Z = si.Z, KP = mlp::padded_out(Z), np = mlp::nparams(Z);
  for (int k = 0; k < Z; ++k)
    if (!std::isfinite(norm->y_mean[k]) || !(norm->y_scale[k] > 0.0) ||
        !std::isfinite(norm->y_scale[k]))
      return set_error(ION_EINVAL, "norm: y_mean[%d] must be finite, y_scale[%d] > 0", k, k);
  std::vector<float> h((size_t)np);
  cudaError_t e = cudaMemcpy(h.data(), P, sizeof(float) * np, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess)
    return set_error(ION_ECUDA, "reading the parameters: %s", cudaGetErrorString(e));
  for (int i = 0; i < np; ++i)
    if (!std::isfinite(h[i])) return set_error(ION_EINVAL, "parameter %d is not finite", i);
  std::vector<float> beta((size_t)nbins * Z, 0.0f);
  if (bound)
    for (size_t i = 0; i < beta.size(); ++i) {
      if (!(bound[i] >= 0.0f) || !std::isfinite(bound[i]))
        return set_error(ION_EINVAL, "bound[%zu] must be finite and >= 0", i);
      beta[i] = (float)(std::exp2((double)bound[i]) - 1.0);
    }
  Dev* img = new (std::nothrow) Dev();
  if (!img) return set_error(ION_ENOMEM, "host allocation failed");
  std::memset(img, 0, sizeof(Dev));
  // each weight as the pair bf16(w), bf16(w - bf16(w))
  auto put = [](uint8_t (&dst)[2][64 * 128], int r, int k, float v) {
    const uint16_t hi = to_bf16(v);
    const uint32_t hb = (uint32_t)hi << 16;
    float hf;
    std::memcpy(&hf, &hb, 4);
    const uint16_t lo = to_bf16(v - hf);
    std::memcpy(dst[0] + sg::sw128_offset(r, k), &hi, 2);
    std::memcpy(dst[1] + sg::sw128_offset(r, k), &lo, 2);
  };
  // W2 halved (exactly), so that layer 2's accumulators arrive halved
  for (int o = 0; o < mlp::H; ++o)
    for (int k = 0; k < mlp::H; ++k)
      put(img->W2img, o, k, 0.5f * h[mlp::off_W2() + o * mlp::H + k]);
  for (int r = 0; r < KP; ++r)
    for (int k = 0; k < mlp::H; ++k)
      put(img->W3img, r, k, r < Z ? h[mlp::off_W3() + r * mlp::H + k] : 0.0f);
  sg::Consts& c = img->k;
  for (int i = 0; i < mlp::H; ++i) {
    c.W1h[i] = 0.5f * h[mlp::off_W1() + i];
    c.b1h[i] = 0.5f * h[mlp::off_b1() + i];
    c.b2h[i] = 0.5f * h[mlp::off_b2() + i];
  }
  for (int k = 0; k < Z; ++k) {
    c.yscale[k] = (float)norm->y_scale[k];
    c.yoff[k] = (float)(norm->y_scale[k] * (double)h[mlp::off_b3(Z) + k] + norm->y_mean[k]);
  }
  const double span = norm->log2E_max - norm->log2E_min;
  c.xa = (float)(2.0 / span);
  c.xb = (float)(-1.0 - norm->log2E_min * 2.0 / span);
  c.l2lo = (float)norm->log2E_min;
  c.l2hi = (float)norm->log2E_max;
  c.yfloor = (float)norm->y_floor;
  c.bin_a = (float)(nbins / span);
  c.bin_b = (float)(-norm->log2E_min * nbins / span);
  c.nbins = nbins;
  c.Z = Z;
  c.KP = KP;
  img->tab = *si.host;
  ion_surrogate* s = new (std::nothrow) ion_surrogate();
  if (!s) {
    delete img;
    return set_error(ION_ENOMEM, "host allocation failed");
  }
  s->device = si.device;
  s->num_sms = si.num_sms;
  s->Z = Z;
  s->KP = KP;
  s->nbins = nbins;
  s->dev = nullptr;
  s->bound = nullptr;
  s->norm = *norm;
  e = cudaMalloc(&s->dev, sizeof(Dev));
  if (e == cudaSuccess) e = cudaMemcpy(s->dev, img, sizeof(Dev), cudaMemcpyHostToDevice);
  delete img;
  if (e == cudaSuccess && bound) {
    e = cudaMalloc(&s->bound, sizeof(float) * beta.size());
    if (e == cudaSuccess)
      e = cudaMemcpy(s->bound, beta.data(), sizeof(float) * beta.size(), cudaMemcpyHostToDevice);
  }
  if (e == cudaSuccess) e = prepare(kernel_of<false>(KP), KP, &s->fit_rates);
  if (e == cudaSuccess) e = prepare(kernel_of<true>(KP), KP, &s->fit_step);
  if (e != cudaSuccess) {
    if (s->dev) cudaFree(s->dev);
    if (s->bound) cudaFree(s->bound);
    delete s;
    return set_error(e == cudaErrorMemoryAllocation ? ION_ENOMEM : ION_ECUDA,
                     "ion_surrogate_create: %s", cudaGetErrorString(e));
  }
  *out = s;
  return set_error(ION_OK, "%s", "");
}

int ion_surrogate_test_timeout(ion_surrogate* s, int on) {
  const int rc = check_surrogate(s);
  if (rc) return rc;
  const int v = on ? 1 : 0;
  const cudaError_t e = cudaMemcpy(reinterpret_cast<char*>(s->dev) + offsetof(Dev, k) +
                                       offsetof(ion::sg::Consts, dead_wait),
                                   &v, sizeof v, cudaMemcpyHostToDevice);
  if (e != cudaSuccess)
    return ion::set_error(ION_ECUDA, "ion_surrogate_test_timeout: %s", cudaGetErrorString(e));
  return ion::set_error(ION_OK, "%s", "");
}

int ion_surrogate_validate(ion_surrogate* s, int nbins, int per_bin, double margin,
                           double floor_add, float* bound_out, void* stream) {
  using namespace ion;
  int rc = check_surrogate(s);
  if (rc) return rc;
  if (nbins < 1 || nbins > 65536 || per_bin < 2 || per_bin > 4096 ||
      (int64_t)nbins * per_bin > (int64_t(1) << 24))
    return set_error(ION_EINVAL,
                     "need 1 <= nbins <= 65536, 2 <= per_bin <= 4096, nbins*per_bin <= 2^24");
  if (!(margin >= 1.0) || !std::isfinite(margin) || !(floor_add >= 0.0) ||
      !std::isfinite(floor_add))
    return set_error(ION_EINVAL, "need finite margin >= 1 and floor_add >= 0");
  const int Z = s->Z;
  const int64_t n = (int64_t)nbins * per_bin;
  auto up = [](size_t x) { return (x + 255) / 256 * 256; };
  const size_t oE = 0, oW = up(4 * (size_t)n), oB = oW + up(4 * (size_t)n * Z),
               oF = oB + up(4 * (size_t)nbins * Z), total = oF + 256;
  char* buf = nullptr;
  cudaError_t e = cudaMalloc(&buf, total);
  if (e != cudaSuccess)
    return set_error(e == cudaErrorMemoryAllocation ? ION_ENOMEM : ION_ECUDA,
                     "ion_surrogate_validate scratch: %s", cudaGetErrorString(e));
  float* Eg = reinterpret_cast<float*>(buf + oE);
  float* Wn = reinterpret_cast<float*>(buf + oW);
  float* bd = reinterpret_cast<float*>(buf + oB);
  unsigned* bad = reinterpret_cast<unsigned*>(buf + oF);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  std::vector<float> hb((size_t)nbins * Z);
  unsigned hbad = 0;
  e = cudaMemsetAsync(bad, 0, sizeof(unsigned), st);
  if (e == cudaSuccess) {
    sg::bound_points_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(
        nbins, per_bin, s->norm.log2E_min, s->norm.log2E_max, Eg);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    StepArgs a;
    std::memset(&a, 0, sizeof a);
    a.W_out = Wn;
    a.ldw = n;
    a.ncells = n;
    a.E = Eg;
    e = launch(s, false, a, st);
  }
  if (e == cudaSuccess) {
    const int64_t q = (int64_t)nbins * Z;
    sg::bound_kernel<<<(unsigned)((q + 127) / 128), 128, 0, st>>>(
        &s->dev->tab, Eg, Wn, n, nbins, per_bin, Z, s->norm.y_floor, margin, floor_add, bd, bad);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(hb.data(), bd, sizeof(float) * hb.size(), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&hbad, bad, sizeof hbad, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(buf);
  if (e != cudaSuccess)
    return set_error(ION_ECUDA, "ion_surrogate_validate: %s", cudaGetErrorString(e));
  if (hbad)
    return set_error(ION_ETIMEOUT, "ion_surrogate_validate: a tensor-core wait gave up");
  if ((rc = install_bound(s, hb.data(), nbins))) return rc;
  if (bound_out) std::memcpy(bound_out, hb.data(), sizeof(float) * hb.size());
  return set_error(ION_OK, "%s", "");
}

int ion_surrogate_destroy(ion_surrogate* s) {
  if (!s) return ion::set_error(ION_OK, "%s", "");
  if (s->dev) cudaFree(s->dev);
  if (s->bound) cudaFree(s->bound);
  s->dev = nullptr;
  delete s;
  return ion::set_error(ION_OK, "%s", "");
}

int ion_surrogate_rates(const ion_surrogate* s, const float* E, int64_t ncells, float* W_out,
                        int64_t ldw, void* stream) {
  int rc = check_surrogate(s);
  if (rc) return rc;
  if (ncells < 0 || ncells >= (int64_t(1) << 31))
    return ion::set_error(ION_EINVAL, "ncells=%lld outside [0, 2^31)", (long long)ncells);
  if (ncells == 0) return ion::set_error(ION_OK, "%s", "");
  if (!E || !W_out || !al4(E) || !al4(W_out))
    return ion::set_error(ION_EINVAL, "E and W_out must be non-NULL and 4-byte aligned");
  if (ldw < ncells) return ion::set_error(ION_EINVAL, "ldw < ncells");
  StepArgs a;
  std::memset(&a, 0, sizeof a);
  a.W_out = W_out;
  a.ldw = ldw;
  a.ncells = ncells;
  a.E = E;
  const cudaError_t e = launch(s, false, a, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess)
    return ion::set_error(ION_ECUDA, "ion_surrogate_rates launch: %s", cudaGetErrorString(e));
  return ion::set_error(ION_OK, "%s", "");
}

int ion_step_surrogate(const ion_surrogate* s, const float* E, float* N, int64_t ld,
                       int64_t ncells, double dt_fs, uint8_t* k_lo, uint8_t* k_hi, float* dne,
                       const float* n_gas, const ion_step_opts* opts, double pop_tol,
                       void* workspace, size_t workspace_bytes, void* stream) {
  using namespace ion;
  int rc = check_surrogate(s);
  if (rc) return rc;
  if (ncells < 0 || ncells >= (int64_t(1) << 31))
    return set_error(ION_EINVAL, "ncells=%lld outside [0, 2^31)", (long long)ncells);
  if (ncells > 0) {
    if (!E || !N || !k_lo || !k_hi || !dne)
      return set_error(ION_EINVAL, "E, N, k_lo, k_hi and dne must be non-NULL");
    if (ld < ncells || ld > (int64_t(1) << 40))
      return set_error(ION_EINVAL, "ld=%lld must lie in [ncells, 2^40]", (long long)ld);
    if (!al4(E) || !al4(N) || !al4(dne) || (n_gas && !al4(n_gas)))
      return set_error(ION_EINVAL, "E, N, dne and n_gas must be 4-byte aligned");
  }
  if (!(pop_tol >= 0.0) || !std::isfinite(pop_tol))
    return set_error(ION_EINVAL, "pop_tol must be finite and >= 0");
  StepArgs a;
  std::memset(&a, 0, sizeof a);
  if ((rc = policy_from_args(dt_fs, opts, ION_F32, &a.pol))) return rc;
  if ((rc = workspace_ok(workspace, workspace_bytes, step_workspace_bytes(ncells, false))))
    return rc;
  bind_workspace(a.ws, workspace, ncells);
  JobIO& J = a.J;
  J.tab = &s->dev->tab;
  J.Z = s->Z;
  J.E = E;
  J.N = N;
  J.ld = ld;
  J.ncells = (int)ncells;
  J.lo = k_lo;
  J.hi = k_hi;
  J.dne = dne;
  J.n_gas = n_gas;
  a.pop_tol = (float)pop_tol;
  a.bound = s->bound;
  a.ncells = ncells;
  a.E = E;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemsetAsync(a.ws.hdr, 0, kHdrWords * sizeof(uint32_t), st);
  if (e == cudaSuccess) e = launch(s, true, a, st);
  if (e == cudaSuccess && ncells > 0) {
    BatchArgs b;
    std::memset(&b, 0, sizeof b);
    b.njobs = 1;
    b.job[0] = J;
    b.pol = a.pol;
    b.ws = a.ws;
    e = launch_stiff_f32(b, s->num_sms, st);
    if (e == cudaSuccess) e = launch_fb_f32(b, s->num_sms, st);
  }
  if (e != cudaSuccess)
    return set_error(ION_ECUDA, "ion_step_surrogate launch: %s", cudaGetErrorString(e));
  return set_error(ION_OK, "%s", "");
}

}  // extern "C"
