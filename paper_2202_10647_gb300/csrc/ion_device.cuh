// ion_device.cuh -- device-side building blocks of the ionization step:
// the species table, the ADK rate in log2 form (Eq. 1), exponential divided
// differences, and the windowed Bateman update (Eqs. 3-9).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "ionize.h"

namespace ion {

// ---------------------------------------------------------------------------
// Species table.  Eq. 1 with x = E_a/|E| is W = A x^b exp(-c x), so
//   log2 W[1/fs] = a2 - b log2|E| - C/|E|
// with b = 2n* - |m| - 3/2, C = (2/3)(Q/n*)^3 E_a / ln 2 and
//   a2 = log2(A) + b log2(E_a),
//   A  = w_a sqrt(3 n*^3/(pi Q^3)) Q^2/(2 n*^2) (2e/n*)^(2n*) f(l,m)/(2 pi n*)
//        (2 Q^3/n*^3)^(2n* - |m| - 1).
// Built once per species on the host in double (api.cu, build_table).
// ---------------------------------------------------------------------------
struct SpeciesTable {
  int Z;
  double a2[ION_MAX_Z];
  double b[ION_MAX_Z];
  double C[ION_MAX_Z];
};

// Exponent (2/3)(Q/n*)^3 E_a/|E| above which W is set to 0; in the log2 units
// of C/|E| that is 700/ln 2.
constexpr double kCutoffLog2 = 1009.8865286222745;
// |E| at or below which W is set to 0 (GV/m).
constexpr double kEmin = 1e-6;

// FP32 copy of the table staged in shared memory, each double held as an
// unevaluated sum hi + lo of two floats, with log2(dt) folded into a.
// Entries Z.. are padding (never staged): a window's slots past its top
// may index them, and their rates are masked.  ecold[k] (staged by the
// streaming kernel only): a field strength below which W_j dt < 2^kColdLog2
// for every j >= k, 0 where none was found safely.
struct StagedF32 {
  float4 hi[ION_MAX_Z + ION_MAX_WINDOW];  // {a_hi, b_hi, C_hi, a_lo}: one 16-byte load
  float2 lo[ION_MAX_Z + ION_MAX_WINDOW];  // {b_lo, C_lo}
  float ecold[ION_MAX_Z + ION_MAX_WINDOW];
};

struct StagedF64 {
  double a[ION_MAX_Z + 1];  // a2 + log2(dt)
  double b[ION_MAX_Z + 1];
  double C[ION_MAX_Z + 1];
};

__device__ __forceinline__ void split_f64(double x, float& hi, float& lo) {
  hi = __double2float_rn(x);
  lo = isfinite(x) ? __double2float_rn(x - (double)hi) : 0.0f;
}

// Threads [0, Z) of the block stage the table; the caller syncs.
__device__ __forceinline__ void stage_f32(const SpeciesTable* t, double log2dt,
                                          StagedF32* s) {
  const int Z = t->Z;
  for (int k = threadIdx.x; k < Z; k += blockDim.x) {
    float ah, al, bh, bl, ch, cl;
    split_f64(t->a2[k] + log2dt, ah, al);
    split_f64(t->b[k], bh, bl);
    split_f64(t->C[k], ch, cl);
    s->hi[k] = make_float4(ah, bh, ch, al);
    s->lo[k] = make_float2(bl, cl);
  }
}

__device__ __forceinline__ void stage_f64(const SpeciesTable* t, double log2dt,
                                          StagedF64* s) {
  const int Z = t->Z;
  for (int k = threadIdx.x; k < Z; k += blockDim.x) {
    s->a[k] = t->a2[k] + log2dt;
    s->b[k] = t->b[k];
    s->C[k] = t->C[k];
  }
}

// ---------------------------------------------------------------------------
// Rate times dt in FP32 with float-float exponent arithmetic.  The exponent
// y = a - b log2|E| - C/|E| is a sum of terms of size up to ~10^3 whose
// result matters to ~1e-7 absolute (relative error of W*dt), so the large
// terms are carried as hi+lo pairs (Dekker/Knuth two-sum and fma two-product).
// ---------------------------------------------------------------------------
struct FieldF32 {
  float E, rE;   // |E| and an approximation of 1/|E| (its error is corrected)
  float ex, lm;  // log2|E| = ex + lm, ex integer, lm in [0,1)
  float lg;      // ex + lm rounded to float
  bool zero;     // W = 0 for every state
};

template <bool Precise = false>
__device__ __forceinline__ FieldF32 field_f32(float E_in) {
  FieldF32 f;
  float E = fabsf(E_in);
  f.zero = !(E > (float)kEmin) || isinf(E);
  E = f.zero ? 1.0f : E;
  // E is normal here: split the exponent and the mantissa in [1, 2)
  const int bits = __float_as_int(E);
  const float mant = __int_as_float((bits & 0x007fffff) | 0x3f800000);
  f.ex = (float)((bits >> 23) - 127);
  f.lm = Precise ? log2f(mant) : __log2f(mant);
  f.lg = f.ex + f.lm;
  f.E = E;
  f.rE = Precise ? __frcp_rn(E) : __fdividef(1.0f, E);
  return f;
}

// 2^x by the SFU (ex2.approx.ftz.f32: about 2 ulp; results below 2^-126
// flush to 0, which no population can see).
__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// W dt below 2^kColdLog2 (9.3e-10) is far under the 1.5e-9 at which the FP32
// Taylor series takes its first term (2 W dt > kThrF32[0]); below
// 2^kColdLog2F64 (3.5e-18) likewise for the FP64 series (kThrF64[0] = 2e-17).
constexpr float kColdLog2 = -30.0f;
constexpr float kColdLog2F64 = -58.0f;

// Field strength E_c below which y(E) = a - b log2 E - C/E, the log2 of W dt
// (Eq. 1), lies under tlog2; 0 when no such bound is found safely.  With
// u = log2 E, g(u) = y - tlog2 is concave in u (g'' = -C ln^2 2 2^-u), so
// Newton's iterates that start where g' > 0 approach the root from below
// after their first step.  E_c is the last iterate less 2^-8 relative:
// g(log2 E_c) <= about -0.25, margin for the FP32 arithmetic here and for
// the rate evaluation that E_c stands in for.  Below the root g increases
// with u, so every E < E_c has y < tlog2 as well.
__device__ __forceinline__ float cold_field(double a_d, double b_d, double C_d, float tlog2) {
  const float am = (float)a_d - tlog2, b = (float)b_d, C = (float)C_d;
  constexpr float kLn2 = 0.693147181f;
  // the start u0 = log2(C / am) has g'(u0) = am ln 2 - b; demand a margin
  if (!(C > 0.0f) || !(am * kLn2 > b + 1.0f) || !(am < 1e30f)) return 0.0f;
  float u = __log2f(__fdividef(C, am));
  for (int i = 0; i < 12; ++i) {
    const float e = C * ex2_approx(-u);
    const float gp = fmaf(e, kLn2, -b);
    if (!(gp > 0.0f)) return 0.0f;
    u -= __fdividef(am - b * u - e, gp);
  }
  const float g = am - b * u - C * ex2_approx(-u);
  if (!(g <= 0.01f) || !(u < 126.0f)) return 0.0f;
  return ex2_approx(u) * (1.0f - 1.0f / 256.0f);
}

// One warp: ecold[0 .. ION_MAX_Z + ION_MAX_WINDOW) of one species for the
// target 2^tlog2 (threads k < Z of the table in two rounds of 32), each
// state's own cold field turned into the minimum over the states at or
// above it by a suffix scan; the padding past Z holds 0 (never cold).
__device__ __forceinline__ void stage_cold(const SpeciesTable* t, double log2dt, float tlog2,
                                           float* ecold, int lane) {
  const int Z = t->Z;
  const float kInf = __int_as_float(0x7f800000);
  float m[2];
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int k = lane + 32 * h;
    m[h] = k < Z ? cold_field(t->a2[k] + log2dt, t->b[k], t->C[k], tlog2) : kInf;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const float x = __shfl_down_sync(0xffffffffu, m[h], o);
      if (lane + o < 32) m[h] = fminf(m[h], x);
    }
  }
  m[0] = fminf(m[0], __shfl_sync(0xffffffffu, m[1], 0));
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int k = lane + 32 * h;
    ecold[k] = k < Z ? m[h] : 0.0f;
  }
  if (lane + 64 < ION_MAX_Z + ION_MAX_WINDOW) ecold[lane + 64] = 0.0f;
}



__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// y = a - b log2|E| - C/|E| (log2 of W dt).  A plain FP32 evaluation first;
// where it says W dt < 2^-12 its error (below 2^-10 relative for terms up
// to 10^3) moves W dt by less than 3e-7 and no population can see it, so
// only larger rates take the float-float evaluation.
template <bool Precise = false>
__device__ __forceinline__ float rate_dt_f32(const StagedF32& t, int k,
                                             const FieldF32& f) {
  if (f.zero) return 0.0f;
  const float4 h = t.hi[k];  // a_hi, b_hi, C_hi, a_lo
  const float q = h.z * f.rE;
  if (q > (float)kCutoffLog2) return 0.0f;
  if (!Precise) {
    const float y0 = fmaf(-h.y, f.lg, h.x) - q;
    if (y0 < -12.0f) return ex2_approx(y0);
  }
  const float2 l = t.lo[k];  // b_lo, C_lo
  const float ql = (fmaf(-q, f.E, h.z) + l.y) * f.rE;  // C/E = q + ql
  const float p = h.y * f.ex;
  const float pe = fmaf(h.y, f.ex, -p);  // b_hi*ex = p + pe exactly
  float s1, e1, s2, e2;
  two_sum(h.x, -p, s1, e1);
  two_sum(s1, -q, s2, e2);
  const float small = ((h.w - pe) - ql) - fmaf(h.y, f.lm, l.x * f.lg);
  const float tail = (e1 + e2) + small;
  if (Precise) {
    // 2^(s2 + tail) as 2^s2 2^tail keeps the relative error at a few ulp for
    // any size of the exponent (rounding s2 + tail to one float would cost
    // up to |y| 2^-24 relative).
    return s2 > 99.0f ? exp2f(99.0f) : exp2f(s2) * exp2f(tail);
  }
  float y = s2 + tail;
  y = fminf(y, 99.0f);  // W dt <= 2^99: keeps every later product finite
  return ex2_approx(y);
}

// The float-float branch of rate_dt_f32 alone, for a rate its plain FP32
// evaluation already found live and above 2^-12 (non-zero field, C/|E|
// under the cutoff): the same value, without re-testing those.
__device__ __forceinline__ float rate_ff_f32(const StagedF32& t, int k, const FieldF32& f) {
  const float4 h = t.hi[k];  // a_hi, b_hi, C_hi, a_lo
  const float2 l = t.lo[k];  // b_lo, C_lo
  const float q = h.z * f.rE;
  const float ql = (fmaf(-q, f.E, h.z) + l.y) * f.rE;  // C/E = q + ql
  const float p = h.y * f.ex;
  const float pe = fmaf(h.y, f.ex, -p);  // b_hi*ex = p + pe exactly
  float s1, e1, s2, e2;
  two_sum(h.x, -p, s1, e1);
  two_sum(s1, -q, s2, e2);
  const float small = ((h.w - pe) - ql) - fmaf(h.y, f.lm, l.x * f.lg);
  const float tail = (e1 + e2) + small;
  return ex2_approx(fminf(s2 + tail, 99.0f));
}

// The field's part of the FP64 exponent, once per cell: log2|E| and 1/|E|.
struct FieldF64 {
  double lg, rE;
  bool zero;
};

__device__ __forceinline__ FieldF64 field_f64(double E_in) {
  FieldF64 f;
  const double E = fabs(E_in);
  f.zero = !(E > kEmin) || isinf(E);
  f.lg = f.zero ? 0.0 : log2(E);
  f.rE = f.zero ? 0.0 : 1.0 / E;
  return f;
}

// W_k dt in FP64.  C/|E| is taken as C (1/|E|), one rounding more than a
// division: a relative error of 2^-52 in a term below 1010, far under the
// 1e-12 the FP64 form is held to.
__device__ __forceinline__ double rate_dt_f64(const StagedF64& t, int k, const FieldF64& f) {
  if (f.zero) return 0.0;
  const double q = t.C[k] * f.rE;
  if (q > kCutoffLog2) return 0.0;
  double y = t.a[k] - t.b[k] * f.lg - q;
  y = fmin(y, 1000.0);
  return exp2(y);
}

__device__ __forceinline__ double rate_dt_f64(const StagedF64& t, int k, double E_in) {
  return rate_dt_f64(t, k, field_f64(E_in));
}

// log2(W_k dt) in FP64 straight from the exponent of rate_dt_f64 (no exp2 /
// log2 round trip), clamped below at `floor`, which also stands for W = 0.
__device__ __forceinline__ double log2_rate_f64(const StagedF64& t, int k, const FieldF64& f,
                                                double floor) {
  if (f.zero) return floor;
  const double q = t.C[k] * f.rE;
  if (q > kCutoffLog2) return floor;
  return fmax(fmin(t.a[k] - t.b[k] * f.lg - q, 1000.0), floor);
}

// ---------------------------------------------------------------------------
// Divided differences of exp.
//
// For nodes z_0..z_{NR-1} (z = -W dt) the Bateman coefficient of Eqs. 4-5
// that carries population from state j to state i > j is
//   P_ij = (prod_{q=j}^{i-1} W_q dt) * exp[z_j, ..., z_i],
// exp[...] the divided difference of exp on those nodes; P_ii = e^{z_i}.
// For distinct rates this is the sum of exponentials of Eq. 4 (Eqs. 6-8 for
// four levels); written as a divided difference it stays defined and
// accurate for equal and nearly equal rates.
//
// dd_exp_ranges fills D[j..i] = exp[z_j, ..., z_i] for every contiguous
// range of nodes, shortest ranges first:
//   * spread s = max z - min z of the range >= TAU: the two-term recurrence
//     that removes one end of the range,
//       D[j..i] = (D[j+1..i] - D[j..i-1]) / (z_i - z_j).
//     When the ends are the range's smallest and largest nodes the divisor
//     is its spread, which bounds the cancellation (both terms are positive);
//     a range whose ends are close while an inner node lies far off is
//     instead evaluated on its nodes in increasing order (dd_set).
//   * s < TAU: the Taylor series of the divided difference about a node c
//     of the range,
//       exp[S] = e^{c} sum_{r>=0} h_r(z - c) / (|S|-1+r)!,
//     h_r the complete homogeneous symmetric polynomial of degree r,
//     truncated at the first R with s^(R+1)/(R+1)! below the target (FP64)
//     or at the R that TAU itself needs (FP32).
// ---------------------------------------------------------------------------
// Number of Taylor terms: the smallest R with x^(R+1)/(R+1)! below the
// target, i.e. the number of thresholds kThr[i] = (target (i+1)!)^(1/(i+1))
// that lie below x.  FP64: target 2e-17.  FP32: target 3e-8 (half an ulp of
// 1, and 1.5 % of the 2e-6 the FP32 form is held to) for the second and
// later terms; the first term is taken from x > 3e-9 on, so that no rate
// whose first-order effect exceeds that is dropped, step after step.
__device__ constexpr float kThrF32[19] = {
    3e-09f,    0.000244949f, 0.00564622f, 0.0291295f, 0.0815193f, 0.166882f,
    0.284591f, 0.431847f,    0.605168f,   0.801103f,  1.01652f,   1.24869f,
    1.49528f,  1.75432f,     2.02414f,    2.30334f,   2.59073f,   2.88531f,
    3.18621f};
__device__ constexpr double kThrF64[20] = {
    2e-17,     6.32456e-09, 4.93242e-06, 0.000148017, 0.00119136, 0.00493242,
    0.0139108, 0.0307836,   0.0578509,   0.0968455,   0.148911,   0.214675,
    0.294354,  0.387859,    0.494882,    0.614969,    0.747572,   0.892092,
    1.04791,   1.21439};

// 1/n! for n = 0..17 (the Taylor branch needs n <= 4 + 12), in each
// precision (the FP32 path reads no double: conversions run on the FP64 pipe).
__device__ constexpr double kInvFact[18] = {
    1.0, 1.0, 1.0 / 2, 1.0 / 6, 1.0 / 24, 1.0 / 120, 1.0 / 720, 1.0 / 5040,
    1.0 / 40320, 1.0 / 362880, 1.0 / 3628800, 1.0 / 39916800, 1.0 / 479001600,
    1.0 / 6227020800.0, 1.0 / 87178291200.0, 1.0 / 1307674368000.0,
    1.0 / 20922789888000.0, 1.0 / 355687428096000.0};
__device__ constexpr float kInvFactF[18] = {
    1.0f, 1.0f, 1.0f / 2, 1.0f / 6, 1.0f / 24, 1.0f / 120, 1.0f / 720, 1.0f / 5040,
    1.0f / 40320, 1.0f / 362880, 1.0f / 3628800, 1.0f / 39916800, 1.0f / 479001600,
    1.0f / 6227020800.0f, 1.0f / 87178291200.0f, 1.0f / 1307674368000.0f,
    1.0f / 20922789888000.0f, 1.0f / 355687428096000.0f};

template <typename T>
struct DDParams;

template <>
struct DDParams<float> {
  static constexpr float tau = 1.0f;   // Taylor below this subset spread
  static constexpr int RMAX = 10;      // terms needed at spread tau
  static constexpr float prop_max = 1.0f;  // Taylor propagation up to max W dt
  static constexpr int PMAX = 16;      // bound on the terms (14 needed at 2 * prop_max)
  static constexpr bool kUniform = true;  // every Taylor term up to RMAX
  static constexpr float end_ratio = 4.0f;  // dd_exp_ranges' recurrence bound
  __device__ static __forceinline__ int terms(float x, int rmax) {
    int R = 0;
#pragma unroll
    for (int i = 0; i < 17; ++i)
      if (i < rmax) R += x > kThrF32[i] ? 1 : 0;
    return R;
  }
  __device__ static __forceinline__ float div(float a, float b) { return __fdividef(a, b); }
  __device__ static __forceinline__ float inv_fact(int n) { return kInvFactF[n]; }
};

template <>
struct DDParams<double> {
  static constexpr double tau = 0.25;
  static constexpr int RMAX = 12;
  static constexpr double prop_max = 0.5;
  static constexpr int PMAX = 18;
  static constexpr bool kUniform = false;  // terms(s) of them
  static constexpr double end_ratio = 4.0;
  __device__ static __forceinline__ int terms(double x, int rmax) {
    int R = 0;
#pragma unroll
    for (int i = 0; i < 20; ++i)
      if (i < rmax) R += x > kThrF64[i] ? 1 : 0;
    return R;
  }
  __device__ static __forceinline__ double div(double a, double b) { return a / b; }
  __device__ static __forceinline__ double inv_fact(int n) { return kInvFact[n]; }
};

// mask of the contiguous node range [j, i]
__host__ __device__ constexpr int range_mask(int j, int i) {
  return ((1 << (i + 1)) - 1) & ~((1 << j) - 1);
}



// Taylor values of every contiguous range of nodes:
// C[a][b] = sum_r h_r(z[a..b] - z[a]) / (b-a+r)!, the divided difference of
// exp over z[a..b] without the factor e^{z[a]}.  The complete homogeneous
// polynomials obey h_r(x_1..x_k) = h_r(x_1..x_{k-1}) + x_k h_{r-1}(x_1..x_k),
// so one chain per left end a adds the nodes a+1, a+2, ... in turn and reads
// off every range [a, b] on the way: NR(NR-1)/2 node additions for all the
// ranges, instead of one series per range over its whole subset.  The series
// is the same about any centre inside the range; about its first node the
// offsets are at most the range's spread in size (either sign), which bounds
// the terms as about the largest node.
template <typename T, int NR>
__device__ __forceinline__ void taylor_chains(const T (&z)[NR], int R, T (&C)[NR][NR]) {
  using P = DDParams<T>;
#pragma unroll
  for (int a = 0; a + 1 < NR; ++a) {
    T H[P::RMAX + 1];
    H[0] = T(1);
#pragma unroll
    for (int r = 1; r <= P::RMAX; ++r) H[r] = T(0);
#pragma unroll
    for (int b = a + 1; b < NR; ++b) {
      const T x = z[b] - z[a];
#pragma unroll
      for (int r = 1; r <= P::RMAX; ++r)
        if (r <= R) H[r] = fma(x, H[r - 1], H[r]);
      T acc = T(0);
#pragma unroll
      for (int r = P::RMAX; r >= 0; --r)  // smallest terms first
        if (r <= R) acc = fma(H[r], P::inv_fact(b - a + r), acc);
      C[a][b] = acc;
    }
  }
}

template <typename T>
__device__ __noinline__ T dd_set(T z0, T z1, T z2, T z3, T z4, T e0, T e1, T e2, T e3, T e4,
                                 int m);

// The divided differences of exp over the contiguous ranges [j, i] that
// dd_update reads, in any node order.  A range of spread below TAU takes its
// Taylor value (taylor_chains); a wider one the recurrence that removes its
// first or its last node, which stays on contiguous ranges (NR(NR-1)/2 of
// them instead of the 2^NR - NR - 1 subsets of a recurrence that removes the
// smallest and the largest node).  When the range's ends are its extremes
// (rates falling or rising along the window) that is the same recurrence.
// Otherwise the two terms can cancel.  Each term is about (len-1) D[j..i]
// when the nodes lie within a few units and about (2 max z - z_i - z_j)
// D[j..i] for a wide range, and their difference is |z_i - z_j| D[j..i]; the
// ratio, the factor by which the subtraction magnifies the terms' rounding,
// stays below 2 END_RATIO (as with sorted nodes, whose end gap is the
// spread) while |z_i - z_j| >= TAU and the spread is at most
// END_RATIO |z_i - z_j|.  A live range (i < nlive; nodes past nlive are not
// read by dd_update) outside those bounds is evaluated on its own nodes
// sorted (dd_set).
template <typename T, int NR>
__device__ __forceinline__ void dd_exp_ranges(const T (&z)[NR], const T (&ez)[NR], int nlive,
                                              T (&D)[1 << NR]) {
  using P = DDParams<T>;
#pragma unroll
  for (int i = 0; i < NR; ++i) D[1 << i] = ez[i];
  // spread of every range from running extremes
  T S[NR][NR];
  bool close = false;  // some live range has spread below TAU
  T smax = T(0);       // the largest such spread
#pragma unroll
  for (int j = 0; j < NR; ++j) {
    T mn = z[j], mx = z[j];
#pragma unroll
    for (int i = j + 1; i < NR; ++i) {
      mn = fmin(mn, z[i]);
      mx = fmax(mx, z[i]);
      const T s = mx - mn;
      S[j][i] = s;
      if (i < nlive) {
        close = close || s < P::tau;
        smax = s < P::tau ? fmax(smax, s) : smax;
      }
    }
  }
  T C[NR][NR];
#pragma unroll
  for (int a = 0; a < NR; ++a)
#pragma unroll
    for (int b = 0; b < NR; ++b) C[a][b] = T(0);
  if (close) taylor_chains<T, NR>(z, P::kUniform ? P::RMAX : P::terms(smax, P::RMAX), C);
#pragma unroll
  for (int len = 2; len <= NR; ++len) {
#pragma unroll
    for (int j = 0; j + len <= NR; ++j) {
      const int i = j + len - 1;
      const T s = S[j][i];
      const T dz = z[i] - z[j];
      T d;
      if (s < P::tau) {
        d = ez[j] * C[j][i];
      } else if (len > 2 && i < nlive &&
                 (fabs(dz) < P::tau || s > P::end_ratio * fabs(dz))) {
        // the range's own nodes, padded with z = 0 (the largest a node can be)
        d = dd_set<T>(z[j], z[j + 1], z[j + 2 < NR ? j + 2 : j],
                      len > 3 ? z[j + 3 < NR ? j + 3 : j] : T(0),
                      len > 4 ? z[j + 4 < NR ? j + 4 : j] : T(0), ez[j], ez[j + 1],
                      ez[j + 2 < NR ? j + 2 : j], len > 3 ? ez[j + 3 < NR ? j + 3 : j] : T(1),
                      len > 4 ? ez[j + 4 < NR ? j + 4 : j] : T(1), len);
      } else {
        d = P::div(D[range_mask(j + 1, i)] - D[range_mask(j, i - 1)], dz);
      }
      D[range_mask(j, i)] = d;
    }
  }
}

// exp[z_0, ..., z_{m-1}] (3 <= m <= 5; the slots past m hold z = 0,
// e^z = 1): the nodes sorted by a 9-comparator network, then the table of
// their contiguous ranges level by level in place (d[j] = D[j..j+len-1]):
// removing the smallest and the largest node, or the Taylor series about
// the largest node below TAU.  Kept out of line and in loops: only ranges
// with close ends and a far inner node come here.
template <typename T>
__device__ __noinline__ T dd_set(T z0, T z1, T z2, T z3, T z4, T e0, T e1, T e2, T e3, T e4,
                                 int m) {
  using P = DDParams<T>;
  T z[5] = {z0, z1, z2, z3, z4};
  T d[5] = {e0, e1, e2, e3, e4};
  constexpr int kNet[9][2] = {{0, 1}, {3, 4}, {2, 4}, {2, 3}, {0, 3},
                              {0, 2}, {1, 4}, {1, 3}, {1, 2}};
#pragma unroll
  for (int c = 0; c < 9; ++c) {
    const int p = kNet[c][0], q = kNet[c][1];
    const bool sw = z[p] > z[q];
    const T zp = z[p], dp = d[p];
    z[p] = sw ? z[q] : zp;
    d[p] = sw ? d[q] : dp;
    z[q] = sw ? zp : z[q];
    d[q] = sw ? dp : d[q];
  }
#pragma unroll 1
  for (int len = 2; len <= m; ++len) {
#pragma unroll 1
    for (int j = 0; j + len <= m; ++j) {
      const int i = j + len - 1;
      const T zi = z[i], s = zi - z[j];
      if (s >= P::tau) {
        d[j] = P::div(d[j + 1] - d[j], s);
      } else {
        const int R = P::kUniform ? P::RMAX : P::terms(s, P::RMAX);
        T H[P::RMAX + 1];
        H[0] = T(1);
#pragma unroll
        for (int r = 1; r <= P::RMAX; ++r) H[r] = T(0);
#pragma unroll 1
        for (int k = j; k < i; ++k) {
          const T x = z[k] - zi;
#pragma unroll
          for (int r = 1; r <= P::RMAX; ++r)
            if (r <= R) H[r] = fma(x, H[r - 1], H[r]);
        }
        T acc = T(0);
#pragma unroll
        for (int r = P::RMAX; r >= 0; --r)
          if (r <= R) acc = fma(H[r], P::inv_fact(len - 1 + r), acc);
        d[j] = exp(zi) * acc;
      }
    }
  }
  return d[0];
}

// Small rates: N' = sum_k (dt A)^k N / k! applied to the window vector
// directly.  With every W dt <= prop_max the norm of dt A is at most
// 2 prop_max, the terms shrink from the first, and R terms leave a remainder
// below (2 prop_max)^(R+1)/(R+1)!.  inc[] collects N' - N without forming
// the difference, so the freed electrons carry no cancellation.
//   v, lam, w as in dd_update below; returns the electrons released.
template <typename T, int WM, int PMAX = DDParams<T>::PMAX>
__device__ __forceinline__ T taylor_propagate(T (&v)[WM], const T (&lam)[WM],
                                              int w, T lmax) {
  using P = DDParams<T>;
  const int R = P::terms(T(2) * lmax, PMAX);
  T t[WM], inc[WM];
#pragma unroll
  for (int i = 0; i < WM; ++i) {
    t[i] = i < w ? v[i] : T(0);
    inc[i] = T(0);
  }
#pragma unroll
  for (int k = 1; k <= PMAX; ++k) {
    if (k > R) break;
    const T rk = T(1.0 / k);
#pragma unroll
    for (int i = WM - 1; i >= 0; --i) {
      const T gain = i > 0 ? lam[i - 1] * t[i - 1] : T(0);
      t[i] = (gain - lam[i] * t[i]) * rk;
      inc[i] += t[i];
    }
  }
  T cum = T(0), dne = T(0);
#pragma unroll
  for (int r = 0; r < WM; ++r) {
    if (r < w - 1) {
      cum -= inc[r];  // population that left states <= r
      dne += cum;
    }
    if (r < w) v[r] += inc[r];
  }
  return dne;
}

// ---------------------------------------------------------------------------
// Windowed update of one cell (Eqs. 3-9) with the divided-difference
// (Bateman) coefficients.
//   v[0..w-1]  populations of the window states lo..hi (in), N' (out);
//              entries r >= w are left alone.
//   lam[r]     W_{lo+r} dt for r < w-1; lam[r] = 0 for r >= w-1 (the top
//              state of the window absorbs, as in Eqs. 6-9).
//   WM         compile-time bound on w (2 <= w <= WM).
// Rows r < w-1 use the coefficients; the absorbing top state gets what the
// others lost, so the window's sum is kept (Eq. 9 is 1 - Eqs. 6-8 column by
// column).  Returns the electrons released, sum_k k (N'_k - N_k) = the sum
// over the w-1 internal boundaries of the population that crossed them.
// (Cells whose rates are all small take taylor_propagate instead.)
// ---------------------------------------------------------------------------
template <typename T, int WM>
__device__ __forceinline__ T dd_update(T (&v)[WM], const T (&lam)[WM], int w) {
  constexpr int NR = WM - 1;
  T z[NR], ez[NR];
#pragma unroll
  for (int r = 0; r < NR; ++r) {
    const T l = r < w - 1 ? lam[r] : T(0);
    z[r] = -l;
    ez[r] = exp(-l);
  }
  // (Rates fall along the window in the usual ladder near threshold, each
  // state harder to ionize than the one below, and rise far above the
  // barrier, where Eq. 1 grows with the charge; both give ranges whose ends
  // are their extremes.)  Only the window's own w-1 nodes are judged, so
  // that the result does not depend on the bound WM.
  T D[1 << NR];
  dd_exp_ranges<T, NR>(z, ez, w - 1, D);
  T out[NR];
#pragma unroll
  for (int i = 0; i < NR; ++i) {
    T acc = T(0), prod = T(1);
#pragma unroll
    for (int j = i; j >= 0; --j) {
      if (j < i) prod *= (j < w - 1 ? lam[j] : T(0));
      acc = fma(prod * D[range_mask(j, i)], v[j], acc);
    }
    out[i] = acc;
  }
  // electrons: flux across boundary b (between b and b+1) is S_b - S'_b
  T S = T(0), S1 = T(0), dne = T(0), tot = T(0), lost = T(0);
#pragma unroll
  for (int r = 0; r < WM; ++r) tot += r < w ? v[r] : T(0);
#pragma unroll
  for (int r = 0; r < NR; ++r) {
    if (r < w - 1) {
      S += v[r];
      S1 += out[r];
      dne += S - S1;
      lost += out[r];
    }
  }
  const T top = tot - lost;
#pragma unroll
  for (int r = 0; r < WM; ++r) {
    if (r < w - 1)
      v[r] = out[r];
    else if (r == w - 1)
      v[r] = top;
  }
  return dne;
}

// North-star degeneracy test: some pair of the window's rates with
// |W_i - W_j| < gap * max(W_i, W_j).
template <typename T, int WM>
__device__ __forceinline__ bool near_degenerate(const T (&lam)[WM], int w,
                                                T gap) {
  bool deg = false;
#pragma unroll
  for (int i = 0; i < WM - 1; ++i)
#pragma unroll
    for (int j = i + 1; j < WM - 1; ++j)
      if (j < w - 1)
        deg |= fabs(lam[i] - lam[j]) < gap * fmax(lam[i], lam[j]);
  return deg;
}

// Window slide after the step (Sec. 3): while the lowest state holds less
// than eps and the top is below Z, move the window up one state, at most
// w-1 times.  lo/hi are updated in place.
template <typename T, int WM>
__device__ __forceinline__ void slide_window(const T (&v)[WM], int w, int Z,
                                             T eps, int& lo, int& hi) {
  bool go = true;
#pragma unroll
  for (int r = 0; r < WM - 1; ++r) {
    go = go && (r < w - 1) && (hi < Z) && (v[r] < eps);
    lo += go ? 1 : 0;
    hi += go ? 1 : 0;
  }
}

// Adaptive window (ION_WINDOW_ADAPTIVE), after the step: while the lowest
// state holds less than eps (at most w-1 moves) it is dropped if the width
// exceeds wmin, else the window slides (never past hi = Z); then, if the old
// top state holds more than eps_grow, the state above joins (width at most
// wmax, never past Z).  v is the window after the step, w its width.
// Kept out of line (scalar arguments, result lo | hi << 8) so that kernels
// running the fixed rule carry none of it.
template <typename T>
__device__ __noinline__ int adapt_window_call(T v0, T v1, T v2, T v3, T v4, T v5, int w, int Z,
                                              T eps, int wmin, int wmax, T eps_grow, int lo,
                                              int hi) {
  const T v[6] = {v0, v1, v2, v3, v4, v5};
  bool go = true;
#pragma unroll
  for (int r = 0; r < 5; ++r) {
    go = go && (r < w - 1) && (v[r] < eps);
    if (go) {
      if (hi - lo + 1 > wmin) {
        ++lo;
      } else if (hi < Z) {
        ++lo;
        ++hi;
      } else {
        go = false;
      }
    }
  }
  T top = T(0);
#pragma unroll
  for (int r = 0; r < 6; ++r) top = (r == w - 1) ? v[r] : top;
  if (top > eps_grow && hi < Z && hi - lo + 1 < wmax) ++hi;
  return lo | (hi << 8);
}

template <typename T, int WM>
__device__ __forceinline__ void adapt_window(const T (&v)[WM], int w, int Z, T eps, int wmin,
                                             int wmax, T eps_grow, int& lo, int& hi) {
  T u[6];
#pragma unroll
  for (int r = 0; r < 6; ++r) u[r] = r < WM ? v[r < WM ? r : 0] : T(0);
  const int p = adapt_window_call<T>(u[0], u[1], u[2], u[3], u[4], u[5], w, Z, eps, wmin, wmax,
                                     eps_grow, lo, hi);
  lo = p & 0xff;
  hi = p >> 8;
}

}  // namespace ion
