// mlp_device.cuh -- device arithmetic of the rate surrogate's network, shared
// by the training kernels (mlp_train.cu) and the tensor-core inference
// (surrogate.cu):
//   h1 = g(W1 x + b1), h2 = g(W2 h1 + b2), y = W3 h2 + b3,
// H = 64 hidden units, K <= 63 outputs, g the GELU in its tanh form
//   g(z) = z/2 (1 + tanh(c (z + 0.044715 z^3))), c = sqrt(2/pi).
// Parameters are one FP32 array: W1[H], b1[H], W2[H][H] (row o = weights
// into unit o), b2[H], W3[K][H], b3[K].
#pragma once

#include <cuda_bf16.h>
#include <cstdint>

namespace ion {
namespace mlp {

constexpr int H = 64;
constexpr int kMaxOut = 63;
constexpr float kGeluC = 0.7978845608028654f;  // sqrt(2/pi)
constexpr float kGeluA = 0.044715f;

// Offsets into the flat parameter array.
__host__ __device__ constexpr int off_W1() { return 0; }
__host__ __device__ constexpr int off_b1() { return H; }
__host__ __device__ constexpr int off_W2() { return 2 * H; }
__host__ __device__ constexpr int off_b2() { return 2 * H + H * H; }
__host__ __device__ constexpr int off_W3() { return 3 * H + H * H; }
__host__ __device__ constexpr int off_b3(int K) { return 3 * H + H * H + K * H; }
__host__ __device__ constexpr int nparams(int K) { return 3 * H + H * H + K * H + K; }

// Output count rounded up to the padded widths the kernels are built for.
__host__ __device__ constexpr int padded_out(int K) {
  return K <= 16 ? 16 : K <= 32 ? 32 : K <= 48 ? 48 : 64;
}

__device__ __forceinline__ float tanh_approx(float x) {
  float y;
  asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ float bf16_round(float x) {
  return __bfloat162float(__float2bfloat16_rn(x));
}

// The inference arithmetic carries each value of W2, W3, h1 and h2 as a pair
// of bf16 numbers, hi = bf16(v) and lo = bf16(v - hi), and the tensor cores
// sum hi*hi' + hi*lo' + lo*hi' in FP32 (the lo*lo' product, about 2^-16 of
// the others, is left out).  The pair holds v to about 2^-16 relative;
// split_round is hi + lo (exact in FP32).
__device__ __forceinline__ float split_round(float x) {
  const float hi = bf16_round(x);
  return hi + bf16_round(x - hi);
}

// GELU and the tanh it used.  Fast: the SFU tanh (the inference arithmetic);
// otherwise tanhf.
template <bool Fast>
__device__ __forceinline__ float gelu(float z, float& t) {
  // u = c (z + a z^3) = z (c + c a z^2); g = z/2 + (z/2) t
  const float u = z * fmaf(kGeluC * kGeluA, z * z, kGeluC);
  t = Fast ? tanh_approx(u) : tanhf(u);
  const float hz = 0.5f * z;
  return fmaf(hz, t, hz);
}

template <bool Fast>
__device__ __forceinline__ float gelu(float z) {
  float t;
  return gelu<Fast>(z, t);
}

// gelu<true>(2 zh) from zh, bit for bit (every step is the same operation
// scaled by a power of two), with one multiplication less: the inference
// kernels keep W1, b1, W2 and b2 halved (exactly), so that their
// pre-activations arrive halved.
__device__ __forceinline__ float gelu_half(float zh) {
  const float u = zh * fmaf(8.0f * (kGeluC * kGeluA), zh * zh, 2.0f * kGeluC);
  return fmaf(zh, tanh_approx(u), zh);
}

// dg/dz given the tanh of the forward pass.
__device__ __forceinline__ float gelu_grad(float z, float t) {
  const float du = kGeluC * fmaf(3.0f * kGeluA, z * z, 1.0f);
  return fmaf(0.5f * z * (1.0f - t * t), du, 0.5f * (1.0f + t));
}

}  // namespace mlp
}  // namespace ion
