// mlp_train.cu -- training of the rate surrogate on the GPU: the loss and its
// gradient for a batch (forward pass, chain rule, batch reductions), the Adam
// update, and a plain (CUDA-core) forward pass used as the reference of the
// tensor-core inference.  Network and parameter layout: mlp_device.cuh.
//
//   loss  L = (1/(B K)) sum_b sum_k (y_bk - t_bk)^2
//   mlp_fwd, mlp_bwd  one thread per sample: the forward pass, then the
//                   backward pass down to dL/dz1; they write the per-sample
//                   factors of the weight gradients (h1, h2, dL/dz1, dL/dz2,
//                   dL/dy).
//   mlp_grad_part   one thread per parameter and batch slice: the sum over
//                   the slice's samples of the outer-product terms.
//   mlp_grad_sum    sums the slices in a fixed order (deterministic), and the
//                   per-block loss partials.
//   mlp_adam        Adam with bias-corrected moments.
// With ION_MLP_BF16 the forward pass rounds W2, W3, h1 and h2 to their
// bf16 pairs (split_round) and takes the SFU tanh, as the tensor-core
// inference does; the backward pass then treats the rounding as the identity
// (straight-through).
#include <cmath>
#include <cstdint>

#include "ion_step.cuh"
#include "ionize.h"
#include "mlp_device.cuh"

namespace ion {
namespace mlp {
namespace {

constexpr int kThreads = 128;
constexpr int kSlices = 16;

struct Acts {
  float* h1;    // [B][H]
  float* h2;    // [B][H]
  float* dz1;   // [B][H]
  float* dz2;   // [B][H]
  float* dy;    // [B][KP]
  float* part;  // [kSlices][nparams]
  float* lossp; // [blocks]
};

size_t round256(size_t x) { return (x + 255) / 256 * 256; }

int fwd_blocks(int64_t B) { return (int)((B + kThreads - 1) / kThreads); }

size_t ws_bytes(int K, int64_t B) {
  const size_t b = (size_t)B;
  return 4 * round256(4 * b * H) + round256(4 * b * padded_out(K)) +
         round256(4 * (size_t)kSlices * nparams(K)) + round256(4 * (size_t)fwd_blocks(B));
}

Acts bind(void* ws, int K, int64_t B) {
  char* p = static_cast<char*>(ws);
  const size_t b = (size_t)B;
  Acts a;
  a.h1 = reinterpret_cast<float*>(p);
  p += round256(4 * b * H);
  a.h2 = reinterpret_cast<float*>(p);
  p += round256(4 * b * H);
  a.dz1 = reinterpret_cast<float*>(p);
  p += round256(4 * b * H);
  a.dz2 = reinterpret_cast<float*>(p);
  p += round256(4 * b * H);
  a.dy = reinterpret_cast<float*>(p);
  p += round256(4 * b * padded_out(K));
  a.part = reinterpret_cast<float*>(p);
  p += round256(4 * (size_t)kSlices * nparams(K));
  a.lossp = reinterpret_cast<float*>(p);
  return a;
}

// The network staged in shared memory; output rows k >= K are zero.
template <int KP>
struct Net {
  float W1[H], b1[H], b2[H];
  float W2[H * H];
  float W3[KP * H];
  float b3[KP];
};

template <int KP, bool Q>
__device__ __forceinline__ void stage(const float* __restrict__ P, int K, Net<KP>& n) {
  for (int i = threadIdx.x; i < H; i += blockDim.x) {
    n.W1[i] = P[off_W1() + i];
    n.b1[i] = P[off_b1() + i];
    n.b2[i] = P[off_b2() + i];
  }
  for (int i = threadIdx.x; i < H * H; i += blockDim.x) {
    const float w = P[off_W2() + i];
    n.W2[i] = Q ? split_round(w) : w;
  }
  for (int i = threadIdx.x; i < KP * H; i += blockDim.x) {
    const float w = i < K * H ? P[off_W3() + i] : 0.0f;
    n.W3[i] = Q ? split_round(w) : w;
  }
  for (int k = threadIdx.x; k < KP; k += blockDim.x) n.b3[k] = k < K ? P[off_b3(K) + k] : 0.0f;
}

// The loops over hidden units o are kept rolled: each iteration is a dot
// product over the register arrays (h1, y, dy, acc) fully unrolled, so the
// arrays stay in registers at a modest code size.

// Training forward pass: h1, z2 (pre-activation of layer 2), h2, dL/dy and
// the block's partial of sum (y - t)^2.
template <int KP, bool Q>
__global__ void __launch_bounds__(kThreads)
    mlp_fwd(const float* __restrict__ P, int K, const float* __restrict__ x,
            const float* __restrict__ t, int B, float two_over_BK, Acts a) {
  __shared__ Net<KP> n;
  __shared__ float red[kThreads / 32];
  stage<KP, Q>(P, K, n);
  __syncthreads();
  const int b = blockIdx.x * kThreads + threadIdx.x;
  const bool on = b < B;
  const int bb = on ? b : 0;
  const float xb = on ? x[b] : 0.0f;
  float h1[H];
#pragma unroll
  for (int i = 0; i < H; ++i) {
    const float h = gelu<Q>(fmaf(n.W1[i], xb, n.b1[i]));
    h1[i] = Q ? split_round(h) : h;
    if (on) a.h1[(int64_t)b * H + i] = h1[i];
  }
  float y[KP];
#pragma unroll
  for (int k = 0; k < KP; ++k) y[k] = n.b3[k];
#pragma unroll 1
  for (int o = 0; o < H; ++o) {
    float z = n.b2[o];
#pragma unroll
    for (int i = 0; i < H; ++i) z = fmaf(n.W2[o * H + i], h1[i], z);
    float h = gelu<Q>(z);
    h = Q ? split_round(h) : h;
    if (on) {
      a.dz2[(int64_t)bb * H + o] = z;  // z2, overwritten by dL/dz2 later
      a.h2[(int64_t)bb * H + o] = h;
    }
#pragma unroll
    for (int k = 0; k < KP; ++k) y[k] = fmaf(n.W3[k * H + o], h, y[k]);
  }
  float l = 0.0f;
#pragma unroll
  for (int k = 0; k < KP; ++k) {
    const float d = (on && k < K) ? y[k] - t[(int64_t)b * K + k] : 0.0f;
    l = fmaf(d, d, l);
    if (on) a.dy[(int64_t)b * KP + k] = two_over_BK * d;  // dL/dy
  }
#pragma unroll
  for (int s = 16; s > 0; s >>= 1) l += __shfl_xor_sync(0xffffffffu, l, s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = l;
  __syncthreads();
  if (threadIdx.x == 0) {
    float s = 0.0f;
#pragma unroll
    for (int w = 0; w < kThreads / 32; ++w) s += red[w];
    a.lossp[blockIdx.x] = s;
  }
}

// Training backward pass: dL/dz2 (in place of z2) and dL/dz1.
template <int KP, bool Q>
__global__ void __launch_bounds__(kThreads)
    mlp_bwd(const float* __restrict__ P, int K, const float* __restrict__ x, int B, Acts a) {
  __shared__ Net<KP> n;
  stage<KP, Q>(P, K, n);
  __syncthreads();
  const int b = blockIdx.x * kThreads + threadIdx.x;
  if (b >= B) return;
  const float xb = x[b];
  float dy[KP], acc[H];
#pragma unroll
  for (int k = 0; k < KP; ++k) dy[k] = a.dy[(int64_t)b * KP + k];
#pragma unroll
  for (int i = 0; i < H; ++i) acc[i] = 0.0f;
#pragma unroll 1
  for (int o = 0; o < H; ++o) {
    float g = 0.0f;
#pragma unroll
    for (int k = 0; k < KP; ++k) g = fmaf(dy[k], n.W3[k * H + o], g);
    const float z = a.dz2[(int64_t)b * H + o];
    float th;
    gelu<Q>(z, th);
    const float d = g * gelu_grad(z, th);  // dL/dz2
    a.dz2[(int64_t)b * H + o] = d;
#pragma unroll
    for (int i = 0; i < H; ++i) acc[i] = fmaf(d, n.W2[o * H + i], acc[i]);
  }
#pragma unroll
  for (int i = 0; i < H; ++i) {
    const float z1 = fmaf(n.W1[i], xb, n.b1[i]);
    float th;
    gelu<Q>(z1, th);
    a.dz1[(int64_t)b * H + i] = acc[i] * gelu_grad(z1, th);
  }
}

// Parameter p's sum over the samples of slice blockIdx.y.
__global__ void __launch_bounds__(kThreads)
    mlp_grad_part(int K, int KP, const float* __restrict__ x, int B, Acts a) {
  const int np = nparams(K);
  const int p = blockIdx.x * kThreads + threadIdx.x;
  if (p >= np) return;
  const int s = blockIdx.y;
  const int b0 = (int)((int64_t)B * s / kSlices), b1 = (int)((int64_t)B * (s + 1) / kSlices);
  // each parameter is the sum over samples of u[b] * v[b]
  const float* u;
  const float* v = nullptr;  // nullptr: v = 1 (biases)
  int64_t su, sv = 0;
  if (p < off_b1()) {  // W1[i]: dz1[b][i] x[b]
    u = a.dz1 + p;
    su = H;
    v = x;
    sv = 1;
  } else if (p < off_W2()) {  // b1[i]
    u = a.dz1 + (p - off_b1());
    su = H;
  } else if (p < off_b2()) {  // W2[o][i]: dz2[b][o] h1[b][i]
    const int q = p - off_W2();
    u = a.dz2 + q / H;
    su = H;
    v = a.h1 + q % H;
    sv = H;
  } else if (p < off_W3()) {  // b2[o]
    u = a.dz2 + (p - off_b2());
    su = H;
  } else if (p < off_b3(K)) {  // W3[k][o]: dy[b][k] h2[b][o]
    const int q = p - off_W3();
    u = a.dy + q / H;
    su = KP;
    v = a.h2 + q % H;
    sv = H;
  } else {  // b3[k]
    u = a.dy + (p - off_b3(K));
    su = KP;
  }
  float acc = 0.0f;
  if (v) {
    for (int b = b0; b < b1; ++b) acc = fmaf(u[(int64_t)b * su], v[(int64_t)b * sv], acc);
  } else {
    for (int b = b0; b < b1; ++b) acc += u[(int64_t)b * su];
  }
  a.part[(int64_t)s * np + p] = acc;
}

__global__ void __launch_bounds__(kThreads)
    mlp_grad_sum(int np, int nloss, Acts a, float* __restrict__ grad, float* __restrict__ loss,
                 float inv_BK) {
  const int p = blockIdx.x * kThreads + threadIdx.x;
  if (p < np) {
    float g = 0.0f;
#pragma unroll
    for (int s = 0; s < kSlices; ++s) g += a.part[(int64_t)s * np + p];
    grad[p] = g;
  }
  if (p == 0 && loss) {
    float l = 0.0f;
    for (int i = 0; i < nloss; ++i) l += a.lossp[i];
    *loss = l * inv_BK;
  }
}

__global__ void __launch_bounds__(256)
    mlp_adam(float* __restrict__ P, const float* __restrict__ g, float* __restrict__ m,
             float* __restrict__ v, int64_t n, float lr, float b1, float b2, float eps,
             float bc1, float bc2) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = fmaf(b1, m[i], (1.0f - b1) * gi);
    const float vi = fmaf(b2, v[i], (1.0f - b2) * gi * gi);
    m[i] = mi;
    v[i] = vi;
    P[i] -= lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
  }
}

template <int KP, bool Q>
__global__ void __launch_bounds__(kThreads)
    mlp_forward(const float* __restrict__ P, int K, const float* __restrict__ x, int B,
                float* __restrict__ y_out) {
  __shared__ Net<KP> n;
  stage<KP, Q>(P, K, n);
  __syncthreads();
  const int b = blockIdx.x * kThreads + threadIdx.x;
  if (b >= B) return;
  const float xb = x[b];
  float h1[H];
#pragma unroll
  for (int i = 0; i < H; ++i) {
    const float h = gelu<Q>(fmaf(n.W1[i], xb, n.b1[i]));
    h1[i] = Q ? split_round(h) : h;
  }
  float y[KP];
#pragma unroll
  for (int k = 0; k < KP; ++k) y[k] = n.b3[k];
#pragma unroll 1
  for (int o = 0; o < H; ++o) {
    float z = n.b2[o];
#pragma unroll
    for (int i = 0; i < H; ++i) z = fmaf(n.W2[o * H + i], h1[i], z);
    float h = gelu<Q>(z);
    h = Q ? split_round(h) : h;
#pragma unroll
    for (int k = 0; k < KP; ++k) y[k] = fmaf(n.W3[k * H + o], h, y[k]);
  }
#pragma unroll
  for (int k = 0; k < KP; ++k)
    if (k < K) y_out[(int64_t)b * K + k] = y[k];
}

template <int KP>
cudaError_t launch_fwd_bwd(bool q, const float* P, int K, const float* x, const float* t, int B,
                           float two_over_BK, const Acts& a, cudaStream_t s) {
  const int g = fwd_blocks(B);
  if (q) {
    mlp_fwd<KP, true><<<g, kThreads, 0, s>>>(P, K, x, t, B, two_over_BK, a);
    mlp_bwd<KP, true><<<g, kThreads, 0, s>>>(P, K, x, B, a);
  } else {
    mlp_fwd<KP, false><<<g, kThreads, 0, s>>>(P, K, x, t, B, two_over_BK, a);
    mlp_bwd<KP, false><<<g, kThreads, 0, s>>>(P, K, x, B, a);
  }
  return cudaGetLastError();
}

template <int KP>
cudaError_t launch_forward(bool q, const float* P, int K, const float* x, int B, float* y,
                           cudaStream_t s) {
  const int g = fwd_blocks(B);
  if (q)
    mlp_forward<KP, true><<<g, kThreads, 0, s>>>(P, K, x, B, y);
  else
    mlp_forward<KP, false><<<g, kThreads, 0, s>>>(P, K, x, B, y);
  return cudaGetLastError();
}

constexpr int64_t kMaxBatch = int64_t(1) << 24;

int check_common(const char* who, const float* P, int K, const float* x, int64_t B, int flags) {
  if (K < 1 || K > kMaxOut)
    return set_error(ION_EINVAL, "%s: K=%d outside [1, %d]", who, K, kMaxOut);
  if (B < 1 || B > kMaxBatch)
    return set_error(ION_EINVAL, "%s: B=%lld outside [1, 2^24]", who, (long long)B);
  if (!P || !x) return set_error(ION_EINVAL, "%s: NULL pointer", who);
  if (flags & ~ION_MLP_BF16) return set_error(ION_EINVAL, "%s: unknown flags 0x%x", who, flags);
  if ((reinterpret_cast<uintptr_t>(P) | reinterpret_cast<uintptr_t>(x)) % 4)
    return set_error(ION_EINVAL, "%s: arrays must be 4-byte aligned", who);
  return ION_OK;
}

// ---- training data ---------------------------------------------------------
// x = clamp(2 (log2|E| - l2lo) / (l2hi - l2lo) - 1, -1, 1) in FP64.
__global__ void mlp_inputs_kernel(const float* E, int64_t n, double l2lo, double l2hi,
                                  float* x) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double l2 = log2(fabs((double)E[i]));
  const double v = 2.0 * (l2 - l2lo) / (l2hi - l2lo) - 1.0;
  x[i] = (float)fmin(fmax(v, -1.0), 1.0);  // fmax of NaN and -1 is -1
}

constexpr int kColThreads = 1024;

// One block per column k of Y (n rows of K): the sum over the rows in a
// fixed order (thread t takes rows t, t + 1024, ...; then a tree over the
// threads).  Without `mean`: out[k] = sum / n.  With it: out[k] =
// max(sqrt(sum (Y - mean_k)^2 / (n - 1)), min_scale).
__global__ void __launch_bounds__(kColThreads)
    mlp_column_kernel(const double* Y, int64_t n, int K, const double* mean, double min_scale,
                      double* out) {
  __shared__ double part[kColThreads];
  const int k = blockIdx.x;
  const double m = mean ? mean[k] : 0.0;
  double acc = 0.0;
  for (int64_t r = threadIdx.x; r < n; r += kColThreads) {
    const double d = Y[r * K + k] - m;
    acc += mean ? d * d : d;
  }
  part[threadIdx.x] = acc;
  __syncthreads();
  for (int w = kColThreads / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) part[threadIdx.x] += part[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0)
    out[k] = mean ? fmax(sqrt(part[0] / (double)(n - 1)), min_scale) : part[0] / (double)n;
}

__global__ void mlp_normalize_kernel(const double* Y, int64_t n, int K, const double* mean,
                                     const double* scale, float* T) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n * K) return;
  const int k = (int)(i % K);
  T[i] = (float)((Y[i] - mean[k]) / scale[k]);
}

}  // namespace
}  // namespace mlp
}  // namespace ion

using namespace ion::mlp;

extern "C" {

int64_t ion_mlp_nparams(int K) {
  return (K < 1 || K > kMaxOut) ? (int64_t)ION_EINVAL : (int64_t)nparams(K);
}

size_t ion_mlp_workspace_bytes(int K, int64_t B) {
  if (K < 1 || K > kMaxOut || B < 1 || B > kMaxBatch) return 0;
  return ws_bytes(K, B);
}

int ion_mlp_loss_grad(const float* P, int K, const float* x, const float* t, int64_t B,
                      int flags, float* grad, float* loss, void* workspace,
                      size_t workspace_bytes, void* stream) {
  int rc = check_common("ion_mlp_loss_grad", P, K, x, B, flags);
  if (rc) return rc;
  if (!t || !grad) return ion::set_error(ION_EINVAL, "ion_mlp_loss_grad: NULL pointer");
  if (!workspace || workspace_bytes < ws_bytes(K, B) ||
      reinterpret_cast<uintptr_t>(workspace) % 256)
    return ion::set_error(ION_EINVAL,
                          "ion_mlp_loss_grad: workspace must be 256-byte aligned and hold "
                          "%zu bytes",
                          ws_bytes(K, B));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const Acts a = bind(workspace, K, B);
  const bool q = (flags & ION_MLP_BF16) != 0;
  const float two_over_BK = (float)(2.0 / ((double)B * K));
  const int KP = padded_out(K);
  cudaError_t e;
  switch (KP) {
    case 16:
      e = launch_fwd_bwd<16>(q, P, K, x, t, (int)B, two_over_BK, a, s);
      break;
    case 32:
      e = launch_fwd_bwd<32>(q, P, K, x, t, (int)B, two_over_BK, a, s);
      break;
    case 48:
      e = launch_fwd_bwd<48>(q, P, K, x, t, (int)B, two_over_BK, a, s);
      break;
    default:
      e = launch_fwd_bwd<64>(q, P, K, x, t, (int)B, two_over_BK, a, s);
      break;
  }
  if (e == cudaSuccess) {
    const int np = nparams(K);
    const dim3 grid((np + kThreads - 1) / kThreads, kSlices);
    mlp_grad_part<<<grid, kThreads, 0, s>>>(K, KP, x, (int)B, a);
    mlp_grad_sum<<<(np + kThreads - 1) / kThreads, kThreads, 0, s>>>(
        np, fwd_blocks(B), a, grad, loss, (float)(1.0 / ((double)B * K)));
    e = cudaGetLastError();
  }
  if (e != cudaSuccess)
    return ion::set_error(ION_ECUDA, "ion_mlp_loss_grad launch: %s", cudaGetErrorString(e));
  return ion::set_error(ION_OK, "%s", "");
}

int ion_mlp_adam(float* P, const float* grad, float* m, float* v, int64_t n, float lr,
                 float beta1, float beta2, float eps, int t, void* stream) {
  if (!P || !grad || !m || !v || n < 1)
    return ion::set_error(ION_EINVAL, "ion_mlp_adam: NULL pointer or n < 1");
  if (t < 1) return ion::set_error(ION_EINVAL, "ion_mlp_adam: step t=%d < 1", t);
  if (!(beta1 >= 0.0f && beta1 < 1.0f && beta2 >= 0.0f && beta2 < 1.0f && eps > 0.0f &&
        std::isfinite(lr)))
    return ion::set_error(ION_EINVAL, "ion_mlp_adam: bad hyper-parameters");
  const float bc1 = (float)(1.0 - std::pow((double)beta1, (double)t));
  const float bc2 = (float)(1.0 - std::pow((double)beta2, (double)t));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int64_t blocks = (n + 255) / 256;
  mlp_adam<<<(int)(blocks < 1024 ? blocks : 1024), 256, 0, s>>>(P, grad, m, v, n, lr, beta1,
                                                               beta2, eps, bc1, bc2);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess)
    return ion::set_error(ION_ECUDA, "ion_mlp_adam launch: %s", cudaGetErrorString(e));
  return ion::set_error(ION_OK, "%s", "");
}

int ion_mlp_forward(const float* P, int K, const float* x, int64_t B, int flags, float* y,
                    void* stream) {
  int rc = check_common("ion_mlp_forward", P, K, x, B, flags);
  if (rc) return rc;
  if (!y) return ion::set_error(ION_EINVAL, "ion_mlp_forward: y is NULL");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const bool q = (flags & ION_MLP_BF16) != 0;
  cudaError_t e;
  switch (padded_out(K)) {
    case 16:
      e = launch_forward<16>(q, P, K, x, (int)B, y, s);
      break;
    case 32:
      e = launch_forward<32>(q, P, K, x, (int)B, y, s);
      break;
    case 48:
      e = launch_forward<48>(q, P, K, x, (int)B, y, s);
      break;
    default:
      e = launch_forward<64>(q, P, K, x, (int)B, y, s);
      break;
  }
  if (e != cudaSuccess)
    return ion::set_error(ION_ECUDA, "ion_mlp_forward launch: %s", cudaGetErrorString(e));
  return ion::set_error(ION_OK, "%s", "");
}

int ion_mlp_inputs(const float* E, int64_t n, double l2lo, double l2hi, float* x,
                   void* stream) {
  if (n < 0 || n >= (int64_t(1) << 40))
    return ion::set_error(ION_EINVAL, "ion_mlp_inputs: n=%lld outside [0, 2^40)",
                          (long long)n);
  if (!(l2lo < l2hi) || !std::isfinite(l2lo) || !std::isfinite(l2hi))
    return ion::set_error(ION_EINVAL, "ion_mlp_inputs: need finite l2lo < l2hi");
  if (n == 0) return ion::set_error(ION_OK, "%s", "");
  if (!E || !x || (reinterpret_cast<uintptr_t>(E) & 3u) || (reinterpret_cast<uintptr_t>(x) & 3u))
    return ion::set_error(ION_EINVAL, "ion_mlp_inputs: E and x must be non-NULL, 4-byte aligned");
  const int64_t blocks = (n + 255) / 256;
  mlp_inputs_kernel<<<(unsigned)blocks, 256, 0, static_cast<cudaStream_t>(stream)>>>(
      E, n, l2lo, l2hi, x);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess)
    return ion::set_error(ION_ECUDA, "ion_mlp_inputs launch: %s", cudaGetErrorString(e));
  return ion::set_error(ION_OK, "%s", "");
}

int ion_mlp_standardize(const double* Y, int64_t n, int K, double min_scale, double* mean_out,
                        double* scale_out, float* T, void* stream) {
  if (n < 2 || n >= (int64_t(1) << 32))
    return ion::set_error(ION_EINVAL, "ion_mlp_standardize: n=%lld outside [2, 2^32)",
                          (long long)n);
  if (K < 1 || K > ION_MAX_Z)
    return ion::set_error(ION_EINVAL, "ion_mlp_standardize: K=%d outside [1, %d]", K,
                          ION_MAX_Z);
  if (!(min_scale > 0.0) || !std::isfinite(min_scale))
    return ion::set_error(ION_EINVAL, "ion_mlp_standardize: min_scale must be finite and > 0");
  auto al = [](const void* p, uintptr_t a) { return (reinterpret_cast<uintptr_t>(p) & (a - 1)) == 0; };
  if (!Y || !mean_out || !scale_out || !T || !al(Y, 8) || !al(mean_out, 8) ||
      !al(scale_out, 8) || !al(T, 4))
    return ion::set_error(ION_EINVAL,
                          "ion_mlp_standardize: Y, mean_out, scale_out (8-byte aligned) and T "
                          "(4-byte aligned) must be non-NULL");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  mlp_column_kernel<<<K, kColThreads, 0, s>>>(Y, n, K, nullptr, min_scale, mean_out);
  mlp_column_kernel<<<K, kColThreads, 0, s>>>(Y, n, K, mean_out, min_scale, scale_out);
  const int64_t blocks = (n * K + 255) / 256;
  mlp_normalize_kernel<<<(unsigned)blocks, 256, 0, s>>>(Y, n, K, mean_out, scale_out, T);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess)
    return ion::set_error(ION_ECUDA, "ion_mlp_standardize launch: %s", cudaGetErrorString(e));
  return ion::set_error(ION_OK, "%s", "");
}

}  // extern "C"
