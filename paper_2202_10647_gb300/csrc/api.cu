// api.cu -- the C ABI of ionize.h: species tables, argument checking, the
// ion_rates kernel, and dispatch of ion_step to the FP32 or FP64 kernels.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>

#include "ion_device.cuh"
#include "ion_step.cuh"
#include "ionize.h"

struct ion_species {
  int device;
  int num_sms;
  int Z;
  ion::SpeciesTable host;
  ion::SpeciesTable* dev;
};

namespace {

thread_local std::string g_err;

int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

int ok() {
  g_err.clear();
  return ION_OK;
}

int cuda_fail(cudaError_t e, const char* what) {
  return fail(ION_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

double factorial(int n) {
  double f = 1.0;
  for (int i = 2; i <= n; ++i) f *= (double)i;
  return f;
}

bool aligned(const void* p, size_t a) {
  return (reinterpret_cast<uintptr_t>(p) % a) == 0;
}

// Species table in double on the host: log2 W[1/fs] = a2 - b log2|E| - C/|E|
// (the log2 form of Eq. 1 with x = E_a/|E|; see ion_device.cuh).
void build_table(const double* U, const int* l, const int* m, int Z,
                 const ion_constants& c, ion::SpeciesTable* t) {
  std::memset(t, 0, sizeof *t);
  t->Z = Z;
  const double omega_fs = c.omega_a_per_s * 1e-15;
  for (int k = 0; k < Z; ++k) {
    const double Q = (double)(k + 1);
    const int am = m[k] < 0 ? -m[k] : m[k];
    const double ns = Q * std::sqrt(c.U_H_eV / U[k]);
    const double b = 2.0 * ns - (double)am - 1.5;
    const double cnat = (2.0 / 3.0) * std::pow(Q / ns, 3.0);
    const double flm = (2.0 * l[k] + 1.0) * factorial(l[k] + am) /
                       (std::ldexp(1.0, am) * factorial(am) * factorial(l[k] - am));
    const double log2A =
        std::log2(omega_fs) + 0.5 * std::log2(3.0 * ns * ns * ns / (M_PI * Q * Q * Q)) +
        std::log2(Q * Q / (2.0 * ns * ns)) + 2.0 * ns * std::log2(2.0 * M_E / ns) +
        std::log2(flm / (2.0 * M_PI * ns)) +
        (2.0 * ns - (double)am - 1.0) * std::log2(2.0 * Q * Q * Q / (ns * ns * ns));
    t->a2[k] = log2A + b * std::log2(c.E_a_GVm);
    t->b[k] = b;
    t->C[k] = cnat * c.E_a_GVm / M_LN2;
  }
}

// ---------------------------------------------------------------------------
// ion_rates kernels: one thread per cell, rates of states k_lo..k_hi-1.
// ---------------------------------------------------------------------------
__global__ void rates_f32_kernel(const ion::SpeciesTable* t, const float* E,
                                 int ncells, int k_lo, int k_hi, float* W,
                                 int64_t ldw) {
  __shared__ ion::StagedF32 tab;
  ion::stage_f32(t, 0.0, &tab);
  __syncthreads();
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncells) return;
  const ion::FieldF32 f = ion::field_f32<true>(E[c]);
  for (int k = k_lo; k < k_hi; ++k)
    W[(int64_t)(k - k_lo) * ldw + c] = ion::rate_dt_f32<true>(tab, k, f);
}

__global__ void rates_f64_kernel(const ion::SpeciesTable* t, const double* E,
                                 int ncells, int k_lo, int k_hi, double* W,
                                 int64_t ldw) {
  __shared__ ion::StagedF64 tab;
  ion::stage_f64(t, 0.0, &tab);
  __syncthreads();
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncells) return;
  const double e = E[c];
  for (int k = k_lo; k < k_hi; ++k)
    W[(int64_t)(k - k_lo) * ldw + c] = ion::rate_dt_f64(tab, k, e);
}

int check_species(const ion_species* sp) {
  if (!sp || !sp->dev) return fail(ION_EINVAL, "species is NULL or destroyed");
  return ION_OK;
}

}  // namespace

int ion::set_error(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

extern "C" {

const char* ion_last_error(void) { return g_err.c_str(); }

int ion_species_init(const double* U_ion_eV, const int* l, const int* m, int Z,
                     const ion_constants* c, ion_species** out) {
  if (!out) return fail(ION_EINVAL, "out is NULL");
  *out = nullptr;
  if (!U_ion_eV || !l || !m) return fail(ION_EINVAL, "U_ion_eV, l and m must be non-NULL");
  if (Z < 1 || Z > ION_MAX_Z) return fail(ION_EINVAL, "Z=%d outside [1, %d]", Z, ION_MAX_Z);
  for (int k = 0; k < Z; ++k) {
    const int am = m[k] < 0 ? -m[k] : m[k];
    if (!(U_ion_eV[k] > 0.0) || !std::isfinite(U_ion_eV[k]))
      return fail(ION_EINVAL, "U_ion_eV[%d] must be finite and > 0", k);
    if (l[k] < 0 || l[k] > 20 || am > l[k])
      return fail(ION_EINVAL, "state %d: need 0 <= |m| <= l <= 20 (l=%d m=%d)", k, l[k], m[k]);
  }
  ion_constants cc = {4.13e16, 510.0, 13.6};
  if (c) {
    if (!(c->omega_a_per_s > 0) || !(c->E_a_GVm > 0) || !(c->U_H_eV > 0))
      return fail(ION_EINVAL, "constants must be > 0");
    cc = *c;
  }
  ion_species* sp = new (std::nothrow) ion_species();
  if (!sp) return fail(ION_ENOMEM, "host allocation failed");
  build_table(U_ion_eV, l, m, Z, cc, &sp->host);
  sp->Z = Z;
  cudaError_t e = cudaGetDevice(&sp->device);
  if (e == cudaSuccess)
    e = cudaDeviceGetAttribute(&sp->num_sms, cudaDevAttrMultiProcessorCount, sp->device);
  if (e != cudaSuccess) {
    delete sp;
    return cuda_fail(e, "no usable CUDA device");
  }
  e = cudaMalloc(&sp->dev, sizeof(ion::SpeciesTable));
  if (e != cudaSuccess) {
    delete sp;
    return fail(ION_ENOMEM, "cudaMalloc of the species table: %s", cudaGetErrorString(e));
  }
  e = cudaMemcpy(sp->dev, &sp->host, sizeof(ion::SpeciesTable), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaFree(sp->dev);
    delete sp;
    return cuda_fail(e, "copy of the species table");
  }
  *out = sp;
  return ok();
}

int ion_species_destroy(ion_species* sp) {
  if (!sp) return ok();
  if (sp->dev) cudaFree(sp->dev);
  sp->dev = nullptr;
  delete sp;
  return ok();
}

int ion_species_z(const ion_species* sp) {
  int rc = check_species(sp);
  return rc ? rc : sp->Z;
}

int ion_rates(const ion_species* sp, const void* E, int64_t ncells, int k_lo,
              int k_hi, void* W_out, int64_t ldw, int dtype, void* stream) {
  int rc = check_species(sp);
  if (rc) return rc;
  if (ncells < 0 || ncells >= (int64_t(1) << 31))
    return fail(ION_EINVAL, "ncells=%lld outside [0, 2^31)", (long long)ncells);
  if (k_lo < 0 || k_hi > sp->Z || k_lo > k_hi)
    return fail(ION_EINVAL, "need 0 <= k_lo <= k_hi <= Z (k_lo=%d k_hi=%d Z=%d)", k_lo, k_hi, sp->Z);
  if (dtype != ION_DTYPE_F32 && dtype != ION_DTYPE_F64)
    return fail(ION_EINVAL, "dtype must be ION_DTYPE_F32 or ION_DTYPE_F64");
  if (ncells == 0 || k_lo == k_hi) return ok();
  if (!E || !W_out) return fail(ION_EINVAL, "E and W_out must be non-NULL");
  if (ldw < ncells) return fail(ION_EINVAL, "ldw < ncells");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int threads = 256;
  const int blocks = (int)((ncells + threads - 1) / threads);
  if (dtype == ION_DTYPE_F32)
    rates_f32_kernel<<<blocks, threads, 0, s>>>(sp->dev, static_cast<const float*>(E),
                                                (int)ncells, k_lo, k_hi,
                                                static_cast<float*>(W_out), ldw);
  else
    rates_f64_kernel<<<blocks, threads, 0, s>>>(sp->dev, static_cast<const double*>(E),
                                                (int)ncells, k_lo, k_hi,
                                                static_cast<double*>(W_out), ldw);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? ok() : cuda_fail(e, "ion_rates launch");
}

size_t ion_step_workspace_bytes(int64_t ncells, int flags) {
  if (ncells < 0) ncells = 0;
  return ion::step_workspace_bytes(ncells, (flags & ION_F64_PLAIN) != 0);
}

int ion_step(const ion_species* sp, const void* E, void* N, int64_t ld,
             int64_t ncells, double dt_fs, uint8_t* k_lo, uint8_t* k_hi,
             void* dne, const void* n_gas, const ion_step_opts* opts, int flags,
             void* workspace, size_t workspace_bytes, void* stream) {
  int rc = check_species(sp);
  if (rc) return rc;
  const int known = ION_F64_PLAIN | ION_NO_WINDOW_UPDATE | ION_NO_FP64_FALLBACK |
                    ION_FORCE_FP64_COEF;
  if (flags & ~known) return fail(ION_EINVAL, "unknown flag bits 0x%x", flags & ~known);
  const bool f64 = (flags & ION_F64_PLAIN) != 0;
  if (f64 && (flags & (ION_NO_FP64_FALLBACK | ION_FORCE_FP64_COEF)))
    return fail(ION_EINVAL, "fallback flags apply to ION_F32 only");
  if ((flags & ION_NO_FP64_FALLBACK) && (flags & ION_FORCE_FP64_COEF))
    return fail(ION_EINVAL, "ION_NO_FP64_FALLBACK and ION_FORCE_FP64_COEF exclude each other");
  if (ncells < 0 || ncells >= (int64_t(1) << 31))
    return fail(ION_EINVAL, "ncells=%lld outside [0, 2^31)", (long long)ncells);
  if (!(dt_fs >= 0.0) || !std::isfinite(dt_fs))
    return fail(ION_EINVAL, "dt_fs must be finite and >= 0 (got %g)", dt_fs);
  ion_step_opts o = {1e-6, 1e-3};
  if (opts) o = *opts;
  if (!(o.eps_shift >= 0.0) || !std::isfinite(o.eps_shift))
    return fail(ION_EINVAL, "eps_shift must be finite and >= 0");
  if (!(o.degen_gap >= 0.0) || !(o.degen_gap < 1.0))
    return fail(ION_EINVAL, "degen_gap must lie in [0, 1)");
  if (!workspace) return fail(ION_EINVAL, "workspace is NULL");
  const size_t need = ion_step_workspace_bytes(ncells, flags);
  if (workspace_bytes < need)
    return fail(ION_EINVAL, "workspace has %zu bytes, %zu needed", workspace_bytes, need);
  if (!aligned(workspace, 256)) return fail(ION_EINVAL, "workspace must be 256-byte aligned");
  if (ncells > 0) {
    if (!E || !N || !k_lo || !k_hi || !dne)
      return fail(ION_EINVAL, "E, N, k_lo, k_hi and dne must be non-NULL");
    if (ld < ncells) return fail(ION_EINVAL, "ld=%lld < ncells", (long long)ld);
    if (ld > (int64_t(1) << 40)) return fail(ION_EINVAL, "ld too large");
    const size_t el = f64 ? 8 : 4;
    if (!aligned(E, el) || !aligned(N, el) || !aligned(dne, el) ||
        (n_gas && !aligned(n_gas, el)))
      return fail(ION_EINVAL, "E, N, dne and n_gas must be aligned to their element size");
    if (!f64 && (!aligned(k_lo, 4) || !aligned(k_hi, 4)))
      return fail(ION_EINVAL, "k_lo and k_hi must be 4-byte aligned");
  }
  ion::StepArgs a;
  a.tab = sp->dev;
  a.Z = sp->Z;
  a.E = E;
  a.N = N;
  a.ld = ld;
  a.ncells = (int)ncells;
  a.zero_dt = dt_fs == 0.0;
  a.log2dt = dt_fs > 0.0 ? std::log2(dt_fs) : 0.0;
  a.lo = k_lo;
  a.hi = k_hi;
  a.dne = dne;
  a.n_gas = n_gas;
  a.eps = o.eps_shift;
  a.gap = o.degen_gap;
  a.flags = flags;
  a.vec = aligned(E, 16) && aligned(N, 16) && aligned(dne, 16) && (ld % 4) == 0;
  ion::bind_workspace(a, workspace);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = f64 ? ion::launch_step_f64(a, s) : ion::launch_step_f32(a, sp->num_sms, s);
  return e == cudaSuccess ? ok() : cuda_fail(e, "ion_step launch");
}

}  // extern "C"
