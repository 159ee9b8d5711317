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
    // the cycle-averaging factor sqrt(3 n*^3 |E| / (pi Q^3 E_a)) contributes
    // |E|^(1/2), i.e. -1/2 to the power of E_a/|E|
    const bool avg = c.rate_model != ION_ADK_STATIC;
    const double b = 2.0 * ns - (double)am - (avg ? 1.5 : 1.0);
    const double cnat = (2.0 / 3.0) * std::pow(Q / ns, 3.0);
    const double flm = (2.0 * l[k] + 1.0) * factorial(l[k] + am) /
                       (std::ldexp(1.0, am) * factorial(am) * factorial(l[k] - am));
    const double log2A =
        std::log2(omega_fs) +
        (avg ? 0.5 * std::log2(3.0 * ns * ns * ns / (M_PI * Q * Q * Q)) : 0.0) +
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
  const ion::FieldF64 f = ion::field_f64(E[c]);
  for (int k = k_lo; k < k_hi; ++k)
    W[(int64_t)(k - k_lo) * ldw + c] = ion::rate_dt_f64(tab, k, f);
}

__global__ void log2_rates_kernel(const ion::SpeciesTable* t, const float* E, int64_t ncells,
                                  int k_lo, int k_hi, double floor, double* out, int64_t ldo) {
  __shared__ ion::StagedF64 tab;
  ion::stage_f64(t, 0.0, &tab);
  __syncthreads();
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= ncells) return;
  const ion::FieldF64 f = ion::field_f64((double)E[c]);
  for (int k = k_lo; k < k_hi; ++k) out[c * ldo + (k - k_lo)] = ion::log2_rate_f64(tab, k, f, floor);
}

template <typename T>
__global__ void field_magnitude_kernel(const T* Ex, const T* Ey, const T* Ez, int64_t n,
                                       T* out) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= n) return;
  const T x = Ex[c];
  T e2 = x * x;
  if (Ey) e2 = fma(Ey[c], Ey[c], e2);
  if (Ez) e2 = fma(Ez[c], Ez[c], e2);
  out[c] = (Ey || Ez) ? sqrt(e2) : fabs(x);
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
  ion_constants cc = {4.13e16, 510.0, 13.6, ION_ADK_CYCLE_AVERAGED};
  if (c) {
    if (!(c->omega_a_per_s > 0) || !(c->E_a_GVm > 0) || !(c->U_H_eV > 0) ||
        !std::isfinite(c->omega_a_per_s) || !std::isfinite(c->E_a_GVm) ||
        !std::isfinite(c->U_H_eV))
      return fail(ION_EINVAL, "constants must be finite and > 0");
    if (c->rate_model != ION_ADK_CYCLE_AVERAGED && c->rate_model != ION_ADK_STATIC)
      return fail(ION_EINVAL, "unknown rate_model %d", c->rate_model);
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

int ion_log2_rates(const ion_species* sp, const float* E, int64_t ncells, int k_lo, int k_hi,
                   double floor, double* out, int64_t ldo, void* stream) {
  int rc = check_species(sp);
  if (rc) return rc;
  if (ncells < 0 || ncells >= (int64_t(1) << 31))
    return fail(ION_EINVAL, "ncells=%lld outside [0, 2^31)", (long long)ncells);
  if (k_lo < 0 || k_hi > sp->Z || k_lo >= k_hi)
    return fail(ION_EINVAL, "need 0 <= k_lo < k_hi <= Z (k_lo=%d, k_hi=%d, Z=%d)", k_lo, k_hi,
                sp->Z);
  if (!std::isfinite(floor)) return fail(ION_EINVAL, "floor must be finite");
  if (ncells == 0) return ok();
  if (!E || !out) return fail(ION_EINVAL, "E and out must be non-NULL");
  if ((reinterpret_cast<uintptr_t>(E) & 3u) || (reinterpret_cast<uintptr_t>(out) & 7u))
    return fail(ION_EINVAL, "E must be 4-byte and out 8-byte aligned");
  if (ldo < k_hi - k_lo) return fail(ION_EINVAL, "ldo=%lld < k_hi - k_lo", (long long)ldo);
  int cur = -1;
  if (cudaGetDevice(&cur) != cudaSuccess || cur != sp->device)
    return fail(ION_EINVAL, "the species lives on device %d; make it current", sp->device);
  const int threads = 256;
  const int64_t blocks = (ncells + threads - 1) / threads;
  log2_rates_kernel<<<(unsigned)blocks, threads, 0, static_cast<cudaStream_t>(stream)>>>(
      sp->dev, E, ncells, k_lo, k_hi, floor, out, ldo);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? ok() : cuda_fail(e, "ion_log2_rates launch");
}

size_t ion_step_workspace_bytes(int64_t ncells, int flags) {
  if (ncells < 0) ncells = 0;
  return ion::step_workspace_bytes(ncells, (flags & ION_F64_PLAIN) != 0);
}

int ion_field_magnitude(const void* Ex, const void* Ey, const void* Ez, int64_t ncells,
                        int dtype, void* E_abs, void* stream) {
  if (ncells < 0 || ncells >= (int64_t(1) << 31))
    return fail(ION_EINVAL, "ncells=%lld outside [0, 2^31)", (long long)ncells);
  if (dtype != ION_DTYPE_F32 && dtype != ION_DTYPE_F64)
    return fail(ION_EINVAL, "dtype must be ION_DTYPE_F32 or ION_DTYPE_F64");
  if (ncells == 0) return ok();
  if (!Ex || !E_abs) return fail(ION_EINVAL, "Ex and E_abs must be non-NULL");
  const uintptr_t a = dtype == ION_DTYPE_F32 ? 3u : 7u;
  for (const void* p : {Ex, Ey, Ez, static_cast<const void*>(E_abs)})
    if (reinterpret_cast<uintptr_t>(p) & a)
      return fail(ION_EINVAL, "the field arrays must be aligned to their element size");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const unsigned blocks = (unsigned)((ncells + 255) / 256);
  if (dtype == ION_DTYPE_F32)
    field_magnitude_kernel<float><<<blocks, 256, 0, s>>>(
        static_cast<const float*>(Ex), static_cast<const float*>(Ey),
        static_cast<const float*>(Ez), ncells, static_cast<float*>(E_abs));
  else
    field_magnitude_kernel<double><<<blocks, 256, 0, s>>>(
        static_cast<const double*>(Ex), static_cast<const double*>(Ey),
        static_cast<const double*>(Ez), ncells, static_cast<double*>(E_abs));
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? ok() : cuda_fail(e, "ion_field_magnitude launch");
}

size_t ion_step_field_workspace_bytes(int64_t ncells, int flags) {
  if (ncells < 0) ncells = 0;
  const size_t elem = (flags & ION_F64_PLAIN) ? 8 : 4;
  const size_t step = (ion_step_workspace_bytes(ncells, flags) + 255) / 256 * 256;
  return step + ((size_t)ncells * elem + 255) / 256 * 256;
}

}  // extern "C"

namespace {

int check_flags(int flags) {
  const int known = ION_F64_PLAIN | ION_NO_WINDOW_UPDATE | ION_NO_FP64_FALLBACK |
                    ION_FORCE_FP64_COEF | ION_CONSERVATION_CHECK;
  if (flags & ~known) return fail(ION_EINVAL, "unknown flag bits 0x%x", flags & ~known);
  const bool f64 = (flags & ION_F64_PLAIN) != 0;
  if (f64 && (flags & (ION_NO_FP64_FALLBACK | ION_FORCE_FP64_COEF)))
    return fail(ION_EINVAL, "fallback flags apply to ION_F32 only");
  if ((flags & ION_NO_FP64_FALLBACK) && (flags & ION_FORCE_FP64_COEF))
    return fail(ION_EINVAL, "ION_NO_FP64_FALLBACK and ION_FORCE_FP64_COEF exclude each other");
  return ION_OK;
}

int make_policy(double dt_fs, const ion_step_opts* opts, int flags, ion::Policy* pol) {
  if (!(dt_fs >= 0.0) || !std::isfinite(dt_fs))
    return fail(ION_EINVAL, "dt_fs must be finite and >= 0 (got %g)", dt_fs);
  ion_step_opts o = {1e-6, 1e-3, ION_WINDOW_FIXED, 2, ION_MAX_WINDOW, 1e-6};
  if (opts) o = *opts;
  if (o.window_policy != ION_WINDOW_FIXED && o.window_policy != ION_WINDOW_ADAPTIVE)
    return fail(ION_EINVAL, "unknown window_policy %d", o.window_policy);
  if (o.window_policy == ION_WINDOW_ADAPTIVE &&
      (o.w_min < 2 || o.w_min > o.w_max || o.w_max > ION_MAX_WINDOW ||
       !(o.eps_grow >= 0.0) || !std::isfinite(o.eps_grow)))
    return fail(ION_EINVAL,
                "adaptive windows need 2 <= w_min <= w_max <= %d and finite eps_grow >= 0",
                ION_MAX_WINDOW);
  if (!(o.eps_shift >= 0.0) || !std::isfinite(o.eps_shift))
    return fail(ION_EINVAL, "eps_shift must be finite and >= 0");
  if (!(o.degen_gap >= 0.0) || !(o.degen_gap < 1.0))
    return fail(ION_EINVAL, "degen_gap must lie in [0, 1)");
  pol->zero_dt = dt_fs == 0.0;
  pol->log2dt = dt_fs > 0.0 ? std::log2(dt_fs) : 0.0;
  pol->eps = o.eps_shift;
  pol->gap = o.degen_gap;
  pol->flags = flags;
  pol->adaptive = o.window_policy == ION_WINDOW_ADAPTIVE;
  pol->wmin = o.w_min;
  pol->wmax = o.w_max;
  pol->eps_grow = o.eps_grow;
  pol->eps_f = (float)o.eps_shift;
  pol->gap_f = (float)o.degen_gap;
  pol->eps_grow_f = (float)o.eps_grow;
  return ION_OK;
}

// Checks one job's arrays and fills its JobIO (Q: cells per lane of the
// FP32 launch, for the alignment of vector copies).
int make_job(const ion_species* sp, const void* E, void* N, int64_t ld, int64_t ncells,
             uint8_t* k_lo, uint8_t* k_hi, void* dne, const void* n_gas, bool f64, int Q,
             const char* who, ion::JobIO* J) {
  int rc = check_species(sp);
  if (rc) return rc;
  if (ncells < 0 || ncells >= (int64_t(1) << 31))
    return fail(ION_EINVAL, "%s: ncells=%lld outside [0, 2^31)", who, (long long)ncells);
  if (ncells > 0) {
    if (!E || !N || !k_lo || !k_hi || !dne)
      return fail(ION_EINVAL, "%s: E, N, k_lo, k_hi and dne must be non-NULL", who);
    if (ld < ncells) return fail(ION_EINVAL, "%s: ld=%lld < ncells", who, (long long)ld);
    if (ld > (int64_t(1) << 40)) return fail(ION_EINVAL, "%s: ld too large", who);
    const size_t el = f64 ? 8 : 4;
    if (!aligned(E, el) || !aligned(N, el) || !aligned(dne, el) ||
        (n_gas && !aligned(n_gas, el)))
      return fail(ION_EINVAL, "%s: E, N, dne and n_gas must be aligned to their element size",
                  who);
    if (!f64 && (!aligned(k_lo, 4) || !aligned(k_hi, 4)))
      return fail(ION_EINVAL, "%s: k_lo and k_hi must be 4-byte aligned", who);
  }
  J->tab = sp->dev;
  J->Z = sp->Z;
  J->E = E;
  J->N = N;
  J->ld = ld;
  J->ncells = (int)ncells;
  J->lo = k_lo;
  J->hi = k_hi;
  J->dne = dne;
  J->n_gas = n_gas;
  J->chunk0 = 0;
  const size_t vb = 4 * (size_t)Q;
  J->vec = aligned(E, vb) && aligned(N, vb) && aligned(dne, vb) && (ld % Q) == 0;
  return ION_OK;
}

int check_workspace(void* workspace, size_t have, size_t need) {
  if (!workspace) return fail(ION_EINVAL, "workspace is NULL");
  if (have < need) return fail(ION_EINVAL, "workspace has %zu bytes, %zu needed", have, need);
  if (!aligned(workspace, 256)) return fail(ION_EINVAL, "workspace must be 256-byte aligned");
  return ION_OK;
}

}  // namespace

int ion::species_info(const ion_species* sp, SpeciesInfo* out) {
  const int rc = check_species(sp);
  if (rc) return rc;
  out->device = sp->device;
  out->num_sms = sp->num_sms;
  out->Z = sp->Z;
  out->host = &sp->host;
  out->dev = sp->dev;
  return ION_OK;
}

int ion::policy_from_args(double dt_fs, const ion_step_opts* opts, int flags, Policy* pol) {
  return make_policy(dt_fs, opts, flags, pol);
}

int ion::job_from_args(const ion_species* sp, const void* E, void* N, int64_t ld,
                       int64_t ncells, uint8_t* k_lo, uint8_t* k_hi, void* dne,
                       const void* n_gas, bool f64, int Q, const char* who, JobIO* J) {
  return make_job(sp, E, N, ld, ncells, k_lo, k_hi, dne, n_gas, f64, Q, who, J);
}

int ion::workspace_ok(void* workspace, size_t have, size_t need) {
  return check_workspace(workspace, have, need);
}

namespace {

int run_batch(const ion_batch_job* jobs, int njobs, double dt_fs, const ion_step_opts* opts,
              int flags, const ion_launch_shape* shape, void* workspace, size_t ws_bytes,
              void* stream) {
  if (njobs < 1 || njobs > ion::kMaxJobs)
    return fail(ION_EINVAL, "njobs=%d outside [1, %d]", njobs, ion::kMaxJobs);
  if (!jobs) return fail(ION_EINVAL, "jobs is NULL");
  int rc = check_flags(flags);
  if (rc) return rc;
  ion::LaunchShape sh = ion::default_shape();
  if (shape) {
    sh = {shape->cells_per_lane, shape->warps_per_block, shape->blocks_per_sm};
    if (!ion::valid_shape(sh))
      return fail(ION_EINVAL,
                  "launch shape (%d cells/lane, %d warps/block, %d blocks/SM) is not built",
                  sh.cells_per_lane, sh.warps_per_block, sh.blocks_per_sm);
  }
  const bool f64 = (flags & ION_F64_PLAIN) != 0;
  ion::BatchArgs a;
  std::memset(&a, 0, sizeof a);
  a.njobs = njobs;
  if ((rc = make_policy(dt_fs, opts, flags, &a.pol))) return rc;
  int64_t total = 0;
  for (int j = 0; j < njobs; ++j) {
    const ion_batch_job& b = jobs[j];
    char who[32];
    snprintf(who, sizeof who, "job %d", j);
    if ((rc = make_job(b.species, b.E, b.N, b.ld, b.ncells, b.k_lo, b.k_hi, b.dne, b.n_gas,
                       f64, sh.cells_per_lane, who, &a.job[j])))
      return rc;
    if (b.species->device != jobs[0].species->device)
      return fail(ION_EINVAL, "job %d: its species lives on another device", j);
    total += b.ncells;
  }
  if (total >= (int64_t(1) << 31))
    return fail(ION_EINVAL, "%lld cells in one call; the limit is 2^31 - 1", (long long)total);
  if ((rc = check_workspace(workspace, ws_bytes, ion::step_workspace_bytes(total, f64))))
    return rc;
  ion::bind_workspace(a.ws, workspace, total);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e;
  if (f64) {
    e = cudaMemsetAsync(a.ws.hdr, 0, ion::kHdrWords * sizeof(uint32_t), s);
    for (int j = 0; j < njobs && e == cudaSuccess; ++j)
      e = ion::launch_step_f64(a.job[j], a.pol, a.ws.hdr, s);
  } else {
    e = ion::launch_batch_f32(a, sh, jobs[0].species->num_sms, s);
  }
  return e == cudaSuccess ? ok() : cuda_fail(e, "ion_step launch");
}

}  // namespace

extern "C" {

size_t ion_step_batched_workspace_bytes(const ion_batch_job* jobs, int njobs, int flags) {
  int64_t total = 0;
  for (int j = 0; jobs && j < njobs; ++j) total += jobs[j].ncells > 0 ? jobs[j].ncells : 0;
  return ion::step_workspace_bytes(total, (flags & ION_F64_PLAIN) != 0);
}

int ion_step(const ion_species* sp, const void* E, void* N, int64_t ld, int64_t ncells,
             double dt_fs, uint8_t* k_lo, uint8_t* k_hi, void* dne, const void* n_gas,
             const ion_step_opts* opts, int flags, void* workspace, size_t workspace_bytes,
             void* stream) {
  int rc = check_species(sp);
  if (rc) return rc;
  const ion_batch_job job = {sp, E, N, ld, ncells, k_lo, k_hi, dne, n_gas};
  return run_batch(&job, 1, dt_fs, opts, flags, nullptr, workspace, workspace_bytes, stream);
}

int ion_step_field(const ion_species* sp, const void* Ex, const void* Ey, const void* Ez,
                   void* N, int64_t ld, int64_t ncells, double dt_fs, uint8_t* k_lo,
                   uint8_t* k_hi, void* dne, const void* n_gas, const ion_step_opts* opts,
                   int flags, void* workspace, size_t workspace_bytes, void* stream) {
  int rc = check_species(sp);
  if (rc) return rc;
  if (!Ey && !Ez)
    return ion_step(sp, Ex, N, ld, ncells, dt_fs, k_lo, k_hi, dne, n_gas, opts, flags,
                    workspace, workspace_bytes, stream);
  if (ncells < 0 || ncells >= (int64_t(1) << 31))
    return fail(ION_EINVAL, "ncells=%lld outside [0, 2^31)", (long long)ncells);
  const size_t need = ion_step_field_workspace_bytes(ncells, flags);
  if (!workspace || workspace_bytes < need)
    return fail(ION_EINVAL, "workspace: %zu bytes given, %zu needed", workspace_bytes, need);
  if (reinterpret_cast<uintptr_t>(workspace) & 255u)
    return fail(ION_EINVAL, "workspace must be 256-byte aligned");
  const size_t step = (ion_step_workspace_bytes(ncells, flags) + 255) / 256 * 256;
  void* Emag = static_cast<char*>(workspace) + step;
  rc = ion_field_magnitude(Ex, Ey, Ez, ncells,
                           (flags & ION_F64_PLAIN) ? ION_DTYPE_F64 : ION_DTYPE_F32, Emag, stream);
  if (rc) return rc;
  return ion_step(sp, Emag, N, ld, ncells, dt_fs, k_lo, k_hi, dne, n_gas, opts, flags,
                  workspace, step, stream);
}

int ion_step_batched(const ion_batch_job* jobs, int njobs, double dt_fs,
                     const ion_step_opts* opts, int flags, const ion_launch_shape* shape,
                     void* workspace, size_t workspace_bytes, void* stream) {
  return run_batch(jobs, njobs, dt_fs, opts, flags, shape, workspace, workspace_bytes, stream);
}

int ion_autotune(const ion_batch_job* jobs, int njobs, double dt_fs, const ion_step_opts* opts,
                 int flags, void* workspace, size_t workspace_bytes, int reps, void* stream,
                 ion_launch_shape* best, float* best_ms) {
  if (!best) return fail(ION_EINVAL, "best is NULL");
  if (flags & ION_F64_PLAIN) return fail(ION_EINVAL, "ion_autotune tunes the FP32 form only");
  if (reps < 1 || reps > 64) return fail(ION_EINVAL, "reps=%d outside [1, 64]", reps);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e != cudaSuccess) return cuda_fail(e, "ion_autotune events");
  float best_t = -1.0f;
  ion_launch_shape bs = {0, 0, 0};
  const int Qs[] = {1, 2, 4}, Ws[] = {2, 4, 8}, Bs[] = {0, 1, 2, 3, 4};
  int rc = ION_OK;
  for (int Q : Qs) {
    for (int W : Ws) {
      for (int B : Bs) {
        const ion_launch_shape sh = {Q, W, B};
        // one untimed launch, then the median of `reps` timed ones
        rc = run_batch(jobs, njobs, dt_fs, opts, flags, &sh, workspace, workspace_bytes, stream);
        if (rc) break;
        float ts[64];
        for (int r = 0; r < reps && rc == ION_OK; ++r) {
          cudaEventRecord(e0, s);
          rc = run_batch(jobs, njobs, dt_fs, opts, flags, &sh, workspace, workspace_bytes,
                         stream);
          cudaEventRecord(e1, s);
          if (rc) break;
          if ((e = cudaEventSynchronize(e1)) != cudaSuccess) {
            rc = cuda_fail(e, "ion_autotune");
            break;
          }
          cudaEventElapsedTime(&ts[r], e0, e1);
        }
        if (rc) break;
        for (int i = 1; i < reps; ++i)  // insertion sort; reps is small
          for (int k = i; k > 0 && ts[k] < ts[k - 1]; --k) {
            const float t = ts[k];
            ts[k] = ts[k - 1];
            ts[k - 1] = t;
          }
        const float med = ts[reps / 2];
        if (best_t < 0.0f || med < best_t) {
          best_t = med;
          bs = sh;
        }
      }
      if (rc) break;
    }
    if (rc) break;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) return rc;
  *best = bs;
  if (best_ms) *best_ms = best_t;
  return ok();
}

}  // extern "C"
