// ion_step.cuh -- launch arguments shared by the step kernels and the host
// launchers.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "ion_device.cuh"

namespace ion {

// Workspace header (uint32 words at the start of the workspace).
constexpr int kHdrFallback = 0;  // cells whose coefficients were done in FP64
constexpr int kHdrInvalid = 1;   // cells skipped because their window is invalid
constexpr int kHdrStiff = 2;     // stiff-cell records (written by the stiff kernel: 6 + 7)
constexpr int kHdrSurrogate = 3; // surrogate step: cells whose rates came from the network
constexpr int kHdrPlain = 4;     // surrogate step: cells that took the rates of Eq. 1
constexpr int kHdrTimeout = 5;   // surrogate step: non-zero if a bounded wait gave up
constexpr int kHdrRecNarrow = 6; // records of windows of <= kRecNarrow states (from the front)
constexpr int kHdrRecWide = 7;   // records of wider windows (from the back of the arrays)
constexpr int kHdrChunk = 8;     // streaming kernels: next chunk or group to hand out
constexpr int kHdrHot = 9;       // (reserved)
constexpr int kHdrCons = 10;     // ION_CONSERVATION_CHECK: largest |change of sum_k N_k|
constexpr int kHdrWords = 11;
// Records of at most this many window states take the short divided-difference
// table (3 rates, 7 subsets); wider ones the long one (5 rates, 31 subsets).
constexpr int kRecNarrow = 4;
constexpr size_t kHdrBytes = 256;
static_assert(kHdrWords * 4 <= (int)kHdrBytes, "the header words fit the header");

// Largest number of species one batched launch advances.
constexpr int kMaxJobs = 8;

// Where one job's cells live.
struct JobIO {
  const SpeciesTable* tab;
  int Z;
  const void* E;
  void* N;
  int64_t ld;
  int ncells;
  uint8_t* lo;
  uint8_t* hi;
  void* dne;
  const void* n_gas;
  int chunk0;  // first chunk of this job in the launch's chunk numbering
  int vec;     // E, N, dne aligned for vector copies of a lane's cells
};

// Per-call policy shared by all jobs.
struct Policy {
  double log2dt;
  int zero_dt;
  double eps;
  double gap;
  int flags;
  int adaptive;     // ION_WINDOW_ADAPTIVE
  int wmin, wmax;   // adaptive widths
  double eps_grow;  // adaptive: the top grows above this population
  float eps_f, gap_f, eps_grow_f;  // the same in FP32 (no per-cell conversion)
};

// eps, gap, eps_grow of the policy in the precision of the caller.
template <typename T>
__device__ __forceinline__ T pol_eps(const Policy& p);
template <>
__device__ __forceinline__ float pol_eps<float>(const Policy& p) { return p.eps_f; }
template <>
__device__ __forceinline__ double pol_eps<double>(const Policy& p) { return p.eps; }
template <typename T>
__device__ __forceinline__ T pol_gap(const Policy& p);
template <>
__device__ __forceinline__ float pol_gap<float>(const Policy& p) { return p.gap_f; }
template <>
__device__ __forceinline__ double pol_gap<double>(const Policy& p) { return p.gap; }
template <typename T>
__device__ __forceinline__ T pol_grow(const Policy& p);
template <>
__device__ __forceinline__ float pol_grow<float>(const Policy& p) { return p.eps_grow_f; }
template <>
__device__ __forceinline__ double pol_grow<double>(const Policy& p) { return p.eps_grow; }

// Workspace views.
struct Scratch {
  uint32_t* hdr;      // kHdr* words
  uint32_t* queue;    // FP64-coefficient cells
  uint8_t* queue_job;
  // stiff-cell records: cell, job, |E|, lo | hi << 8, window planes
  // rec_V[r * rec_cap + i]
  uint32_t* rec_c;
  uint8_t* rec_job;
  float* rec_E;
  uint16_t* rec_lohi;
  float* rec_V;
  int64_t rec_cap;
};

struct BatchArgs {
  int njobs;
  int nchunks;  // full chunks over all jobs (queue form: groups)
  JobIO job[kMaxJobs];
  Policy pol;
  Scratch ws;
};

// Launch shape of the FP32 streaming kernel (chosen by default or by
// ion_autotune).
struct LaunchShape {
  int cells_per_lane;   // 1, 2 or 4
  int warps_per_block;  // 2, 4 or 8
  int blocks_per_sm;    // 0: as many as fit
};

// Workspace layout of the FP32 form (bound by bind_workspace, step_f32.cu):
// the header, the FP64-coefficient queue (cell, job) and the stiff-cell
// records (cell, job, |E|, lo | hi << 8, ION_MAX_WINDOW planes), each
// section 256-byte aligned.  The FP64 form uses the header alone.
constexpr size_t round256(size_t x) { return (x + 255) / 256 * 256; }
constexpr size_t f32_workspace_bytes(size_t n) {
  return kHdrBytes + round256(4 * n) + round256(n) + round256(4 * n) + round256(n) +
         round256(4 * n) + round256(2 * n) + round256(4 * n * ION_MAX_WINDOW);
}
size_t step_workspace_bytes(int64_t ncells, bool f64);
void bind_workspace(Scratch& s, void* ws, int64_t ncells);

// Sets the calling thread's ion_last_error() message and returns `code`
// (api.cu).
int set_error(int code, const char* fmt, ...);

// Argument checking shared by the entry points (api.cu); each returns ION_OK
// or sets the thread's error message and returns the ION_E* code.
struct SpeciesInfo {
  int device, num_sms, Z;
  const SpeciesTable* host;  // host copy
  const SpeciesTable* dev;   // device copy
};
int species_info(const ion_species* sp, SpeciesInfo* out);
int policy_from_args(double dt_fs, const ion_step_opts* opts, int flags, Policy* pol);
int job_from_args(const ion_species* sp, const void* E, void* N, int64_t ld, int64_t ncells,
                  uint8_t* k_lo, uint8_t* k_hi, void* dne, const void* n_gas, bool f64, int Q,
                  const char* who, JobIO* J);
int workspace_ok(void* workspace, size_t have, size_t need);

// Launchers.  They only enqueue; the caller has validated.  `a.job[j].chunk0`
// and `a.nchunks` are filled in by launch_batch_f32.
cudaError_t launch_batch_f32(BatchArgs& a, const LaunchShape& shape, int num_sms,
                             cudaStream_t s);
// The stiff-cell records and the FP64-coefficient queue left by a previous
// kernel of the same call (step_f32.cu).
cudaError_t launch_stiff_f32(const BatchArgs& a, int num_sms, cudaStream_t s);
cudaError_t launch_fb_f32(const BatchArgs& a, int num_sms, cudaStream_t s);
cudaError_t launch_step_f64(const JobIO& job, const Policy& pol, uint32_t* hdr,
                            cudaStream_t s);
LaunchShape default_shape();
bool valid_shape(const LaunchShape& s);

}  // namespace ion
