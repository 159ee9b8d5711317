// noalloc.cu -- ion_step_noalloc: ion_step with its scratch in a fixed-size
// __device__ array of this library instead of a caller-provided workspace,
// for callers that cannot allocate device memory (see ionize.h).
#include <mutex>

#include "ion_step.cuh"
#include "ionize.h"

namespace {

constexpr int64_t kMaxCells = ION_STEP_NOALLOC_MAX_CELLS;
constexpr size_t kScratchBytes = ION_STEP_NOALLOC_SCRATCH_BYTES;
constexpr int kMaxDevices = 64;
static_assert(ion::f32_workspace_bytes(kMaxCells) == kScratchBytes,
              "ION_STEP_NOALLOC_SCRATCH_BYTES must equal the FP32 workspace of "
              "ION_STEP_NOALLOC_MAX_CELLS cells");

// One array per device that loads the library; its size covers
// ion_step_workspace_bytes(kMaxCells, ION_F32).
__device__ __align__(256) unsigned char g_scratch[kScratchBytes];

std::mutex g_mu;
void* g_addr[kMaxDevices] = {};  // device address of g_scratch, per device

}  // namespace

extern "C" int ion_step_noalloc(const ion_species* sp, const void* E, void* N,
                                int64_t ld, int64_t ncells, double dt_fs,
                                uint8_t* k_lo, uint8_t* k_hi, void* dne,
                                const void* n_gas, const ion_step_opts* opts,
                                int flags, void* stream) {
  if (ncells < 0 || ncells > kMaxCells)
    return ion::set_error(ION_EINVAL,
                          "ion_step_noalloc: ncells=%lld outside [0, %lld]; split the call",
                          (long long)ncells, (long long)kMaxCells);
  const size_t need = ion_step_workspace_bytes(ncells, flags);
  if (need > kScratchBytes)
    return ion::set_error(ION_EINVAL, "ion_step_noalloc: %zu scratch bytes needed, %zu held",
                          need, kScratchBytes);
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return ion::set_error(ION_ECUDA, "ion_step_noalloc: no usable current device (%s)",
                          cudaGetErrorString(e));
  void* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_scratch);
      if (e != cudaSuccess || !p)
        return ion::set_error(ION_ECUDA, "ion_step_noalloc: cudaGetSymbolAddress: %s",
                              cudaGetErrorString(e));
      g_addr[dev] = p;
    }
    scratch = g_addr[dev];
  }
  return ion_step(sp, E, N, ld, ncells, dt_fs, k_lo, k_hi, dne, n_gas, opts, flags,
                  scratch, kScratchBytes, stream);
}
