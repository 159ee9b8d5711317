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
constexpr int kHdrStiff = 2;     // stiff-cell records written by the streaming kernel
constexpr int kHdrWords = 3;
constexpr size_t kHdrBytes = 256;

struct StepArgs {
  const SpeciesTable* tab;
  int Z;
  const void* E;
  void* N;
  int64_t ld;
  int ncells;
  double log2dt;
  int zero_dt;
  uint8_t* lo;
  uint8_t* hi;
  void* dne;
  const void* n_gas;
  double eps;
  double gap;
  int flags;
  int vec;          // E, N 16-byte aligned and ld % 4 == 0: 16-byte copies
  uint32_t* hdr;    // workspace header (kHdr* words)
  uint32_t* queue;  // cells for the FP64-coefficient kernel
  // stiff-cell records (FP32 form): cell, |E|, lo | hi << 8, window planes
  // rec_V[r * rec_cap + i]
  uint32_t* rec_c;
  float* rec_E;
  uint16_t* rec_lohi;
  float* rec_V;
  int64_t rec_cap;
};

// Workspace layout (step.cu).
size_t step_workspace_bytes(int64_t ncells, bool f64);
void bind_workspace(StepArgs& a, void* ws);

// Sets the calling thread's ion_last_error() message and returns `code`
// (api.cu).
int set_error(int code, const char* fmt, ...);

// Launchers (step.cu).  They only enqueue; the caller has validated.
cudaError_t launch_step_f32(const StepArgs& a, int num_sms, cudaStream_t s);
cudaError_t launch_step_f64(const StepArgs& a, cudaStream_t s);

}  // namespace ion
