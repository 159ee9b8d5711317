/*
 * ionize.h -- C ABI of the GB300 (sm_103a) multi-level tunnelling-ionization
 * library: ADK rates and the analytic, locally reduced population update of
 * Cheng & Samulyak, "Efficient numerical algorithm for multi-level ionization
 * of high-atomic-number gases" (arXiv 2202.10647).
 *
 * Conventions shared by every entry point
 *   - Pointers named as device arrays are caller-owned CUDA device memory of
 *     the device that was current when the species was created.  The library
 *     owns only the species table it allocates in ion_species_init.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Compute entry points only enqueue work on it: they allocate
 *     nothing, never synchronize, and copy nothing between host and device,
 *     except where a comment says otherwise.
 *   - Return value: ION_OK (0) or a negative ION_E* code; ion_last_error()
 *     then holds a message for the calling thread.  Arguments are checked
 *     before anything is enqueued; a rejected call leaves every buffer as it
 *     was.
 *   - Populations are SoA: plane k (charge state k+, k = 0..Z) of a cell c is
 *     N[k*ld + c].  States are numbered by charge; the rate W_k moves
 *     population from state k to k+1 (Eq. 2), so a species with atomic number
 *     Z has Z rates and Z+1 planes.
 *   - Units: |E| in GV/m, dt in fs, rates in 1/fs, potentials in eV.
 */
#ifndef IONIZE_H
#define IONIZE_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define ION_API __attribute__((visibility("default")))
#else
#define ION_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* ---- return codes ------------------------------------------------------- */
#define ION_OK 0
#define ION_EINVAL (-1)   /* bad argument (null, range, alignment, size)     */
#define ION_ECUDA (-2)    /* a CUDA call or kernel launch failed              */
#define ION_ENOMEM (-3)   /* allocation failed (creation and validation calls) */
#define ION_ETIMEOUT (-4) /* a bounded device-side wait gave up               */

/* ---- flags of ion_step --------------------------------------------------- */
#define ION_F32 0x0              /* FP32 data and arithmetic; the Bateman     */
                                 /* coefficients of cells with a nearly       */
                                 /* degenerate rate pair are computed in FP64 */
#define ION_F64_PLAIN 0x1        /* FP64 data (E, N, dne, n_gas are double)  */
                                 /* and FP64 arithmetic everywhere            */
#define ION_NO_WINDOW_UPDATE 0x2 /* keep k_lo/k_hi as given                  */
#define ION_NO_FP64_FALLBACK 0x4 /* ION_F32 only: FP32 coefficients for all   */
#define ION_FORCE_FP64_COEF 0x8  /* ION_F32 only: FP64 coefficients for every */
                                 /* cell that takes the Bateman form          */
#define ION_CONSERVATION_CHECK 0x10 /* measure each cell's change of its total */
                                 /* population, sum_k N'_k - sum_k N_k (in    */
                                 /* twice the working precision), and leave   */
                                 /* the largest |change| in word 10 of the    */
                                 /* workspace header (float bits)             */

/* ---- dtype codes of ion_rates --------------------------------------------- */
#define ION_DTYPE_F32 0
#define ION_DTYPE_F64 1

/* Largest atomic number and window width the kernels accept. */
#define ION_MAX_Z 63
#define ION_MAX_WINDOW 6

typedef struct ion_species ion_species; /* opaque, owned by the library */

/* Rate models of ion_constants.rate_model. */
#define ION_ADK_CYCLE_AVERAGED 0 /* Eq. 1 as printed */
#define ION_ADK_STATIC 1         /* Eq. 1 without its cycle-averaging factor */
                                 /* sqrt(3 n*^3 |E| / (pi Q^3 E_a)): the rate */
                                 /* in a static field of magnitude |E|, for   */
                                 /* fields given as instantaneous values      */

/* Constants of Eq. 1 and the rate model.  NULL selects the printed values
 * omega_a = 4.13e16 1/s and E_a = 510 GV/m (Sec. 2, text after Eq. 1) with
 * U_H = 13.6 eV (U_H is named there but not given a value) and
 * ION_ADK_CYCLE_AVERAGED.  CODATA values (omega_a = 4.1341374e16 1/s,
 * E_a = 514.22067 GV/m, U_H = 13.605693 eV) are one choice of the others. */
typedef struct {
  double omega_a_per_s;
  double E_a_GVm;
  double U_H_eV;
  int rate_model; /* ION_ADK_CYCLE_AVERAGED or ION_ADK_STATIC */
} ion_constants;

/* Window policies of ion_step_opts.window_policy. */
#define ION_WINDOW_FIXED 0    /* the paper's rule: slide, width kept        */
#define ION_WINDOW_ADAPTIVE 1 /* width adapts between w_min and w_max       */

/* Per-call policy of ion_step.  NULL selects the defaults. */
typedef struct {
  /* The window [lo,hi] slides up by one state while the population of its
   * lowest state after the step is below eps_shift (the "prescribed
   * threshold" of Sec. 3, whose value the paper does not give); default 1e-6.
   * The window keeps its width, slides at most w-1 states per step and
   * never past hi = Z. */
  double eps_shift;
  /* ION_F32: a cell whose window holds two rates with
   * |W_i - W_j| < degen_gap * max(W_i, W_j) gets its Bateman coefficients in
   * FP64; default 1e-3.  0 disables the test. */
  double degen_gap;
  /* ION_WINDOW_FIXED (default): the window slides as above.
   * ION_WINDOW_ADAPTIVE: while the lowest state holds less than eps_shift
   * (at most w-1 moves) it is dropped if the width exceeds w_min, else the
   * window slides; then, if the old top state holds more than eps_grow, the
   * state above joins (width at most w_max, never past Z).  Requires
   * 2 <= w_min <= w_max <= ION_MAX_WINDOW and eps_grow >= 0; the paper has
   * only the fixed rule (Sec. 3), this one trades window traffic for the
   * lag of a fixed window behind fast ionization. */
  int window_policy;
  int w_min;
  int w_max;
  double eps_grow;
} ion_step_opts;

/* ion_species_init -- build the per-state ADK table of one gas (Eq. 1).
 *   U_ion_eV[k], l[k], m[k], k = 0..Z-1: ionization potential, orbital
 *     quantum number and projection of the electron removed by W_k (host
 *     arrays, read during the call only).  Q = k+1 is the charge after
 *     ionization.  Requires 1 <= Z <= ION_MAX_Z, U > 0, 0 <= |m| <= l <= 20.
 *   c: constants of Eq. 1 or NULL for the paper's values.
 *   out: receives the handle.  The table (a few KB) is copied to the current
 *     device synchronously; this is the only entry point that allocates.
 * Errors: ION_EINVAL, ION_ENOMEM, ION_ECUDA. */
ION_API int ion_species_init(const double* U_ion_eV, const int* l, const int* m, int Z,
                     const ion_constants* c, ion_species** out);

/* Frees the table.  NULL is accepted.  Must not race with work that uses it. */
ION_API int ion_species_destroy(ion_species* sp);

/* Atomic number Z of a species (or ION_EINVAL). */
ION_API int ion_species_z(const ion_species* sp);

/* ion_rates -- ADK rates W_k(|E_c|) of Eq. 1 in 1/fs for k in [k_lo, k_hi).
 *   E: device array [ncells] of float (ION_DTYPE_F32) or double
 *     (ION_DTYPE_F64); the magnitude |E| is used.
 *   W_out: device array, W_k of cell c at W_out[(k-k_lo)*ldw + c], same
 *     dtype as E; ldw >= ncells.
 *   Requires 0 <= k_lo <= k_hi <= Z and 0 <= ncells < 2^31.
 * W = 0 where |E| <= 1e-6 GV/m or where the tunnelling exponent
 * (2/3)(Q/n*)^3 E_a/|E| exceeds 700. */
ION_API int ion_rates(const ion_species* sp, const void* E, int64_t ncells, int k_lo,
              int k_hi, void* W_out, int64_t ldw, int dtype, void* stream);

/* Bytes of device workspace ion_step needs for `ncells` cells with `flags`:
 * a 256-byte header plus, for ION_F32, 40 bytes per cell: a 5-byte queue
 * slot (cells whose Bateman coefficients are computed in FP64) and a 35-byte
 * record (cells with a rate W dt > 1, or > 1.5 under a launch shape of one
 * cell per lane, finished by the record kernel from the inputs already
 * loaded). */
ION_API size_t ion_step_workspace_bytes(int64_t ncells, int flags);

/* ion_step -- advance the charge-state populations of every cell by one
 * step dt with the analytic solution of the window's rate equations.
 *
 * For each cell c with window [lo, hi] = [k_lo[c], k_hi[c]] (w = hi-lo+1
 * states, 1 <= w <= ION_MAX_WINDOW, hi <= Z):
 *   1. W_k = W_k(|E_c|) for k = lo..hi-1 by Eq. 1, frozen over the step
 *      (Sec. 3, text after Eq. 3).
 *   2. N[lo..hi] <- exp(dt A) N[lo..hi], A the [lo,hi] block of the
 *      bidiagonal matrix of Eq. 3 with the top state absorbing (as in the
 *      4-level system of Eqs. 6-9).  This is the sum-of-exponentials solution
 *      of Eqs. 4-5 ("the Bateman form"), evaluated in Newton
 *      (divided-difference) form so that equal and nearly equal rates need
 *      no special input; a cell whose rates all have W dt <= 1 (FP32) or
 *      <= 1/2 (FP64) takes the Taylor series of exp(dt A) instead, which
 *      reaches the same result with fewer operations.  States outside the
 *      window are not read or written.
 *   3. dne[c] = sum_k k (N'_k - N_k), the free electrons released per atom,
 *      times n_gas[c] when n_gas is not NULL (overwritten, not accumulated).
 *   4. Unless ION_NO_WINDOW_UPDATE: the window slides up (see
 *      ion_step_opts.eps_shift; Sec. 3, text after Fig. 2 and after Eq. 9).
 *
 * Arguments
 *   E      device [ncells], float (ION_F32) or double (ION_F64_PLAIN).
 *   N      device SoA [(Z+1) * ld], same dtype; updated in place.
 *   ld     plane stride in elements, ld >= ncells.
 *   ncells 0 <= ncells < 2^31 (0 is a no-op).
 *   dt_fs  0 <= dt < inf (0 leaves populations unchanged).
 *   k_lo, k_hi  device uint8 [ncells], in/out.
 *   dne    device [ncells], out, same dtype as E.
 *   n_gas  device [ncells] or NULL, same dtype as E.
 *   workspace  device, >= ion_step_workspace_bytes(ncells, flags) bytes,
 *          256-byte aligned; its contents need no initialization.  After
 *          the step the header holds uint32 counters: word 0 the cells
 *          whose coefficients were computed in FP64, word 1 the cells left
 *          untouched because their window was invalid (lo > hi, hi > Z or
 *          w > ION_MAX_WINDOW), word 2 the cells that had a rate with
 *          W dt > 1 (> 1.5 with one cell per lane; finished by the
 *          record kernel in the Bateman form),
 *          and with ION_CONSERVATION_CHECK word 10 the bits of a float, the largest
 *          |sum_k N'_k - sum_k N_k| over the cells (the states outside a
 *          window are not touched, so this is the step's whole conservation
 *          error; 0 for cells that do not change, NaN if a sum is NaN).
 * Alignment: E, N, dne, n_gas aligned to their element size; with ION_F32
 * k_lo and k_hi 4-byte aligned (they are copied four cells at a time).
 * Calls that share a workspace must not overlap on the device.
 * Errors: ION_EINVAL (checked before any launch), ION_ECUDA. */
ION_API int ion_step(const ion_species* sp, const void* E, void* N, int64_t ld,
             int64_t ncells, double dt_fs, uint8_t* k_lo, uint8_t* k_hi,
             void* dne, const void* n_gas, const ion_step_opts* opts, int flags,
             void* workspace, size_t workspace_bytes, void* stream);

/* ion_field_magnitude -- |E_c| = sqrt(Ex_c^2 + Ey_c^2 + Ez_c^2), the local
 * field magnitude E_L that Eq. 1 takes (Sec. 2), from the components a
 * field solver keeps.  Any of Ey, Ez may be
 * NULL (absent); with Ex alone the result is |Ex|.  Arithmetic in the
 * dtype (ION_DTYPE_F32: fused multiply-adds and a correctly rounded sqrt;
 * ION_DTYPE_F64 likewise).
 *   Ex, Ey, Ez, E_abs  device [ncells] of the dtype, aligned to it.
 * 0 <= ncells < 2^31.  Errors: ION_EINVAL, ION_ECUDA. */
ION_API int ion_field_magnitude(const void* Ex, const void* Ey, const void* Ez, int64_t ncells,
                                int dtype, void* E_abs, void* stream);

/* Workspace bytes of ion_step_field: ion_step's, rounded up to 256, and room
 * for the magnitudes. */
ION_API size_t ion_step_field_workspace_bytes(int64_t ncells, int flags);

/* ion_step_field -- ion_step with the field given by its components (Ey, Ez
 * may be NULL): ion_field_magnitude into the workspace, then ion_step on the
 * magnitudes (with Ex alone, ion_step on Ex directly: Eq. 1 takes |E|).
 * Arguments and errors as ion_step; the components have E's dtype and
 * alignment; workspace >= ion_step_field_workspace_bytes(ncells, flags). */
ION_API int ion_step_field(const ion_species* sp, const void* Ex, const void* Ey,
                           const void* Ez, void* N, int64_t ld, int64_t ncells, double dt_fs,
                           uint8_t* k_lo, uint8_t* k_hi, void* dne, const void* n_gas,
                           const ion_step_opts* opts, int flags, void* workspace,
                           size_t workspace_bytes, void* stream);

/* One species' cells for ion_step_batched: the arguments of ion_step that
 * belong to a species.  The jobs of one call must not share cells. */
typedef struct {
  const ion_species* species;
  const void* E;
  void* N;
  int64_t ld;
  int64_t ncells;
  uint8_t* k_lo;
  uint8_t* k_hi;
  void* dne;
  const void* n_gas;
} ion_batch_job;

/* Launch shape of the FP32 streaming kernels: cells per lane (1, 2 or 4),
 * warps per block (2, 4 or 8), resident blocks per SM (0: as many as fit).
 * NULL selects {2, 8, 0}, which ion_step uses too. */
typedef struct {
  int cells_per_lane;
  int warps_per_block;
  int blocks_per_sm;
} ion_launch_shape;

/* Maximum number of jobs of one ion_step_batched call. */
#define ION_MAX_JOBS 8

/* Workspace bytes of ion_step_batched: ion_step_workspace_bytes of the total
 * cell count of the jobs. */
ION_API size_t ion_step_batched_workspace_bytes(const ion_batch_job* jobs, int njobs,
                                                int flags);

/* ion_step_batched -- ion_step for up to ION_MAX_JOBS species (different Z,
 * cell counts and arrays) in one launch: with ION_F32 one persistent kernel
 * walks the cells of every job (each warp picks its job per chunk of cells)
 * and the follow-up kernels serve all jobs; with ION_F64_PLAIN one
 * persistent kernel per job is launched.  Each job obeys the rules of ion_step's arguments; dt,
 * opts and flags apply to all.  `shape` chooses the launch shape (NULL: the
 * default; ion_autotune finds the fastest).  The total cell count must stay
 * below 2^31.  Errors as ion_step. */
ION_API int ion_step_batched(const ion_batch_job* jobs, int njobs, double dt_fs,
                             const ion_step_opts* opts, int flags,
                             const ion_launch_shape* shape, void* workspace,
                             size_t workspace_bytes, void* stream);

/* ion_autotune -- times ion_step_batched (ION_F32) on the given jobs for every
 * built launch shape (cells per lane x warps per block x blocks per SM) and
 * returns the shape with the smallest median time over `reps` (1..64) timed
 * steps, and that time in ms (best_ms may be NULL).  It runs real steps on
 * the jobs' arrays, so pass copies of the state.  The steps run one after
 * another on the same arrays, so where windows slide each shape is timed on
 * a later state than the one before it: time the chosen shape (and the
 * default) again from the state that matters.  It creates CUDA events and
 * synchronizes on them: call it outside any stream capture.  Errors: those
 * of ion_step_batched, ION_EINVAL for ION_F64_PLAIN or a bad reps. */
ION_API int ion_autotune(const ion_batch_job* jobs, int njobs, double dt_fs,
                         const ion_step_opts* opts, int flags, void* workspace,
                         size_t workspace_bytes, int reps, void* stream,
                         ion_launch_shape* best, float* best_ms);

/* ion_step_noalloc -- ion_step for callers that cannot allocate device
 * memory.  Some callers cannot make a device allocation at the point where
 * they step the populations: code that runs while a CUDA graph is being
 * captured by someone else, plugins whose host forbids device allocations
 * of its guests, or codes that fix their memory footprint at start-up.  This
 * entry point takes the same arguments as ion_step minus the workspace, and
 * uses instead a scratch array that is a file-scope __device__ variable of
 * this library: ION_STEP_NOALLOC_SCRATCH_BYTES (10,486,016 bytes, about 10.5 MB
 * or 10 MiB) on every GPU that loads the library, held until the process
 * exits.  The paper has no
 * counterpart of this call.
 *   - ncells <= ION_STEP_NOALLOC_MAX_CELLS (262144); larger calls return
 *     ION_EINVAL (split the cells into ranges: offset E, N, k_lo, k_hi, dne
 *     and n_gas by the first cell of the range and keep ld).
 *   - It allocates nothing and frees nothing.  The first call on a device
 *     looks up the device address of the array (cudaGetSymbolAddress) with
 *     that device current; make that first call before any stream capture.
 *     The address is kept for the life of the process: do not use this call
 *     on a device after cudaDeviceReset (the array's module is reloaded and
 *     the kept address may no longer be valid).
 *   - Every call on a device shares the one array, which keeps the contents
 *     the last call left; the counters a step needs zeroed are reset by the
 *     step itself.  Calls that overlap on the device (other streams, other
 *     host threads) race on the array: serialize them.
 *   - After the call the array holds the workspace header described for
 *     ion_step; it is not readable through this interface.
 * Errors: those of ion_step, plus ION_EINVAL for ncells beyond the maximum
 * and ION_ECUDA if the array's address cannot be obtained. */
#define ION_STEP_NOALLOC_MAX_CELLS 262144
#define ION_STEP_NOALLOC_SCRATCH_BYTES 10486016
ION_API int ion_step_noalloc(const ion_species* sp, const void* E, void* N,
                             int64_t ld, int64_t ncells, double dt_fs,
                             uint8_t* k_lo, uint8_t* k_hi, void* dne,
                             const void* n_gas, const ion_step_opts* opts,
                             int flags, void* stream);

/* ion_conservation -- the conservation diagnostic of multi-step runs.  The
 * update of Eqs. 4-9 moves population between the states of a window and
 * leaves the other states alone, so sum_k N_k of a cell never changes; this
 * call measures how well a run keeps it.
 *   N        device SoA, plane k of cell c at N[k*ld + c], float
 *            (ION_DTYPE_F32) or double (ION_DTYPE_F64).
 *   ld, ncells  as in ion_step; 0 <= ncells <= ld (0 is a no-op).
 *   nplanes  planes summed per cell, 1..ION_MAX_Z+1 (Z+1 for a species).
 *   target   the expected sum (1 for normalized populations).
 *   out_max  device float, 4-byte aligned: receives
 *            max_c |sum_{k<nplanes} N[k*ld+c] - target| (0 when ncells is
 *            0), the sums taken in double; a NaN sum gives NaN.
 * Enqueues a 4-byte memset of *out_max and one kernel that reads
 * nplanes*ncells elements (graph-capturable).
 * Errors: ION_EINVAL, ION_ECUDA. */
ION_API int ion_conservation(const void* N, int64_t ld, int64_t ncells, int nplanes,
                             double target, int dtype, float* out_max, void* stream);

/* ion_copy_cells -- the cells [offset, offset + ncells) of `nplanes` plane
 * rows of one SoA array (rows ld_src elements apart) into another (rows
 * ld_dst apart), in one strided copy (cudaMemcpy2DAsync, direction from the
 * pointers); a PIC code moving a range of cells between host and device
 * (or between two device arrays) issues one call per array instead of one
 * per plane.  The paper has no counterpart.
 *   dst, src  device or host (pinned host memory for the copy to run
 *             asynchronously) arrays of elem_bytes-sized elements.
 *   elem_bytes 1, 2, 4 or 8; nplanes >= 1; ncells, offset >= 0;
 *   offset + ncells <= min(ld_dst, ld_src).
 * Enqueues on `stream`; allocates nothing.  Errors: ION_EINVAL, ION_ECUDA. */
ION_API int ion_copy_cells(void* dst, int64_t ld_dst, const void* src, int64_t ld_src,
                           int nplanes, int64_t offset, int64_t ncells, int elem_bytes,
                           void* stream);

/* ---- rate surrogate: network and training --------------------------------
 * A small network maps the field magnitude to the logarithms of all Z rates
 * of a species at once (the paper evaluates Eq. 1 directly; the surrogate is
 * the learned alternative and is measured against it):
 *   h1 = g(W1 x + b1), h2 = g(W2 h1 + b2), y = W3 h2 + b3,
 * ION_MLP_HIDDEN = 64 hidden units, K <= ION_MAX_Z outputs, g the GELU in
 * its tanh form g(z) = z/2 (1 + tanh(sqrt(2/pi) (z + 0.044715 z^3))).
 * Parameters are one device FP32 array in the order W1[64], b1[64],
 * W2[64][64] (row o: weights into unit o), b2[64], W3[K][64], b3[K]
 * (ion_mlp_nparams(K) values).  Samples are x[b] and targets t[b*K + k].
 * The training calls below run on the GPU; all arrays are device arrays,
 * 4-byte aligned; batches hold 1..2^24 samples. */
#define ION_MLP_HIDDEN 64
/* Forward pass in the inference arithmetic: W2, W3, h1 and h2 rounded to
 * bf16 pairs (hi = bf16(v), lo = bf16(v - hi); the value hi + lo) and the
 * SFU tanh, as in the tensor-core kernels; the backward pass treats the
 * rounding as the identity (straight-through).  Without it the forward pass
 * is plain FP32 with tanhf. */
#define ION_MLP_BF16 0x1

/* Parameter count for K outputs (ION_EINVAL if K is outside 1..ION_MAX_Z). */
ION_API int64_t ion_mlp_nparams(int K);

/* Workspace bytes of ion_mlp_loss_grad (0 for arguments out of range). */
ION_API size_t ion_mlp_workspace_bytes(int K, int64_t B);

/* ion_mlp_loss_grad -- L = (1/(B K)) sum_b sum_k (y_bk - t_bk)^2 and dL/dP.
 *   P     device [ion_mlp_nparams(K)] parameters (read).
 *   x, t  device [B] inputs and [B*K] targets.
 *   flags 0 or ION_MLP_BF16.
 *   grad  device [ion_mlp_nparams(K)], overwritten with dL/dP.
 *   loss  device float or NULL: L.
 *   workspace  device, 256-byte aligned, >= ion_mlp_workspace_bytes(K, B).
 * The batch sums are taken in a fixed order: equal inputs give equal bits.
 * Errors: ION_EINVAL, ION_ECUDA. */
ION_API int ion_mlp_loss_grad(const float* P, int K, const float* x, const float* t,
                              int64_t B, int flags, float* grad, float* loss,
                              void* workspace, size_t workspace_bytes, void* stream);

/* ion_mlp_adam -- one Adam step (t >= 1) on n parameters in place:
 * m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
 * P -= lr (m/(1-b1^t)) / (sqrt(v/(1-b2^t)) + eps).  m and v start at zero.
 * Errors: ION_EINVAL, ION_ECUDA. */
ION_API int ion_mlp_adam(float* P, const float* grad, float* m, float* v, int64_t n,
                         float lr, float beta1, float beta2, float eps, int t,
                         void* stream);

/* ion_mlp_forward -- y[b*K + k] for B inputs on CUDA cores (FP32, or with
 * ION_MLP_BF16 the inference arithmetic); the reference the tensor-core
 * surrogate kernels are checked against.  Errors: ION_EINVAL, ION_ECUDA. */
ION_API int ion_mlp_forward(const float* P, int K, const float* x, int64_t B, int flags,
                            float* y, void* stream);

/* ---- rate surrogate: training data ---------------------------------------
 * The arithmetic that turns fields and rates into the network's inputs and
 * targets (the paper has no counterpart; the targets are Eq. 1 itself). */

/* ion_log2_rates -- the training targets: max(log2 W_k(|E_c|), floor) with
 * W_k of Eq. 1 in 1/fs, evaluated in FP64 in its log2 form (the exponent
 * a_k - b_k log2|E| - C_k/|E| itself, no exp2/log2 round trip); floor where
 * W_k is 0 (|E| below 1e-6 GV/m, or past the exponent cutoff of Eq. 1).
 *   E     device float [ncells] fields in GV/m (sign ignored).
 *   out   device double, out[c*ldo + (k - k_lo)] for k_lo <= k < k_hi
 *         (cell-major: one row of rates per sample), ldo >= k_hi - k_lo.
 * 0 <= k_lo < k_hi <= Z; 0 <= ncells < 2^31; the species' device is
 * current.  Errors: ION_EINVAL, ION_ECUDA. */
ION_API int ion_log2_rates(const ion_species* sp, const float* E, int64_t ncells, int k_lo,
                           int k_hi, double floor, double* out, int64_t ldo, void* stream);

/* ion_mlp_inputs -- the network's input x_c = clamp(2 (log2|E_c| - l2lo) /
 * (l2hi - l2lo) - 1, -1, 1), computed in FP64 and rounded to float, as the
 * inference kernels map |E| (log2 of 0 is -infinity, so x = -1).
 *   E, x  device float [n], 0 <= n < 2^40; finite l2lo < l2hi.
 * Errors: ION_EINVAL, ION_ECUDA. */
ION_API int ion_mlp_inputs(const float* E, int64_t n, double l2lo, double l2hi, float* x,
                           void* stream);

/* ion_mlp_standardize -- per-column standardization of the targets:
 *   mean_k = (1/n) sum_c Y[c*K + k],
 *   scale_k = max(sqrt(sum_c (Y[c*K + k] - mean_k)^2 / (n - 1)), min_scale),
 *   T[c*K + k] = (float)((Y[c*K + k] - mean_k) / scale_k).
 *   Y          device double [n*K] (cell-major, as ion_log2_rates writes).
 *   mean_out,
 *   scale_out  device double [K].
 *   T          device float [n*K].
 * 2 <= n < 2^32, 1 <= K <= ION_MAX_Z, min_scale > 0.  The sums run in
 * FP64 in a fixed order, one block of threads per column (equal inputs give
 * equal bits).  Allocates nothing.  Errors: ION_EINVAL, ION_ECUDA. */
ION_API int ion_mlp_standardize(const double* Y, int64_t n, int K, double min_scale,
                                double* mean_out, double* scale_out, float* T, void* stream);

/* ---- rate surrogate: inference -------------------------------------------
 * A trained network (parameters as above, K = Z outputs) becomes an
 * ion_surrogate: W2 and W3 as bf16 pairs (hi = bf16(w), lo = bf16(w - hi))
 * laid out for the tensor cores, the other parameters in FP32.  Its kernels
 * evaluate the network for 128 cells at a time: layer 1 (one input) and the
 * GELUs on the CUDA cores, layers 2 and 3 as 128 x 64 x 64 and 128 x N x 64
 * bf16 products with FP32 accumulation on the tensor cores (tcgen05,
 * accumulators in tensor memory), the activations as bf16 pairs too, each
 * product as hi*hi' + hi*lo' + lo*hi' (16 significant bits per operand).
 *
 * Input and output scaling (ion_surrogate_norm):
 *   x = 2 (log2|E| - log2E_min) / (log2E_max - log2E_min) - 1,
 *   log2 W_k [1/fs] = y_mean[k] + y_scale[k] * y_k,  W_k = 0 where that is
 *   below y_floor.
 * The network is trusted only for log2E_min <= log2|E| <= log2E_max, and
 * only where its validation error bound allows (ion_step_surrogate). */
typedef struct ion_surrogate ion_surrogate; /* opaque, owned by the library */

typedef struct {
  double log2E_min, log2E_max; /* trained range of log2(|E| / (GV/m)) */
  double y_floor;              /* log2 W below this is W = 0 */
  double y_mean[ION_MAX_Z];
  double y_scale[ION_MAX_Z];
} ion_surrogate_norm;

/* ion_surrogate_create -- a surrogate of species `sp` (K = Z outputs).
 *   P      device FP32 [ion_mlp_nparams(Z)] trained parameters (read during
 *          the call; synchronous copy).
 *   norm   host, the scaling above; log2E_min < log2E_max.
 *   bound  host [nbins * Z] or NULL: bound[b*Z + k] >= max |log2 W_k(net) -
 *          log2 W_k(Eq. 1)| over the inputs of bin b, the bins splitting
 *          [log2E_min, log2E_max] into nbins equal parts (1 <= nbins <=
 *          65536), values clamped below at y_floor on both sides.  NULL
 *          trusts the network everywhere in range (bound 0).
 * The surrogate keeps its own copy of the species table.  Allocates device
 * memory.  Errors: ION_EINVAL, ION_ENOMEM, ION_ECUDA. */
ION_API int ion_surrogate_create(const ion_species* sp, const float* P,
                                 const ion_surrogate_norm* norm, const float* bound,
                                 int nbins, ion_surrogate** out);
ION_API int ion_surrogate_destroy(ion_surrogate* s);

/* ion_surrogate_rates -- the network's W_k(|E_c|) in 1/fs for every state
 * k < Z of every cell: W_out[k*ldw + c] (device, float, ldw >= ncells).
 * No range check: cells outside the trained range get the network's
 * extrapolation.  Errors: ION_EINVAL, ION_ECUDA.  (A bounded wait for the
 * tensor cores that gives up leaves NaN in the rates of its cells.) */
ION_API int ion_surrogate_rates(const ion_surrogate* s, const float* E, int64_t ncells,
                                float* W_out, int64_t ldw, void* stream);

/* ion_step_surrogate -- ion_step (ION_F32) with the window's rates taken
 * from the network where it can be trusted: for a cell with |E| in the
 * trained range, the network's rates W_r of the window's w-1 transitions
 * give a bound on the population error of the step,
 *   2 dt sum_r (max(W_r, 2^y_floor) (2^bound - 1) + 2^y_floor)
 * (a perturbation of the rate matrix by dA moves the solution of Eq. 3 by
 * at most |dA| in the 1-norm); if it is below pop_tol the network's rates
 * are used, otherwise (and outside the range) the rates of Eq. 1; pop_tol 0
 * never uses the network.  A cell
 * with some rate W dt > 1 always takes the rates of Eq. 1 (its bound would
 * exceed any useful tolerance) and is finished in the Bateman form by
 * ion_step's record kernel.  The update itself is ion_step's (Taylor or
 * Bateman form, FP64 coefficients for nearly degenerate rate pairs, window
 * slide).  Arguments as ion_step with
 * FP32 arrays; pop_tol >= 0.  Workspace: ion_step_workspace_bytes(ncells,
 * ION_F32); after the call its header holds, besides the words described
 * for ion_step, word 3: cells that took the network's rates, word 4: cells
 * that took the rates of Eq. 1, word 5: non-zero if a bounded wait for the
 * tensor cores gave up (the results of the call are then invalid).
 * Errors: ION_EINVAL, ION_ECUDA. */
ION_API int ion_step_surrogate(const ion_surrogate* s, const float* E, float* N, int64_t ld,
                               int64_t ncells, double dt_fs, uint8_t* k_lo, uint8_t* k_hi,
                               float* dne, const float* n_gas, const ion_step_opts* opts,
                               double pop_tol, void* workspace, size_t workspace_bytes,
                               void* stream);

/* ion_surrogate_test_timeout -- test hook of the bounded waits (the paper
 * has no counterpart).  With on != 0, every later call of this surrogate
 * (ion_surrogate_rates, ion_step_surrogate) makes the first tensor-core
 * wait of each tile poll, 64 times, an mbarrier that nothing arrives at, so
 * that the wait gives up exactly as a wait that ran out of its limit would:
 * ion_step_surrogate leaves every cell untouched and sets word 5 of the
 * workspace header, ion_surrogate_rates writes NaN rates, and each CTA waits
 * (bounded) for the matrix products it skipped before it frees its tensor
 * memory.  on = 0 restores the normal waits.  Synchronous (one 4-byte copy
 * to the device).  Errors: ION_EINVAL, ION_ECUDA. */
ION_API int ion_surrogate_test_timeout(ion_surrogate* s, int on);

/* ion_surrogate_validate -- the validation error bound, computed on the GPU
 * and installed in the surrogate (replacing any bound it had): the trained
 * range [log2E_min, log2E_max] is split into nbins equal bins; bin b is
 * sampled at per_bin points l2 = log2E_min + (log2E_max - log2E_min)
 * (b + i/(per_bin - 1))/nbins, i = 0..per_bin-1 (both edges included), at
 * E = (float)2^l2.  There the network's rates (as ion_surrogate_rates gives
 * them) and Eq. 1's in FP64 are compared in log2, both clamped below at
 * y_floor:
 *   bound[b*Z + k] = margin * max_i |log2 W_k(net) - log2 W_k| + floor_add.
 *   bound_out  host float [nbins*Z] or NULL: a copy of the bound.
 * 1 <= nbins <= 65536, 2 <= per_bin <= 4096, nbins * per_bin <= 2^24,
 * finite margin >= 1 and floor_add >= 0.  Allocates and frees device
 * scratch (about 4 (Z + 1) nbins per_bin bytes) and synchronizes the
 * stream; not to be called while another call uses the surrogate.  A bounded tensor-core wait that gives up makes
 * the call fail (ION_ETIMEOUT) and leaves the old bound.
 * Errors: ION_EINVAL, ION_ENOMEM, ION_ECUDA, ION_ETIMEOUT. */
ION_API int ion_surrogate_validate(ion_surrogate* s, int nbins, int per_bin, double margin,
                                   double floor_add, float* bound_out, void* stream);

/* ion_measure_peaks -- throughput of the current device for the arithmetic
 * the step's forms are bound by, from loops of independent dependency chains
 * over all SMs: out[0] FP32 ex2 (SFU) per second, out[1] FP32 tanh (SFU) per
 * second, out[2] FP64 flop/s of fused multiply-adds, out[3] FP64 exp2 per
 * second.  A measurement utility: it allocates 64 bytes, creates events and
 * synchronizes (about 0.1 s).  The paper has no counterpart.
 * Errors: ION_EINVAL, ION_ECUDA. */
ION_API int ion_measure_peaks(double* out);

/* ion_binary_version -- the compute capability the library's device code
 * was compiled for, as the CUDA runtime reports it for the loaded module
 * (major * 10 + minor: 103 for sm_103a), or ION_ECUDA if the current device
 * cannot load it.  A build check; the paper has no counterpart. */
ION_API int ion_binary_version(void);

/* Message of the last failed call on this thread ("" if none). */
ION_API const char* ion_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* IONIZE_H */
