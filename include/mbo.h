/*
 * mbo.h - C ABI of the GB300 (sm_103a) generalized MBO library.
 *
 * The library runs Algorithm 1 ("a:MBO") of Osting & Wang, "A generalized MBO
 * diffusion generated motion for orthogonal matrix-valued fields"
 * (arXiv:1711.01365) on a flat torus [0,1)^d, d = 2 or 3:
 *   diffusion  (Sec. 5.1): every entry A_ij is advanced by the periodic heat
 *              semigroup, A~ = iFFT( g(k) FFT(A_ij) ), g(k) = exp(-4 pi^2 tau |k|^2);
 *   projection (Lemma 1.1): every grid point becomes U V^t, the closest
 *              orthogonal matrix to A~(x) = U S V^t, whose determinant has the
 *              sign of det A~(x) (det A~ = 0 -> +1; A~ = 0 -> identity);
 *   Lyapunov functional (Sec. 4): E(A) = (prod h_j / tau) sum_x (n - <A, e^{tau Lap} A>_F);
 *   stationarity (Prop. 4.6): a step is stationary when no point changes its
 *              determinant sign and every entry moves by at most tol.
 *
 * Conventions shared by every entry point
 *   - Fields are planar arrays of n*n channels: channel c = i*n + j holds matrix
 *     entry (i,j); each channel is a row-major block of P = prod(dims) values
 *     with the last axis (x) fastest.  dims is {Ny, Nx} (d = 2) or
 *     {Nz, Ny, Nx} (d = 3).  Element type: float (MBO_F32) or double (MBO_F64),
 *     as given to mbo_create.
 *   - Field pointers are CALLER-OWNED device pointers, 16-byte aligned, unless
 *     an entry point says otherwise.  The library never frees them.
 *   - stream is a cudaStream_t passed as void*; NULL is the legacy default
 *     stream.  Calls are asynchronous on that stream unless they return a
 *     value on the host (documented per call).
 *   - Every entry point returns an mbo_status; nothing is thrown.  Device-side
 *     problems (non-finite values, a wait that gave up) are recorded in the
 *     handle and reported by the next call that synchronises.
 *   - A handle is not thread safe; distinct handles are independent.
 *   - Supported sizes: every N_j = 2^a 3^b with 2 <= N_j <= 2048; n in {1,2,3,4};
 *     other sizes return MBO_ERR_UNSUPPORTED_SIZE.
 */
#ifndef MBO_GB300_H
#define MBO_GB300_H

#include <stdint.h>

#if defined(__GNUC__)
#define MBO_API __attribute__((visibility("default")))
#else
#define MBO_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mbo_ctx* mbo_handle;

typedef enum { MBO_F32 = 1, MBO_F64 = 2 } mbo_dtype;

typedef enum {
  MBO_OK = 0,
  MBO_ERR_INVALID_ARG = 1,      /* null/misaligned pointer, bad n, tau <= 0, ... */
  MBO_ERR_UNSUPPORTED_SIZE = 2, /* an axis length outside 2^a 3^b in [2, 2048]   */
  MBO_ERR_OOM = 3,              /* device allocation failed                       */
  MBO_ERR_CUDA = 4,             /* a CUDA runtime call failed (see mbo_last_error) */
  MBO_ERR_NUMERIC = 5,          /* NaN or Inf met in the projected field          */
  MBO_ERR_DEVICE_TIMEOUT = 6    /* a bounded device-side wait gave up             */
} mbo_status;

/* Options; mbo_default_config fills the defaults. */
typedef struct {
  double fallback_sigma; /* MBO_F32.  n = 3 and 4: points whose smallest-
                            singular-value estimate |det A~| / |cof A~|_F is at
                            most max(fallback_sigma, 1e-6 |A~|_F), or that are
                            singular to single precision, skip the FP32 Newton
                            iteration and take an exact form instead: for n = 3
                            the quaternion form where (s2 + s3) / |A~|_F is not
                            small, else (and always for n = 4) FP64
                            re-projection from the FP32 A~.  n = 2: points whose
                            smallest singular value is below it are re-projected
                            in FP64.  Default 0.  Ignored for F64.                 */
  int check_interval;    /* run loop: the host reads the step records every this
                            many steps to test for stationarity (default 16).    */
  int use_graph;         /* run loop: replay the step from a captured CUDA graph
                            (default 1).                                          */
  int row_threads;       /* launch shape of the x-axis (row) pass: threads per
                            block, a multiple of 32 in [32, 384]; 0 = automatic.  */
  int axis_threads;      /* threads per block of the y / z passes, a multiple of
                            32 in [64, 384]; 0 = automatic.                       */
  int axis_tx;           /* x-columns per block of the y / z passes: a power of
                            two dividing Nx, at most 16; 0 = automatic.           */
  int axis_stages;       /* MBO_F32 y / z passes of length 256..2048: tile
                            buffers per block, 1 or 2 (2: the next tile's copy is
                            in flight while a tile is transformed), or 3: one
                            tile buffer and a separate transpose buffer (the
                            next copy goes out once a tile is in registers);
                            0 = automatic.                                      */
  int autotune;          /* 1: mbo_create times the candidate launch shapes of
                            this geometry (tile width, tile buffers, threads per
                            block of the strided and row passes, dependent
                            launch, the x pass as one wave of blocks or one
                            block per row group) on a scratch
                            field and keeps the fastest; the choice is cached
                            per (dims, n, dtype) for the process.  Fields set
                            explicitly above are not tuned.  Default 0.        */
  int pdl;               /* MBO_F32 warp-plan passes: programmatic dependent
                            launch, each pass scheduled while the one before it
                            finishes.  1 = on, 2 = off, 0 = automatic (on where
                            the x pass runs in at most two waves of blocks;
                            tuned when autotune is set).                        */
} mbo_config;

/* Per-step record.  Step s maps A_{s} to A_{s+1}. */
typedef struct {
  double energy;           /* E^tau(A_s), accumulated in FP64 (Sec. 4)            */
  double max_delta;        /* max over points and channels |A_{s+1} - A_s|        */
  int64_t det_flips;       /* points where sign det A_{s+1} != sign det A_s       */
  int64_t fallback_points; /* MBO_F32: points re-projected in FP64                */
  int64_t nonfinite;       /* points whose projection is not finite               */
} mbo_stats;

MBO_API void mbo_default_config(mbo_config* cfg);

/* The launch shapes a handle uses (after any autotuning): row_threads,
 * axis_threads, axis_tx, axis_stages and pdl (1 on, 2 off) filled in; the
 * other fields as the handle was created with. */
MBO_API mbo_status mbo_launch_config(mbo_handle h, mbo_config* out);

/* Create a handle for one field geometry.
 *   out   receives the handle (set to NULL on failure).
 *   ndim  2 or 3; dims[ndim] as in the conventions above.
 *   n     matrix order (1 to 4); tau > 0 the diffusion time of one step.
 *   cfg   NULL for the defaults.
 * Allocates the spectral workspace (ceil(n*n/2) complex planes of P points)
 * and small tables on the current device.  Synchronous. */
MBO_API mbo_status mbo_create(mbo_handle* out, int ndim, const int64_t* dims, int n, double tau,
                      mbo_dtype dtype, const mbo_config* cfg);

/* Release the handle and everything it allocated.  Synchronises the device. */
MBO_API mbo_status mbo_destroy(mbo_handle h);

/* Diffusion step of Algorithm 1 alone (Sec. 5.1): A_tilde = e^{tau Lap} A.
 * A and A_tilde are device fields (they may be the same pointer). */
MBO_API mbo_status mbo_diffuse(mbo_handle h, const void* A, void* A_tilde, void* stream);

/* Projection step of Algorithm 1 alone (Lemma 1.1): B(x) = polar factor of
 * A_tilde(x).  det_sign (nullable, int8 per point) receives +1 or -1, the
 * class chosen for B.  A_tilde and B may be the same pointer. */
MBO_API mbo_status mbo_project(mbo_handle h, const void* A_tilde, void* B, int8_t* det_sign,
                       void* stream);

/* Flag for mbo_step: the field is the one the previous mbo_step (or run) on
 * this handle left, unmodified since; its forward row transform, kept in the
 * workspace, is reused and one of the three transform passes is skipped. */
#define MBO_STEP_CONTINUE 1

/* One iteration of Algorithm 1 in place: A <- polar(e^{tau Lap} A), fused
 * (transform passes, heat multiplier, projection, energy, statistics).
 * stats (nullable): if given, the call synchronises the stream and fills the
 * record of this step (energy is that of the input field). */
MBO_API mbo_status mbo_step(mbo_handle h, void* A, int flags, mbo_stats* stats, void* stream);

/* Lyapunov functional E^tau(A) (Sec. 4), in its Parseval form
 *   (1/(P tau)) [ (1/P) sum_k (1 - g(k)) sum_c |A^_c(k)|^2 + sum_x (n - |A(x)|_F^2) ],
 * accumulated in FP64.  Synchronises the stream; result in *E. */
MBO_API mbo_status mbo_lyapunov(mbo_handle h, const void* A, double* E, void* stream);

/* Iterate Algorithm 1 in place until a step is stationary (no determinant
 * sign flips and max |A_{s+1} - A_s| <= tol) or max_steps steps were taken.
 * A may be a device pointer or a host pointer (pageable or pinned); for a host
 * pointer the field is copied to the device, iterated, and copied back.
 * Outputs (all nullable):
 *   steps_taken  number of steps performed;
 *   stationary   1 if the last step was stationary, else 0;
 *   energies     [max_steps + 1]: E^tau(A_0) ... E^tau(A_steps);
 *   max_deltas   [max_steps]: per-step max |A_{s+1} - A_s|;
 *   det_flips    [max_steps]: per-step determinant sign flips;
 *   last         record of the last step.
 * tol < 0 never stops early.  Synchronises the stream before returning. */
MBO_API mbo_status mbo_run_until_stationary(mbo_handle h, void* A, int max_steps, double tol,
                                    int* steps_taken, int* stationary, double* energies,
                                    double* max_deltas, int64_t* det_flips, mbo_stats* last,
                                    void* stream);

/* Per-pass device timing.  While enabled, every kernel pass launched through
 * this handle is bracketed by CUDA events on its stream (the run loop then
 * launches directly instead of replaying its graph).  mbo_profile_enable
 * (re)starts the accumulation; mbo_profile_read synchronises on the recorded
 * events and returns, per pass id below, the summed milliseconds and the
 * number of launches (arrays of length npass, nullable). */
enum {
  MBO_PASS_ROW_FWD = 0,      /* forward x transform of a field                 */
  MBO_PASS_AXIS_FWD = 1,     /* forward y transform (3-D)                      */
  MBO_PASS_AXIS_FGI = 2,     /* last axis: forward, heat multiplier, inverse   */
  MBO_PASS_AXIS_INV = 3,     /* inverse y transform (3-D)                      */
  MBO_PASS_AXIS_ENERGY = 4,  /* last axis: forward + energy only               */
  MBO_PASS_ROW_PROJECT = 5,  /* inverse x, projection, statistics, forward x   */
  MBO_PASS_ROW_INV = 6,      /* inverse x to a real field (mbo_diffuse)        */
  MBO_PASS_PROJECT = 7,      /* pointwise projection (mbo_project)             */
  MBO_PROFILE_PASSES = 8
};
MBO_API mbo_status mbo_profile_enable(mbo_handle h, int enable);
MBO_API mbo_status mbo_profile_read(mbo_handle h, double* ms, int64_t* launches, int npass);

/* Self-test of the device-side timeout path (no paper counterpart).  Every
 * wait inside the library's kernels is bounded; on expiry a kernel sets an
 * error bit in the handle's device state, gives its copies in flight a bounded
 * wait and returns, and the next synchronising call reports
 * MBO_ERR_DEVICE_TIMEOUT (clearing the bit).  This call runs that path on
 * purpose: one block waits, with the same bounded wait, on an mbarrier phase
 * that nothing completes, for limit_cycles SM cycles (1 .. 2e9), then returns.
 * Expected result: MBO_ERR_DEVICE_TIMEOUT, with the handle usable afterwards.
 * Synchronises stream.  Errors: MBO_ERR_INVALID_ARG (null handle, limit out of
 * range), MBO_ERR_CUDA. */
MBO_API mbo_status mbo_selftest_wait_timeout(mbo_handle h, int64_t limit_cycles, void* stream);

/* Throughput of the SIMT fused multiply-add pipes of the current device, in
 * TFLOP/s (2 flops per multiply-add): FP32 scalar FFMA, FP32 packed pairs
 * (two multiply-adds per instruction) and FP64 DFMA, each the best of five
 * timed launches of independent a <- a b + c chains over every SM.  A
 * measurement utility (the paper has no counterpart): the benchmark states
 * the FP64 form's ALU roofline against it.  Allocates 64 bytes; synchronous;
 * changes no clock or power setting.  Errors: MBO_ERR_INVALID_ARG (null
 * output), MBO_ERR_OOM, MBO_ERR_CUDA. */
MBO_API mbo_status mbo_measure_fma_peaks(double* fp32_tflops, double* fp32x2_tflops,
                                         double* fp64_tflops);

/* Diffusion without any device allocation.
 *
 * Same result as mbo_diffuse (A_tilde = e^{tau Lap} A on the grid given by
 * ndim/dims, n, tau and dtype, as in mbo_create), but without a handle and
 * without calling cudaMalloc, cudaFree or any allocating routine.  It is meant
 * for callers that must not allocate device memory: code that runs while a
 * framework's caching allocator already holds the device memory it is allowed
 * to use, loops that cannot take the synchronisation that cudaMalloc/cudaFree
 * may imply, and programs whose device memory budget is fixed in advance.  The
 * paper has no counterpart of this entry point; it only changes where the
 * scratch memory lives.
 *
 * Scratch: one statically sized device array of MBO_NOALLOC_SCRATCH_BYTES
 * (64 MiB) inside this library.  Every GPU that loads the library keeps it
 * until the process exits.  A call needs ceil(n*n/2) * prod(dims) * 2 * w
 * bytes of workspace (w = 4 for MBO_F32, 8 for MBO_F64) plus under 100 KB of
 * tables; a larger problem (for example 1024 x 1024 with n = 3 in MBO_F64)
 * returns MBO_ERR_UNSUPPORTED_SIZE and does nothing.
 *   - The first call on each device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current; make that first call
 *     before any stream capture.
 *   - All calls share the one array, which keeps the last call's contents.
 *     Every call writes the tables and workspace it reads before reading them,
 *     so nothing needs clearing; but calls that overlap on the GPU (different
 *     streams, or host threads without ordering) race on the array: order them,
 *     for example by using one stream.
 * A and A_tilde: caller-owned, 16-byte-aligned fields in the memory of the
 * CURRENT device (the call runs there, with that device's copy of the array);
 * they may be equal.  Asynchronous on stream.  Errors: MBO_ERR_INVALID_ARG
 * (bad argument, or a pointer that is not device memory of the current
 * device), MBO_ERR_UNSUPPORTED_SIZE (axis length, scratch too small, or row /
 * column tiles larger than the device's shared memory per block, e.g. 2048
 * points along x with n = 4 in MBO_F64), MBO_ERR_CUDA (a launch or the address
 * lookup failed).  Every check runs before the first launch. */
#define MBO_NOALLOC_SCRATCH_BYTES (64u << 20)
MBO_API mbo_status mbo_diffuse_noalloc(int ndim, const int64_t* dims, int n, double tau,
                                       mbo_dtype dtype, const void* A, void* A_tilde,
                                       void* stream);

/* ------------------------------------------------------------------------- */
/* Volume-preserving MBO (Sec. 7).  The diffusion step is unchanged; the     */
/* projection is replaced by the assignment of Lemma 7.2: with T+ / T- the   */
/* closest matrices of SO(n) / SO^-(n) to A~(x) (Lemma 7.1) and              */
/* dE(x) = <T+ - T-, A~(x)>_F = 2 sign(det A~) sigma_min(A~), the n_plus      */
/* points of largest dE take T+ and all others T- (Algorithm 3 on a uniform   */
/* grid); equal dE values are ordered by grid index, lower index first.      */
/* ------------------------------------------------------------------------- */

/* One volume-preserving step in place.  n_plus: the number of points that
 * lie in SO(n) after the step (0 <= n_plus <= P); < 0 keeps the number of
 * points of A with det > 0.  stats as in mbo_step (energy of the input).
 * Allocates the step's buffers (a field copy and 8 bytes per point) on first
 * use.  Handles of order n = 4 return MBO_ERR_UNSUPPORTED_SIZE (both volume
 * calls). */
MBO_API mbo_status mbo_step_volume(mbo_handle h, void* A, int64_t n_plus, mbo_stats* stats,
                                   void* stream);

/* Iterate the volume-preserving step until stationary (as
 * mbo_run_until_stationary) with the SO(n) point count fixed at n_plus (< 0:
 * that of the initial field).  A: device field.  energies (nullable,
 * max_steps + 1 values; the last 1024 steps when the run is longer).
 * Synchronises. */
MBO_API mbo_status mbo_run_volume(mbo_handle h, void* A, int64_t n_plus, int max_steps, double tol,
                                  int* steps_taken, int* stationary, double* energies,
                                  void* stream);

/* ------------------------------------------------------------------------- */
/* Batches of independent fields.  Fields may differ in ndim, dims, n and tau */
/* (one dtype per batch).  One step of the batch runs every field's step     */
/* (Algorithm 1) from a single CUDA graph launch whose per-field branches are */
/* independent, so fields of uneven sizes run concurrently.                  */
/* ------------------------------------------------------------------------- */
typedef struct mbo_batch_ctx* mbo_batch;

/* count fields; field i has ndim[i] in {2, 3} and dims dims[3*i .. 3*i+ndim[i]-1]
 * (as in mbo_create), order n[i] and diffusion time tau[i].  Allocates each
 * field's workspace and tables.  Synchronous.  Errors as mbo_create (the
 * first failing field is named by mbo_batch_last_error). */
MBO_API mbo_status mbo_batch_create(mbo_batch* out, int count, const int* ndim, const int64_t* dims,
                                    const int* n, const double* tau, mbo_dtype dtype,
                                    const mbo_config* cfg);
MBO_API mbo_status mbo_batch_destroy(mbo_batch b);

/* One step of every field, in place: A[i] is field i's caller-owned device
 * field (layout as in mbo_step).  flags: MBO_STEP_CONTINUE as in mbo_step.
 * stats (nullable, count records): if given the call synchronises and fills
 * each field's record.  The step graph is captured on first use for a set of
 * field pointers and replayed afterwards. */
MBO_API mbo_status mbo_batch_step(mbo_batch b, void* const* A, int flags, mbo_stats* stats,
                                  void* stream);

/* Iterate every field until its own step is stationary (then its kernels
 * skip further steps) or max_steps steps were taken, as
 * mbo_run_until_stationary.  A[i]: device fields.  Outputs (nullable):
 * steps_taken[count], stationary[count], energies[count * (max_steps + 1)]
 * (row i: E^tau(A_0) .. E^tau(A_steps_i) of field i), last[count].
 * Synchronises the stream before returning. */
MBO_API mbo_status mbo_batch_run(mbo_batch b, void* const* A, int max_steps, double tol,
                                 int* steps_taken, int* stationary, double* energies,
                                 mbo_stats* last, void* stream);

/* Total device bytes the batch holds. */
MBO_API int64_t mbo_batch_workspace_bytes(mbo_batch b);

/* Text of the last error recorded in the batch. */
MBO_API const char* mbo_batch_last_error(mbo_batch b);

/* Bytes of device memory the handle holds (workspace and tables). */
MBO_API int64_t mbo_workspace_bytes(mbo_handle h);

/* Human-readable text for a status code (static storage). */
MBO_API const char* mbo_status_string(mbo_status s);

/* Text of the last error recorded in the handle (empty string if none). */
MBO_API const char* mbo_last_error(mbo_handle h);

#ifdef __cplusplus
}
#endif

#endif /* MBO_GB300_H */
