/*
 * bpm.h -- C ABI of the GB300-native two-beam FFT beam propagation method.
 *
 * Method: Krzywinski & Halavanau, "Time-dependent dynamical Bragg diffraction
 * in deformed crystals by beam propagation method (BPM)", arXiv:2201.08500.
 * For every frequency channel omega_i of an X-ray pulse, the transmitted and
 * reflected slowly varying envelopes E0 (carrier exp(+i h x/2)) and Eh
 * (carrier exp(-i h x/2)) are marched through the crystal in z (Eq. fov10):
 * each step Fourier-transforms both envelopes along x (x and y in 3D),
 * multiplies them by the tilted angular propagators (Eq. fov4 and the shifted
 * operators p+- defined after Eq. fov10), transforms back and couples them
 * pointwise through the first Jacobi-Anger terms of the susceptibility step
 * (Eqs. fov9, fov11, fov12) with the Zassenhaus-like factor and the
 * deformation phase exp(+-i h u) (Eq. Authier).  The time response is the
 * channel sum of Section 3.3 (text after Eq. ref:tdp).
 *
 * Conventions (all calls):
 *  - Units are SI; scalars are double precision.
 *  - Grid: x_j = j dx (j < nx); in 3D y_r = (r - ny/2) dy.  Fields are row-major
 *    [channel][y][x] complex64 (interleaved re, im float32).
 *  - Every call returns a bpm_status and never throws or aborts.  On error the
 *    plan keeps its previous state and bpm_last_error() describes the failure.
 *  - Ownership: the caller owns the CUDA stream and every buffer it passes.
 *    Host arrays are copied before the call returns.  Device pointers passed
 *    in (u_field with u_on_device=1, set_fields/fetch with on_device=1) must
 *    stay valid until the plan's stream has consumed them.  The plan owns its
 *    internal device memory (tables, fields, outputs) until bpm_plan_destroy.
 *  - Threads: a plan is used by one host thread at a time.  Distinct plans may
 *    be used concurrently.  Device work is asynchronous on the plan's stream;
 *    bpm_sync() waits for it and reports device-side failures.
 *  - There is no CPU fallback: without a usable GB300 (sm_103a) device the
 *    calls return BPM_ERR_CUDA or BPM_ERR_UNSUPPORTED.
 */
#ifndef BPM_H_
#define BPM_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define BPM_API __attribute__((visibility("default")))

typedef enum {
  BPM_OK = 0,
  BPM_ERR_INVALID_ARG = 1, /* bad size, pointer, ordering of calls or physics input */
  BPM_ERR_OOM = 2,         /* device allocation failed / batch has no room yet     */
  BPM_ERR_CUDA = 3,        /* a CUDA runtime call or kernel launch failed          */
  BPM_ERR_UNSUPPORTED = 4, /* grid size or option this build does not implement    */
  BPM_ERR_TIMEOUT = 5,     /* a bounded device-side wait gave up                   */
  BPM_ERR_STATE = 6,       /* call out of order (e.g. run before set_pulse)        */
  BPM_ERR_CANCELLED = 7    /* batch entry was cancelled                            */
} bpm_status;

typedef struct bpm_plan_s* bpm_plan;

/* Transverse grid and march.  dims = 2: (x, z), ny must be 1; dims = 3: (x, y, z).
 * nx (and ny) are powers of two: 256..8192 for dims = 2, 64..1024 for dims = 3.
 * split_order (Eq. split-op): 1 = first order (a1 = b1 = 1, Eq. fov4); 2 = Strang
 * (a = (0, 1), b = (1/2, 1/2): half coupling, propagation, half coupling, both
 * halves with Pi and u sampled at z_n; dims = 2 only); 4 = fourth order
 * (t = 1/(2 - 2^(1/3)), a = (0, t, 1-2t, t), b = (t/2, (1-t)/2, (1-t)/2, t/2),
 * every coupling at z_n; dims = 2 only, single plans (not batches), and every
 * transverse mode must propagate: pi/dx + h/2 < k).  zassenhaus: 1 applies exp(D2 dz-hat^2/2),
 * D2 = (chi_h/2/cos alpha)^2, to the zeroth Jacobi-Anger term (Section 2,
 * equation after Eq. split-op); 0 leaves it out. */
typedef struct {
  int32_t dims;
  int32_t nx, ny, nz;
  double dx, dy, dz;
  int32_t split_order;
  int32_t zassenhaus;
} bpm_grid;

/* Creates a plan for n_channels frequency channels on cuda_stream (a
 * cudaStream_t; NULL = legacy default stream).  Validates the grid and
 * allocates the plan's device buffers.
 * Errors: INVALID_ARG (null pointers, n_channels < 1, non-positive steps),
 * UNSUPPORTED (sizes outside the list above, split_order not 1, 2 or 4, or
 * not 1 in 3D), OOM, CUDA. */
BPM_API bpm_status bpm_plan_create(const bpm_grid* grid, int n_channels, void* cuda_stream,
                                   bpm_plan* out);

/* Crystal (Section 2, Eqs. fov8, fov11, fov12, Eq. Authier; geometry of the
 * symmetric Bragg slab described before Section 3): susceptibilities chi0,
 * chi_h, chi_hbar (taken literally as complex numbers); Bragg angle theta_B
 * (rad, 0 <= theta_B < 85 deg, Section 2 notes the method fails near
 * back-scattering) and wavelength lambda_B (m) give h = 4 pi sin(theta_B)/lambda_B;
 * the slab occupies x_surface <= x < x_surface + thickness (all z); u_field is
 * the x-component of the displacement in metres, [nz][ny][nx] float64, or NULL
 * for a perfect crystal; u_on_device says whether u_field is a device pointer.
 * Builds the per-cell factor Pi * exp(+i h u) on the device (FP64 phase).
 * Errors: INVALID_ARG, OOM, CUDA. */
BPM_API bpm_status bpm_set_crystal(bpm_plan plan, double chi0_re, double chi0_im, double chih_re,
                                   double chih_im, double chihbar_re, double chihbar_im,
                                   double theta_B, double lambda_B, double x_surface,
                                   double thickness, const double* u_field, int u_on_device);

/* Crystal shape beyond the symmetric-Bragg slab (the method sets the
 * reflection geometry through the crystal's boundaries, end of Section 2):
 * the entrance surface becomes x = x_surface + z tan_psi (asymmetric Bragg cut,
 * the back surface parallel at thickness along x), and the crystal is cut to
 * z_begin <= z < z_end (with an x range covering the grid this is a symmetric
 * Laue slab).  Pi(x_j, z_n) uses x_j = j dx, z_n = n dz, half-open intervals.
 * Call before or after bpm_set_crystal (the deformation factor is rebuilt).
 * Defaults: tan_psi = 0, unbounded z.  Errors: INVALID_ARG, CUDA. */
BPM_API bpm_status bpm_set_geometry(bpm_plan plan, double tan_psi, double z_begin, double z_end);

/* A crystal of any shape (the Introduction offers the method for crystals of
 * arbitrary shape; the reflection geometry follows from the boundaries, end of
 * Section 2). mask holds nz * ny * nx bytes ([nz][ny][nx], ny = 1 in 2D, x
 * fastest). A nonzero byte is a crystal cell at (x_j, y_r, z_n) = (j dx, r dy,
 * n dz).
 * The mask replaces the boundaries of bpm_set_crystal / bpm_set_geometry for
 * Pi(x, y, z_n). The coupling step is applied only in crystal cells, and the
 * deformation phase e^{i h u} only there. NULL returns to the boundaries.
 * Ownership: the plan keeps its own device copy; mask may be freed after the
 * call. on_device says whether mask is a device pointer.
 * Call before or after bpm_set_crystal (the deformation factor is rebuilt).
 * Errors: INVALID_ARG (null plan), CUDA (allocation or copy). */
BPM_API bpm_status bpm_set_crystal_shape(bpm_plan plan, const unsigned char* mask, int on_device);

/* Incident pulse (Section 3.1 beam, Eq. ref:tdp and the frequency decomposition
 * after it): omega[n_channels] angular frequencies (rad/s, uniformly spaced for
 * the time assembly), weight_re_im[2*n_channels] complex spectral amplitudes
 * S_i, incidence angle theta_i (rad), beam centre x0 (m), waist W0 (m),
 * distance to the waist zx and Rayleigh range zR (m).  Per channel the device
 * builds the propagator tables, the coupling coefficients and the incident
 * field A+ = S_i g(x, y) exp(i (k_i sin theta_i - h/2) x), A- = 0, and resets
 * the march to z = 0.  Requires bpm_set_crystal first.
 * Errors: INVALID_ARG (null arrays, k_i <= h/2), UNSUPPORTED (split_order 4 with
 * a non-propagating mode), STATE, OOM, CUDA. */
BPM_API bpm_status bpm_set_pulse(bpm_plan plan, const double* omega, const double* weight_re_im,
                                 double theta_i, double x0, double w0, double zx, double zR);

/* Replaces both envelopes (complex64 [n_channels][ny][nx]) and sets the march
 * position to z_step (0 <= z_step <= nz): resumes from a checkpoint taken with
 * bpm_fetch_fields.  Reflectivities stay normalised to the incident field of
 * the last bpm_set_pulse.  Errors: INVALID_ARG, STATE, CUDA. */
BPM_API bpm_status bpm_set_fields(bpm_plan plan, const void* e0, const void* eh, int z_step,
                                  int on_device);

/* Channel sharding of one pulse across plans, e.g. one per GPU. Section 3.3
 * solves the frequency components as independent stationary problems. Only two
 * sums combine them: the time response (Section 3.3) and R_int (Section 3.1).
 *
 * The call declares that this plan's n_channels channels are channels
 * first .. first + n_channels - 1 of a pulse of n_total channels spaced
 * d_omega. From then on:
 *   - BPM_FIELD_EH_TIME has n_total rows and holds this shard's part of the
 *     sum, i.e. the channels of the other shards count as zero;
 *   - bpm_fetch_reflectivity's R_int is d_omega times this shard's sum of R_i.
 * The shards' time responses and R_int add up (a sum-reduce) to those of one
 * plan holding all n_total channels.
 *
 * Ownership: the plan grows its time-response buffer to n_total rows when
 * needed.
 * Errors: INVALID_ARG if first < 0, the shard does not fit in [0, n_total), or
 * d_omega is not positive and finite; STATE if called after the march has
 * started (z > 0); CUDA if the buffer cannot be grown. */
BPM_API bpm_status bpm_set_channel_shard(bpm_plan plan, int first, int n_total, double d_omega);

/* Advances every channel n_steps split steps (Eq. fov10) from the current z,
 * then computes per-channel reflectivity R_i = sum|A-|^2 / sum|A+(z=0)|^2 and
 * transmissivity T_i, and, when the march has reached nz, the time response
 * (BPM_FIELD_EH_TIME).  Asynchronous on the plan's stream.
 * Errors: INVALID_ARG (n_steps < 0 or past nz), STATE (no pulse), CUDA. */
BPM_API bpm_status bpm_run(bpm_plan plan, int n_steps);

/* Moves the plan to another stream (a cudaStream_t; NULL = legacy stream): work
 * enqueued later by this plan goes there, ordered after everything already
 * enqueued on the old stream.  Used to reuse pooled plans: set up and fetch on a
 * setup stream while a batch stream keeps marching others.  Errors: CUDA. */
BPM_API bpm_status bpm_set_stream(bpm_plan plan, void* cuda_stream);

/* Waits for the plan's stream and reports device status: TIMEOUT if a bounded
 * device wait gave up, CUDA on an asynchronous error. */
BPM_API bpm_status bpm_sync(bpm_plan plan);

enum {
  BPM_FIELD_E0 = 0,     /* complex64  [n_channels][ny][nx], current z              */
  BPM_FIELD_EH = 1,     /* complex64  [n_channels][ny][nx], current z              */
  BPM_FIELD_EH_TIME = 2 /* complex128 [n_time][ny][nx]: psi_h(t_j, x) =
                           d_omega sum_i A-(omega_i, x) exp(-2 pi i (i - n/2) j / n),
                           t_j = 2 pi j / (n d_omega), envelope about omega_{n/2};
                           n = n_time = n_channels, or the shard's n_total (the sum
                           then runs over the shard's channels only)             */
};

/* Copies one output into dst (bytes must equal its exact size) on the plan's
 * stream, then waits for the copy.  dst_on_device selects a device or host
 * destination.  Errors: INVALID_ARG (size/which), STATE (EH_TIME before the
 * march reached nz), CUDA, TIMEOUT. */
BPM_API bpm_status bpm_fetch_fields(bpm_plan plan, int which, void* dst, size_t bytes,
                                    int dst_on_device);

/* Host copies of R[n_channels], T[n_channels] (either may be NULL) and the
 * integrated reflectivity R_int = d_omega * sum_i R_i (d_omega = omega_1 -
 * omega_0; 1 for a single channel).  Waits for the stream. */
BPM_API bpm_status bpm_fetch_reflectivity(bpm_plan plan, double* R, double* T, double* R_int);

/* Timing and launch accounting of the most recent bpm_run (after bpm_sync):
 * march_ms is the device time of the march kernel(s) measured with CUDA events
 * on the plan's stream (0 unless enabled with bpm_set_timing), launches is the
 * number of kernels bpm_run enqueued; threads_per_channel, channels_per_block,
 * blocks and smem_bytes give the 2D march kernel's launch geometry (3D plans:
 * channels_per_block only, the rest 0).  The paper has no counterpart.
 * bpm_set_timing errors: INVALID_ARG (null plan), CUDA (event creation).
 * bpm_get_stats errors: INVALID_ARG (null argument), STATE (the run has not
 * finished: call bpm_sync first), CUDA. */
typedef struct {
  double march_ms;
  int32_t launches;
  int32_t march_launches;
  int32_t threads_per_channel;
  int32_t channels_per_block;
  int32_t blocks;
  int32_t smem_bytes;
} bpm_stats;
BPM_API bpm_status bpm_set_timing(bpm_plan plan, int enable);
BPM_API bpm_status bpm_get_stats(bpm_plan plan, bpm_stats* out);

/* ---------------------------------------------------------------------------
 * Launch forms and their autotuner.  The paper has no counterpart: these
 * choose how the same arithmetic is laid out on the GPU, never what it
 * computes (every form gives bitwise the same fields).
 *
 *   form               2D march: 0 = propagator tables in shared memory and
 *                      twiddles in registers, one channel group per SM;
 *                      1 = tables and twiddles read from L2, at most 128
 *                      registers, two channel groups per SM (first order,
 *                      Nx <= 4096, channels_per_block = the size's maximum);
 *                      2 = parked: one envelope in registers, the other in
 *                      shared memory, tables and twiddles from L2, one channel
 *                      per block and 512/(Nx/16) blocks per SM (first or
 *                      fourth order, Nx = 1024, 2048, 4096,
 *                      channels_per_block = 1);
 *                      3 = parked with the tables in tensor memory (TMEM)
 *                      instead of L2 (first order or Strang, Nx = 2048, 4096,
 *                      8192, channels_per_block = 1; first order at Nx =
 *                      1024 with channels_per_block = 2, the two channels of
 *                      a block marching independently).
 *                      3D passes: 0 = one block per column group and per row
 *                      tile; 1 = the column pass persistent, each column
 *                      streamed in by a bulk copy; 2 = form 1 plus the
 *                      inner row passes persistent, their tiles streamed in
 *                      and out by tensor copies (row_threads 128 at
 *                      nx = 256, 128 or 256 at nx = 512, 256 at nx = 1024);
 *                      channels_per_block = 1.
 *   channels_per_block 2D march: 1, or the maximum of the size (16, 8, 4, 2, 1
 *                      for Nx = 256, 512, 1024, 2048, >= 4096).
 *   row_threads        3D row pass: 256 or 512 threads per block (form 2:
 *                      see above; its first and last row pass use 256), i.e. a tile
 *                      of 256/T or 512/T rows (T = nx/16); taller tiles move
 *                      longer column segments in the transposed store.
 *   ms                 bpm_tune: median time of `steps` steps in this form. */
typedef struct {
  int32_t form;
  int32_t channels_per_block;
  int32_t row_threads;
  float ms;
} bpm_launch;

/* The plan's launch form (chosen at creation: the tuned form of its shape if
 * bpm_tune or bpm_tune_load provided one, else the default).  Errors: INVALID_ARG. */
BPM_API bpm_status bpm_get_launch(bpm_plan plan, bpm_launch* out);

/* Forces a launch form for later bpm_run calls (ms is ignored).
 * Errors: INVALID_ARG (a form this plan cannot run). */
BPM_API bpm_status bpm_set_launch(bpm_plan plan, const bpm_launch* form);

/* Autotuner: creates a scratch plan of this grid (nz replaced by `steps`) and
 * n_channels, with a synthetic crystal slab over a quarter of x and a Gaussian
 * beam, times every launch form the shape can run (one warm-up and three timed
 * runs of `steps` steps each, CUDA events), and records the fastest for later
 * plans of the same (dims, nx, ny, split_order, n_channels) in this process.
 * best receives the fastest; all (capacity max_all, may be NULL) receives every
 * measured form, and n_all their count.  Runs on its own stream and waits for it.
 * Use a few hundred steps: short runs over-weight one-time costs (the
 * shared-memory form copies each channel's tables once per launch).
 * Errors: INVALID_ARG, UNSUPPORTED, OOM, CUDA. */
BPM_API bpm_status bpm_tune(const bpm_grid* grid, int n_channels, int steps, bpm_launch* best,
                            bpm_launch* all, int max_all, int* n_all);

/* Writes the tuned forms of this process to a text file, one shape per line,
 * tagged with the device name and SM count.  Errors: INVALID_ARG (cannot write). */
BPM_API bpm_status bpm_tune_save(const char* path);

/* Adds the entries of a file written by bpm_tune_save whose device tag matches
 * this GPU (others are skipped); malformed lines are an error.  n_loaded (may
 * be NULL) receives the number of entries taken.  Errors: INVALID_ARG. */
BPM_API bpm_status bpm_tune_load(const char* path, int* n_loaded);

/* Forgets every tuned form of this process. */
BPM_API void bpm_tune_clear(void);

/* Message of the last failed call on this plan (plan = NULL: the last failed
 * bpm_plan_create / batch call of this thread).  Never NULL. */
BPM_API const char* bpm_last_error(bpm_plan plan);

/* Frees the plan and its device memory after its stream has drained.  NULL is a no-op. */
BPM_API void bpm_plan_destroy(bpm_plan plan);

/* Library version string (build tag and target architecture). */
BPM_API const char* bpm_version(void);

/* Device bytes a plan of this grid and channel count allocates (host_u = 1 adds
 * the staging buffer used when bpm_set_crystal receives a host displacement
 * field).  Used for admission by device memory.  0 on invalid input. */
BPM_API size_t bpm_plan_bytes(const bpm_grid* grid, int n_channels, int host_u);

/* ---------------------------------------------------------------------------
 * Batches and continuous batching.  The channels of all plans of a batch are
 * independent stationary problems (Section 3.3: "N stationary tasks"), so one
 * persistent launch marches them together: work items (plan, group of
 * channels) are taken from a device queue, longest first, by blocks that run
 * the resident march of the item's transform size.  Plans keep their fields
 * on the device between rounds.  Batches take 2D plans (dims = 2).
 * ------------------------------------------------------------------------- */
typedef struct bpm_batch_s* bpm_batch;

/* Creates a batch executing on cuda_stream.  hbm_budget_bytes > 0 bounds the
 * sum of bpm_plan_bytes of the admitted, unfinished plans (0 = unbounded).
 * Errors: INVALID_ARG, CUDA. */
BPM_API bpm_status bpm_batch_create(size_t hbm_budget_bytes, void* cuda_stream, bpm_batch* out);

/* Admits a 2D plan whose crystal and pulse are set, of any splitting order (1,
 * 2 or 4); it is marched from its current z to nz by later rounds.  Until its ticket completes (or is cancelled) the
 * plan works on the batch stream (its pending work is ordered before the
 * batch); then its original stream is restored.  The caller keeps ownership
 * and destroys the plan after its ticket reports done (or after cancel).
 * Errors: OOM (budget exhausted: not admitted, retry later), STATE (no pulse,
 * already admitted), UNSUPPORTED (3D plan), INVALID_ARG. */
BPM_API bpm_status bpm_batch_submit(bpm_batch b, bpm_plan plan, uint64_t* ticket);

/* Enqueues one round: every admitted, unfinished plan advances
 * min(chunk_steps, nz - z) steps in one persistent launch (plus a sibling
 * launch for Nx = 8192 on a forked stream); plans that reach nz then get their
 * reflectivity and time response and a completion event.  Asynchronous.
 * Plans admitted after this call join the next round (continuous batching).
 * Errors: INVALID_ARG, CUDA. */
BPM_API bpm_status bpm_batch_step(bpm_batch b, int chunk_steps);

/* One round that takes every admitted plan to nz (a single persistent launch
 * per queue).  Asynchronous. */
BPM_API bpm_status bpm_batch_run(bpm_batch b);

/* Runs the whole hot path of every admitted plan as one CUDA graph: the
 * deformation factor, tables and incident field from the inputs stored by
 * bpm_set_crystal / bpm_set_pulse (device pointers must still be valid), one
 * round to nz and the time responses.  Captured on first use and whenever the
 * set of plans changes, replayed otherwise.  Asynchronous. */
BPM_API bpm_status bpm_batch_run_graph(bpm_batch b);

/* Kernel launches in one replay of the graph bpm_batch_run_graph captured
 * (0 before the first capture).  Errors: INVALID_ARG. */
BPM_API bpm_status bpm_batch_graph_kernels(bpm_batch b, int* kernels);

/* Non-blocking completion test of a ticket; done = 1 once its results can be
 * fetched from its plan (the plan's budget share is then released).
 * Errors: CANCELLED, INVALID_ARG (unknown ticket), CUDA. */
BPM_API bpm_status bpm_batch_poll(bpm_batch b, uint64_t ticket, int* done);

/* Removes an unfinished plan from later rounds (waits for rounds already
 * enqueued).  Errors: STATE (already finishing), INVALID_ARG. */
BPM_API bpm_status bpm_batch_cancel(bpm_batch b, uint64_t ticket);

/* Waits for all enqueued rounds.  Errors: INVALID_ARG (null batch), CUDA (a
 * round's kernels failed). */
BPM_API bpm_status bpm_batch_sync(bpm_batch b);

/* Number of enqueued rounds whose kernels have not finished (0..3).  A step
 * while 3 rounds are in flight waits for the oldest on the host; a caller that
 * must not block (a server feeding several batches) steps only below 3.
 * Errors: INVALID_ARG, CUDA (a round's kernels failed). */
BPM_API bpm_status bpm_batch_pending(bpm_batch b, int* rounds_in_flight);

/* Caps the persistent launches of later rounds at max_blocks blocks (one per
 * SM; <= 0 restores every SM).  Two batches on different streams with caps
 * that add up to the SM count run side by side, e.g. a lane for short requests
 * next to a lane for long ones.  Errors: INVALID_ARG. */
BPM_API bpm_status bpm_batch_set_max_blocks(bpm_batch b, int max_blocks);

/* Admitted unfinished plans, their bytes, rounds enqueued so far and the item
 * counts [small, Nx = 8192] of the last round (any pointer may be NULL). */
BPM_API bpm_status bpm_batch_info(bpm_batch b, int* active, size_t* used_bytes, int* rounds,
                                  int* last_items);

/* Message of the last failed call on this batch (NULL: of this thread). */
BPM_API const char* bpm_batch_last_error(bpm_batch b);

/* Waits for the batch stream and frees the batch (not the plans). */
BPM_API void bpm_batch_destroy(bpm_batch b);

/* ---------------------------------------------------------------------------
 * Measured CUDA-core peak (no counterpart in the paper: the denominator of the
 * march kernels' rooflines).  One launch of independent fused multiply-add
 * chains on every SM: kind BPM_PEAK_FP32 (FFMA) or BPM_PEAK_FP64 (DFMA),
 * `iters` loop trips of 128 FMAs per thread (1024 threads per SM).  Writes the
 * achieved rate in flop/s (an FMA counts 2) and the launch's duration by CUDA
 * events on cuda_stream, and waits for the launch.  Allocates nothing.
 * Returns BPM_ERR_INVALID_ARG for a null output, iters < 1 or an unknown
 * kind, BPM_ERR_UNSUPPORTED without a GB300, BPM_ERR_CUDA if the launch fails.
 * ------------------------------------------------------------------------- */
#define BPM_PEAK_FP32 0
#define BPM_PEAK_FP64 1
BPM_API bpm_status bpm_measure_peak(int kind, int iters, double* flop_per_s, float* ms,
                                    void* cuda_stream);

/* ---------------------------------------------------------------------------
 * Check of the failure path of the kernels that wait on bulk copies (no
 * counterpart in the paper).  Those waits are bounded: after a limit of polls
 * the waiting threads record a status that bpm_sync reports as
 * BPM_ERR_TIMEOUT, instead of spinning forever.  This call makes such a wait
 * run out on purpose, without any copy in flight: one block's mbarrier
 * expects 16 bytes that nothing delivers, and its threads wait with the same
 * bounded wait at `poll_limit` polls.  *gave_up is set to 1 when the wait gave
 * up and the status was recorded (the expected outcome), 0 otherwise.  The
 * context stays usable.  Synchronous on cuda_stream; allocates nothing.
 * Returns BPM_ERR_INVALID_ARG for a null output or poll_limit < 1,
 * BPM_ERR_UNSUPPORTED without a GB300, BPM_ERR_CUDA if the launch fails.
 * ------------------------------------------------------------------------- */
BPM_API bpm_status bpm_check_bounded_wait(int poll_limit, int* gave_up, void* cuda_stream);

/* ---------------------------------------------------------------------------
 * Allocation-free single-instance run.  The paper has no counterpart: this is
 * a deployment convenience of this library.
 *
 * For callers that cannot allocate device memory while they run this code:
 * processes whose device memory is wholly handed out by their own pool (a
 * cudaMalloc there fails or steals memory the pool has promised elsewhere),
 * and latency-bound loops that must not take the allocator's lock or risk
 * fragmenting the heap.  The caller passes the inputs and outputs; every
 * intermediate buffer (deformation factor, propagator tables, coupling
 * coefficients, FFT constants, norms) lives in one fixed device array inside
 * the library (bpm_noalloc_scratch_bytes(), 6.3 MB), which every GPU that
 * loads the library holds until the process exits.  No call here allocates or
 * frees device or pinned memory.
 *
 * Limits (anything larger returns BPM_ERR_UNSUPPORTED and a message in
 * bpm_noalloc_last_error): dims = 2, nx a power of two in [256, 4096],
 * n_channels <= 16, nz * nx <= 524288 cells.
 *
 * Results equal those of a plan created with the same inputs followed by
 * bpm_run(nz): E0 and Eh at z = nz into e0_dev / eh_dev (device complex64
 * [n_channels][nx]), reflectivities R_i into refl_dev (device float64
 * [n_channels]).  u_field_dev is a device float64 [nz][nx] displacement or
 * NULL (perfect crystal); omega and weight_re_im are host arrays as for
 * bpm_set_pulse.  Asynchronous on cuda_stream, except that omega,
 * weight_re_im and the FFT constants are copied into the array with
 * cudaMemcpyAsync from pageable host memory, which the CUDA runtime stages
 * before the call returns.  The call takes no sizes for the
 * caller's buffers: they must hold at least the sizes above (the Python
 * binding checks them).
 *
 * The first call on a device looks up the array's device address (with that
 * device current); make that first call before any stream capture.  All calls
 * share the one array and it keeps the last call's contents: two calls whose
 * work overlaps on the GPU (different streams, or different host threads)
 * race and corrupt each other, so serialise them on one stream.
 * ------------------------------------------------------------------------- */
typedef struct {
  double chi0_re, chi0_im, chih_re, chih_im, chihbar_re, chihbar_im;
  double theta_B, lambda_B, x_surface, thickness;
} bpm_crystal_params;

typedef struct {
  double theta_i, x0, w0, zx, zR;
} bpm_beam_params;

BPM_API bpm_status bpm_run_noalloc(const bpm_grid* grid, int n_channels,
                                   const bpm_crystal_params* crystal, const double* u_field_dev,
                                   const double* omega, const double* weight_re_im,
                                   const bpm_beam_params* beam, void* e0_dev, void* eh_dev,
                                   double* refl_dev, void* cuda_stream);

/* Size in bytes of the fixed device array used by bpm_run_noalloc. */
BPM_API size_t bpm_noalloc_scratch_bytes(void);

/* Message of the last failed bpm_run_noalloc call of this thread. */
BPM_API const char* bpm_noalloc_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* BPM_H_ */
