/*
 * agnlc.h -- C ABI of the GB300 light-curve generator.
 *
 * The library generates batches of AGN Eddington-ratio light curves with a
 * prescribed power spectral density (bending power law, Sec. 2.1.2, Eq. 3) and
 * a prescribed probability density (the Eddington-ratio distribution function,
 * ERDF, Sec. 2.1.1) by the method of Sec. 2.1 of Sartori et al. (2019):
 *   1. a Timmer & Koenig (TK95) Gaussian realisation of the PSD;
 *   2. a random draw of N values from the ERDF (here by inverse CDF);
 *   3. iterative amplitude adjustment (Schreiber & Schmitz 1996 /
 *      Emmanoulopoulos et al. 2013, Sec. 3.2.2): forward FFT, target
 *      amplitudes with the phases kept, inverse FFT, rank-order replacement by
 *      the sorted draws.
 *
 * Conventions shared by every entry point
 *   - Plain C types only; no exceptions cross the boundary; every call returns
 *     an lc_status (0 = LC_OK, negative = error).  Arguments are validated
 *     before any device work is queued; an invalid call changes nothing.
 *   - "device pointer" means memory of the plan's CUDA device (cudaMalloc,
 *     torch, ...); "host pointer" means ordinary or pinned host memory.
 *   - The caller owns every output buffer.  The library owns its plans and
 *     servers and the device workspaces they allocate.
 *   - Streams are passed as `void*` holding a cudaStream_t (NULL = legacy
 *     default stream).  Calls are asynchronous with respect to the host
 *     unless stated otherwise; work is ordered after everything queued on the
 *     stream before the call, and later work on that stream sees the results.
 *   - A series of N = 2^log2n samples is stored contiguously, sample k at time
 *     t_k = k * dt.  A batch is the concatenation of its curves in job order
 *     (curve c starts at sum_{c' < c} N_{c'}).  Element type: float for
 *     LC_FP32, double for LC_FP64.
 *   - Results are deterministic functions of (job, precision): the same job
 *     gives the same bits alone, in any batch, and in the server.
 */
#ifndef AGNLC_H
#define AGNLC_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define LC_API __attribute__((visibility("default")))
#else
#define LC_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    LC_OK = 0,
    LC_PENDING = 1,             /* lc_poll: the job has not finished yet          */
    LC_ERR_INVALID = -1,        /* an argument or job parameter is out of range   */
    LC_ERR_NOMEM = -2,          /* a device or host allocation failed             */
    LC_ERR_CUDA = -3,           /* a CUDA call failed (message: lc_last_error)    */
    LC_ERR_TIMEOUT = -4,        /* a bounded device wait gave up                  */
    LC_ERR_BUSY = -5,           /* lc_submit: the admission queue is full         */
    LC_ERR_UNKNOWN_TICKET = -6  /* lc_poll: no such ticket (or already collected)  */
} lc_status;

typedef enum { LC_FP32 = 0, LC_FP64 = 1 } lc_precision;

/* PSD of Eq. 3 with A = 1: P(f) = [(f/f_br)^alpha_low + (f/f_br)^alpha_high]^-1.
 * f_br is in inverse units of dt (e.g. day^-1 when dt is in days); the PSD
 * falls as f^-alpha_low below and f^-alpha_high above the break.  Equal
 * slopes give the single power law (f/f_br)^-alpha / 2 (Sec. 3.1).
 *   coeffs:  LC_TK_GAUSSIAN (0): TK95 coefficients, Re and Im Gaussian with
 *            variance P_j/2 (the periodogram scatters around the PSD);
 *            LC_TK_FIXED_AMPLITUDE (1): |X_j| = sqrt(P_j) with a uniform
 *            random phase (same mean power, no scatter).
 *   targets: LC_TARGETS_REALISED (0): the iteration imposes the amplitudes of
 *            the realised TK series (E13); LC_TARGETS_PSD (1): the amplitudes
 *            of the PSD itself, sqrt(P_j) normalised to unit variance. */
typedef enum { LC_TK_GAUSSIAN = 0, LC_TK_FIXED_AMPLITUDE = 1 } lc_tk_coeffs;
typedef enum { LC_TARGETS_REALISED = 0, LC_TARGETS_PSD = 1 } lc_targets;

typedef struct {
    double f_br;
    double alpha_low;
    double alpha_high;
    int32_t coeffs;        /* lc_tk_coeffs  */
    int32_t targets;       /* lc_targets    */
} lc_psd;

/* Shape of the ERDF (Sec. 2.1.1). */
typedef enum {
    LC_ERDF_SHARP = 0,     /* broken power law with a sharp break (closed-form inverse CDF) */
    LC_ERDF_SMOOTH = 1,    /* the smooth broken power law of Eq. 1 (tabulated CDF)          */
    LC_ERDF_LOGNORMAL = 2  /* the log-normal of Eq. 2 (tabulated CDF)                        */
} lc_erdf_kind;

/* ERDF on u = log10(lambda) in [log_lmin, log_lmax], with d = u - log_lbreak:
 *   LC_ERDF_SHARP:     dN/du ~ 10^(slope_low d) for d < 0, 10^(slope_high d) above;
 *   LC_ERDF_SMOOTH:    dN/du ~ [10^(-slope_low d) + 10^(-slope_high d)]^-1, i.e.
 *                      Eq. 1 with log lambda* = log_lbreak, delta_1 = -slope_low,
 *                      delta_2 = -slope_high (W17: -0.47, -2.53);
 *   LC_ERDF_LOGNORMAL: dN/du ~ exp(-d^2 / (2 sigma^2)), i.e. Eq. 2 with
 *                      log lambda* = log_lbreak and sigma-tilde = sigma (dex).
 * linear_space != 0 reads the shape as dN/dlambda instead (the linear sampling
 * of Sec. 2.1.1): the density in u gains a factor 10^d (for the power laws
 * both slopes rise by one).  The sharp form is inverted in closed form; the
 * other two through an FP64 table of their CDF (4096 intervals of Simpson's
 * rule, bisection and linear interpolation, inverse error < 1e-6 dex), with
 * the same bits on the GPU and in any IEEE-754 reimplementation that follows
 * the same operation order.  Zero-initialised fields give the sharp form. */
typedef struct {
    double log_lmin;
    double log_lmax;
    double log_lbreak;
    double slope_low;
    double slope_high;
    int32_t linear_space;
    int32_t kind;          /* lc_erdf_kind */
    double sigma;          /* LC_ERDF_LOGNORMAL width in dex; unused otherwise */
} lc_erdf;

/* One light curve (the inputs of Sec. 3.2.4: t_bin = dt, N_steps = 2^log2n).
 * seed and curve_id key the counter-based random streams; two jobs with the
 * same (seed, curve_id) draw the same random numbers. */
typedef struct {
    uint32_t log2n;      /* 4 <= log2n <= 27 (N up to 2^27, Sec. 3.2.3)         */
    uint32_t iters;      /* number of amplitude-adjustment iterations, >= 0     */
    double dt;           /* sampling interval, > 0                              */
    lc_psd psd;
    lc_erdf erdf;
    uint64_t seed;
    uint64_t curve_id;
} lc_job;

typedef struct lc_plan_s* lc_plan;
typedef struct lc_server_s* lc_server;
typedef uint64_t lc_ticket;

/* Human-readable name of a status code (static storage). */
LC_API const char* lc_status_string(lc_status status);

/* Text of the most recent error raised on the calling thread (static per
 * thread; empty string if none). */
LC_API const char* lc_last_error(void);

/* ---------------------------------------------------------------- batches */

/* Validate `njobs` jobs and build a plan for them on CUDA device `device`:
 * the ragged layout, twiddle tables and every device workspace the batch
 * needs (allocated here, owned by the plan).  jobs: host array, read only
 * during the call.  Validation: njobs >= 1, 4 <= log2n <= 27, dt > 0,
 * f_br > 0, finite slopes, -300 <= log_lmin < log_lmax <= 300; for the power
 * laws log_lmin < log_lbreak < log_lmax and |slope| <= 50; for the log-normal
 * sigma >= (log_lmax - log_lmin)/1024 and the centre log_lbreak within 30
 * sigma of the range; otherwise LC_ERR_INVALID.  LC_ERR_NOMEM if the
 * workspace does not fit.  Blocking. */
LC_API lc_status lc_plan_create(const lc_job* jobs, size_t njobs, lc_precision prec, int device,
                         lc_plan* out);

/* Device bytes the plan holds (workspace + tables). */
LC_API lc_status lc_plan_workspace_bytes(lc_plan plan, size_t* bytes);

/* Total samples sum_c N_c of the batch (the length of out_x). */
LC_API lc_status lc_plan_total_samples(lc_plan plan, size_t* samples);

/* The whole generator (Sec. 2.1): TK95 realisation, ERDF draws, then each
 * job's `iters` iterations.  out_x: device pointer, sum_c N_c elements, the
 * final series.  out_tk: device pointer or NULL; when given it receives the
 * normalised TK95 series (zero mean, unit variance) of every curve. */
LC_API lc_status lc_generate(lc_plan plan, void* out_x, void* out_tk, void* stream);

/* As lc_generate, but out_x / out_tk are HOST pointers (pinned memory is
 * fastest); the device-to-host copies are part of the call, which returns
 * after they have completed (blocking). */
LC_API lc_status lc_generate_host(lc_plan plan, void* out_x_host, void* out_tk_host, void* stream);

/* Setup only (steps 1-2 of Sec. 2.1): computes the target amplitudes, the
 * sorted draws and the initial state (the draws in draw order) inside the
 * plan; out_tk as in lc_generate. */
LC_API lc_status lc_setup(lc_plan plan, void* out_tk, void* stream);

/* Run amplitude-adjustment iterations (Sec. 3.2.2) on the plan's current
 * state.  iters = 0 runs each job's own count; iters > 0 runs exactly that
 * many on every curve.  Requires a previous lc_setup or lc_generate. */
LC_API lc_status lc_iterate(lc_plan plan, uint32_t iters, void* stream);

/* Copy the plan's current state (sum_c N_c elements) to / from a device
 * buffer.  lc_set_state lets a caller iterate from a state of its own; the
 * values must then be a permutation of each curve's draws for the output to
 * keep the ERDF exactly. */
LC_API lc_status lc_get_state(lc_plan plan, void* out_x, void* stream);
LC_API lc_status lc_set_state(lc_plan plan, const void* in_x, void* stream);

/* The rank-order replacement step of one iteration on its own (Sec. 2.1,
 * third step; Sec. 3.2.2: the values stay the sorted draws, only their order
 * changes): for every curve c, out_x[perm_c[r]] = s_c[r] for r < N_c, where
 * s_c are the curve's sorted draws and perm_c the stable ascending argsort of
 * x_adj's curve c (ties, -0 = +0 included, keep the lower position first).
 * The plan's own sort path runs (the sample sort of FP32 curves of 2^13 ..
 * 2^20 samples, else the LSD radix passes).
 *   x_adj: device pointer, sum_c N_c elements in the plan's precision and
 *          layout (curve c at the offset of lc_get_state); read only; values
 *          must not be NaN.
 *   out_x: device pointer, same size and layout (caller-owned); may be x_adj.
 * Requires lc_setup or lc_generate before (for s); the plan's state is not
 * touched.  Asynchronous on `stream`. */
LC_API lc_status lc_rank_replace(lc_plan plan, const void* x_adj, void* out_x, void* stream);

/* Read-only view of a plan buffer, valid until lc_plan_destroy:
 * which = 0: state x (sum N elements); 1: target amplitudes A
 * (sum (N/2+1) elements, curve c at sum_{c'<c} (N_{c'}/2+1)); 2: sorted
 * draws s (sum N elements). */
LC_API lc_status lc_plan_buffer(lc_plan plan, int which, const void** device_ptr, size_t* bytes);

/* Number of kernel launches the most recent lc_generate/lc_iterate queued
 * (graph replays count their kernels). */
LC_API lc_status lc_plan_last_launches(lc_plan plan, uint64_t* launches);

/* Device time of the last lc_generate / lc_generate_host / lc_setup +
 * lc_iterate, split into the setup stage and the iteration stage, measured
 * with CUDA events on the plan's stream (blocks until both are known).
 * A stage that did not run reports 0. */
LC_API lc_status lc_plan_timing(lc_plan plan, float* setup_ms, float* iterate_ms);

/* ------------------------------------------------------------ convergence */

/* Turn on the convergence test of Sec. 3.2.2 (Eq. 4) for the plan's later
 * lc_generate / lc_generate_host / lc_iterate runs.  After each iteration i
 * (1-based) every running curve computes
 *     delta_i = rms_n [ log10( x_i(t_n) / x_{i-1}(t_n) ) ],  n = 1..N,
 * the root mean square about zero of the base-10 log ratio between its
 * consecutive iterates (x_0 = the state the run starts from, after lc_setup
 * the draws in draw order), records it, and stops when delta_i is strictly
 * below its threshold: its remaining iterations of that run are skipped and
 * its series stays x_i.  The record is reset at the start of every run.
 *   thresholds: host array of ncurves doubles (job order), read during the
 *               call; NULL = all 0.  A threshold <= 0 never stops its curve
 *               (delta >= 0); +inf stops it after one iteration; NaN is
 *               LC_ERR_INVALID.
 *   history:    1..65536 iterations recorded per curve; later iterations
 *               are still measured and can still stop the curve.
 * The values must be positive (they are for every ERDF); with LC_FP32 a job
 * with log_lmin < -37 is LC_ERR_INVALID (draws below FLT_MIN).  Allocates
 * about ncurves * (history + 2) doubles plus one double per sort tile
 * (owned by the plan) and blocks until done.  Calling it again replaces the
 * thresholds.  Cost per iteration: one extra coalesced pass over the state
 * (the fused kernels write each iterate back to the plan's state buffer; the
 * multi-kernel path reads x_{i-1} and x_i and moves x_i into place). */
LC_API lc_status lc_plan_set_convergence(lc_plan plan, const double* thresholds, uint32_t history);

/* Record of the plan's last run (blocks until the plan's queued work is
 * done).  deltas: host array of ncurves * history doubles or NULL; row c
 * holds delta_1 .. delta_history of curve c, NaN for iterations it did not
 * run.  iters_run: host array of ncurves uint32 or NULL: the iterations each
 * curve ran (its job count, or fewer when it stopped).  LC_ERR_INVALID
 * before lc_plan_set_convergence. */
LC_API lc_status lc_plan_convergence(lc_plan plan, double* deltas, uint32_t* iters_run);

/* ------------------------------------------------------- App. A estimators */

/* Periodogram (App. A, Eq. A2) of every curve of a series laid out like the
 * plan's state: P_j = (2/N^2) |DFT_j|^2 at f_j = j/(N dt), j = 0..N/2; with
 * rms != 0 the fractional rms normalisation of Eq. A4,
 * P_j = 2 dt |DFT_j|^2 / (mu^2 N), mu the curve's mean (a zero-mean curve
 * then gives inf or NaN).  The transform runs in the plan's precision.
 *   x:     device pointer, sum_c N_c elements of the plan's type (float for
 *          LC_FP32, double for LC_FP64), e.g. the out_x of lc_generate; read
 *          only.
 *   out_p: device pointer, sum_c (N_c/2+1) doubles, curve c at
 *          sum_{c'<c} (N_{c'}/2+1) (the layout of the amplitude buffer).
 * Uses the plan's FFT work buffers, so it is ordered with the plan's other
 * calls on the plan's stream (asynchronous like lc_generate). */
LC_API lc_status lc_periodogram(lc_plan plan, const void* x, int rms, double* out_p, void* stream);

/* Structure function (App. A, Eq. A6) of every curve at integer lags:
 * SF(tau)^2 = the mean over the N - tau pairs (x_i, x_{i+tau}) of
 * (x_i - x_{i+tau})^2, i.e. time lag tau * dt of the curve.
 *   x:       device pointer laid out as for lc_periodogram; read only.
 *   lags:    host array of nlags lags in samples, read during the call;
 *            1 <= lag < N of the shortest curve and 1 <= nlags <= 4096,
 *            otherwise LC_ERR_INVALID.
 *   out_sf2: device pointer, ncurves * nlags doubles, row c (job order)
 *            holds SF^2 of curve c at each lag.
 * Sums in FP64 (runs of 64 squares in the plan's precision first). */
LC_API lc_status lc_structure_function(lc_plan plan, const void* x, const uint32_t* lags, size_t nlags,
                                double* out_sf2, void* stream);

/* Profiling: runs ONE more amplitude-adjustment iteration of every curve on
 * the plan's current state, launched kernel by kernel (not from the captured
 * graph) with CUDA events on the plan's stream around each kernel group, and
 * returns the device milliseconds per group:
 *   group_ms[0] transforms and spectral step (multi-kernel path),
 *   group_ms[1] sort histograms and scans (sample sort: sample, histogram
 *   and scan kernels), group_ms[2] sort scatter passes (sample sort: bucket
 *   scatter and on-chip finish), group_ms[3] fused on-chip kernels,
 *   group_ms[4] convergence test.
 * ngroups: entries of group_ms to fill (extra ones get 0).
 * counts (nullable, 4 entries): scatter spans timed (one per radix pass of
 * each radix-sorted class, one per sample-sorted class), samples of the
 * multi-kernel classes, samples of the fused classes, samples of the
 * multi-kernel classes whose argsort is the sample sort.
 * The state advances by one iteration; the iteration counter restarts, so a
 * later lc_iterate(plan, 0) runs each job's count again.  Blocking. */
LC_API lc_status lc_plan_profile(lc_plan plan, float* group_ms, size_t ngroups, uint64_t* counts);

/* Release the plan and its device memory (synchronises its stream). */
LC_API lc_status lc_plan_destroy(lc_plan plan);

/* ------------------------------------------------------- no allocation */

/* Whole generator for ONE FP32 curve without allocating any device memory.
 * There is no counterpart in the paper: this entry point exists for callers
 * that cannot call cudaMalloc -- hosts whose device memory belongs to another
 * allocator (a framework's caching allocator or an accounted memory pool), and
 * real-time or serving loops that must not allocate after start-up, since a
 * cudaMalloc can synchronise the device.  It runs the same kernels as
 * lc_generate on a one-curve plan whose buffers all live in a 4 MiB
 * file-scope device array of the library (held by every device that loads
 * the library until the process exits).
 *   job:    host pointer, read during the call; log2n must be <= 16 (larger
 *           curves do not fit the array: LC_ERR_INVALID with a message).
 *   out_x:  device pointer, 2^log2n floats, the final series (caller-owned).
 *   stream: cudaStream_t (NULL = legacy default stream) of the current device.
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current and sets the kernels'
 * shared-memory limits; make that first call before any stream capture.  The
 * job's descriptor reaches the device as kernel arguments, so no host memory
 * is read after the call returns.  Every call reuses the same array and leaves its
 * contents behind (each call writes every buffer before reading it, so
 * nothing needs clearing); calls whose work overlaps on the GPU, e.g. on two
 * streams, race on the array and must be serialised by the caller. */
LC_API lc_status lc_generate_noalloc(const lc_job* job, void* out_x, void* stream);

/* ---------------------------------------------------------------- serving */

/* A continuous-batching server on `device` (the serving form of Sec. 2.1's
 * generator): jobs submitted at any time are admitted as soon as a slot of
 * the server's device buffers is free for them, run in batched iteration
 * steps alongside the other active jobs, and retired when their iteration
 * count is reached; a retired job's slot is free for the next job at once.
 * At creation the server allocates buffers ("planes") of a power-of-two
 * capacity of C samples in 7/8 of hbm_budget_bytes (state, FFT, draws, sort
 * keys and positions, amplitudes, TK spectrum: about 40 bytes per sample in
 * FP32); every job takes a slot of 2^max(log2n, 4) samples.  Jobs are
 * admitted in arrival order, skipping one whose slot cannot be allocated yet
 * unless it has waited for more than a second, after which no later job is
 * admitted before it.  A host thread owned by the server drives the device.
 * hbm_budget_bytes = 0 uses 80 % of the free device memory; LC_ERR_INVALID if
 * the budget holds no slot of 16 samples, LC_ERR_NOMEM if the planes cannot
 * be allocated. */
LC_API lc_status lc_server_create(int device, size_t hbm_budget_bytes, lc_precision prec,
                           lc_server* out);

/* Queue one job (copied; non-blocking).  LC_ERR_BUSY if the queue is full,
 * LC_ERR_INVALID for a bad job or one longer than the server's capacity. */
LC_API lc_status lc_submit(lc_server server, const lc_job* job, lc_ticket* out);

/* Non-blocking completion check.  LC_PENDING while the job runs; LC_OK when
 * it has finished, after copying its N results into out (host pointer) and
 * the submit-to-finish latency into *latency_ns (either may be NULL); the
 * ticket is then released.  A job whose cohort failed returns that error
 * once (LC_ERR_NOMEM when its cohort's tables could not be allocated with no
 * other cohort running, LC_ERR_CUDA otherwise) and the server keeps serving;
 * LC_ERR_CUDA for every ticket only after an error that leaves the CUDA
 * context unusable.  LC_ERR_UNKNOWN_TICKET otherwise. */
LC_API lc_status lc_poll(lc_server server, lc_ticket ticket, void* out_host, uint64_t* latency_ns);

/* Jobs finished, jobs active on the device, jobs waiting for admission. */
LC_API lc_status lc_server_stats(lc_server server, uint64_t* finished, uint64_t* active,
                          uint64_t* waiting);

/* Device-time record of the server's chunks (CUDA events on the cohorts'
 * streams, up to 65536 chunks): *busy_ms = time with at least one chunk on
 * the device, *overlap_ms = time with chunks of two or more cohorts running
 * at once; *free_samples / *capacity = free and total samples of the planes.
 * Any pointer may be NULL. */
LC_API lc_status lc_server_trace(lc_server server, double* busy_ms, double* overlap_ms, uint64_t* free_samples,
                                 uint64_t* capacity);

/* Stop the server thread, drop unfinished jobs and free its memory. */
LC_API lc_status lc_server_destroy(lc_server server);

/* Device bytes that lc_plan_create allocates for these jobs (the value
 * lc_plan_workspace_bytes then reports), computed on the host from the same
 * layout without any device call.  LC_ERR_INVALID as lc_plan_create for bad
 * jobs. */
LC_API lc_status lc_plan_footprint(const lc_job* jobs, size_t njobs, lc_precision prec, size_t* bytes);

#ifdef __cplusplus
}
#endif

#endif /* AGNLC_H */
