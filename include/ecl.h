/*
 * ecl.h -- C ABI of the GB300 package-scheduling engine.
 *
 * The calls restate the programming interface of EngineCL (Nozal, Bosque,
 * Beivide, "EngineCL: Usability and Performance in Heterogeneous
 * Computing", Sec. 6, Listings 1 and 2): an engine owns the work size, the
 * scheduler and a program; a program owns its input and output buffers, a
 * kernel, the kernel's arguments and an output pattern; run() executes the
 * whole NDRange and the engine can report per-package statistics.
 *
 * On one GB300 the paper's "devices" are groups of persistent CTAs.  D
 * devices of C CTAs each pull packages of work-groups from a package queue
 * in device memory; the package sizes follow the paper's Static, Dynamic and
 * HGuided rules (Sec. 5.3).  A package handed to a device is split into
 * chunks that the device's C CTAs claim one at a time.
 *
 * Conventions for every call:
 *  - Pointers are plain host or device addresses; sizes are in bytes unless
 *    stated.  No call takes or returns a framework type.
 *  - Every call returns an ecl_status.  Errors are never thrown and never
 *    end the process.  An engine counts its errors and keeps the text of
 *    the most recent one for ecl_last_error() (the has_errors/get_errors
 *    analogue of Listing 1).  A NULL handle gives ECL_ERR_ARG.
 *  - The caller owns every buffer it registers; the engine owns the
 *    programs given to it, its package table, queue and statistics memory,
 *    and the device mirrors it makes for host buffers.
 *  - Not thread-safe per engine: one host thread drives one engine.
 */
#ifndef ECL_H
#define ECL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ecl_engine ecl_engine;
typedef struct ecl_program ecl_program;

typedef enum ecl_status {
    ECL_OK = 0,
    ECL_ERR_ARG = 1,     /* bad argument: NULL handle, unknown index, wrong size */
    ECL_ERR_SIZE = 2,    /* work size: gws == 0, gws % lws != 0, lws not allowed */
    ECL_ERR_BUFFER = 3,  /* buffer missing, too small, or not registered */
    ECL_ERR_SCHED = 4,   /* scheduler parameters out of range */
    ECL_ERR_KERNEL = 5,  /* unknown kernel name */
    ECL_ERR_CUDA = 6,    /* a CUDA runtime call failed (text names it) */
    ECL_ERR_TIMEOUT = 7, /* a bounded device-side wait gave up (the run is void) */
    ECL_ERR_STATE = 8    /* call out of order: no program, no work size, ... */
} ecl_status;

/* Schedulers of Sec. 5.3 and Sec. 7.3, plus the plain-grid baseline.
 *  ECL_STATIC      params: D-1 (or D) proportions; device d < D-1 gets
 *                  floor(prop_d * U) units, the last device the rest; no
 *                  params = equal split.  One package per device.  With
 *                  D = 1 the single package [0, G) runs as one grid, one
 *                  CTA per chunk (nothing is left to schedule at run time;
 *                  the kernels with their own claim loop, the GEMMs, keep
 *                  the queue); its package record has t0 = chunk 0's start,
 *                  and there is one worker record per CTA.
 *  ECL_STATIC_REV  same sizes, ranges laid out in reverse device order
 *                  (Sec. 7.3 "Static rev").
 *  ECL_DYNAMIC     params: {num_packages}; equal packages of
 *                  ceil(U / num_packages) units, the last one shorter.
 *  ECL_HGUIDED     params: {k, min_package, P_1 .. P_D}; package for device i
 *                  = floor(G_r P_i / (k n sum_j P_j)) units (the HGuided
 *                  equation, n = D), at least that device's minimum
 *                  max(1, floor(min_package P_i / min_j P_j + 0.5)) and at
 *                  most G_r.  Powers are optional (equal when omitted).
 *                  Defaults k = 2, min_package = 1.
 *  ECL_MONOLITHIC  no package queue: one CTA per fixed block of
 *                  work-groups, like a plain native launch; the reference
 *                  point of the overhead metric (Sec. 7.3).
 * U = number of scheduling units = ceil(G / grain); grain is 1 work-group
 * except for the row-tiled GEMM, whose unit is one row of output tiles. */
typedef enum ecl_sched_kind {
    ECL_STATIC = 0,
    ECL_STATIC_REV = 1,
    ECL_DYNAMIC = 2,
    ECL_HGUIDED = 3,
    ECL_MONOLITHIC = 4
} ecl_sched_kind;

/* One record per package handed out (the Introspector of Sec. 5.2, Figs 5-6).
 * Times are the GPU global timer in ns.  t0 = when the package was taken
 * from the queue, t1 = when the last of its chunks finished. */
typedef struct ecl_pkg_stat {
    uint64_t off_wg;  /* first work-group of the package */
    uint64_t len_wg;  /* number of work-groups */
    uint64_t t0_ns;
    uint64_t t1_ns;
    uint32_t pkg;     /* package index in hand-out order */
    uint32_t device;  /* device (CTA group) that took it */
    uint32_t cta;     /* CTA that took it from the queue */
    uint32_t smid;    /* SM of that CTA */
} ecl_pkg_stat;

/* One record per persistent CTA (per CTA of the grid when Static runs over
 * one device). */
typedef struct ecl_worker_stat {
    uint64_t t_first_ns; /* start of its first chunk (0 if it got none) */
    uint64_t t_last_ns;  /* end of its last chunk */
    uint64_t busy_ns;    /* sum of its chunk durations */
    uint32_t cta;
    uint32_t device;
    uint32_t smid;
    uint32_t chunks;     /* chunks it computed */
} ecl_worker_stat;

/* One batch of "binomial_batch" (80 bytes, the layout of the device table). */
typedef struct ecl_binomial_instance {
    const float *S, *K, *T, *sigma; /* device arrays of n values */
    const int32_t *steps;           /* device int32[n], 1..2048 */
    float *price;                   /* device float[n] */
    float *greeks;                  /* device float2[n] (delta, vega) or NULL */
    int64_t first;                  /* first option of this batch in the NDRange */
    int64_t n;                      /* options in this batch */
    float r;                        /* risk-free rate */
    int32_t pad;
} ecl_binomial_instance;

/* One view of "mandelbrot_batch" (56 bytes, the layout of the device table). */
typedef struct ecl_mandelbrot_view {
    uint32_t *out;                  /* device uint32[W*H], 16-byte aligned */
    int32_t W, H;                   /* pixels */
    float x0, y0, dx, dy;           /* pixel (i, j) -> c = (x0 + i dx, y0 + j dy) */
    int32_t max_iter;
    int32_t pad;
    int64_t first;                  /* first work-group of this view in the NDRange */
    int64_t wgs;                    /* its work-groups: ceil(W*H / 4 / 256) */
} ecl_mandelbrot_view;

/* One image of "gaussian_batch" (48 bytes, the layout of the device table). */
typedef struct ecl_gaussian_image {
    const float *in;                /* device float[W*H] row-major */
    float *out;                     /* device float[W*H], 16-byte aligned */
    const float *w;                 /* device float[31] filter weights */
    int32_t W, H;
    int64_t first;                  /* first work-group (tile) of this image in the NDRange */
    int64_t tiles;                  /* its tiles: ceil(H/32) * ceil(W/224) */
} ecl_gaussian_image;

/* ---------------------------------------------------------------- engine */

/* Creates an engine on CUDA device `device_ordinal` (Sec. 6 and Listing 1:
 * the engine manages the devices, the work sizes, the scheduler and the
 * execution statistics; `engine.use(...)` picks the devices, here one GPU
 * whose CTAs are split into devices by ecl_workers).  `cuda_stream` is a
 * cudaStream_t (NULL = the legacy default stream); every launch and copy
 * of the engine is ordered on it.  Allocates the queue and statistics
 * memory.  Errors: ECL_ERR_ARG (e NULL), ECL_ERR_CUDA. */
ecl_status ecl_engine_create(ecl_engine **e, int device_ordinal, void *cuda_stream);

/* Waits for the engine's stream, then frees the engine, its programs and
 * its device memory (the end of the engine's scope in Listings 1 and 2,
 * where the engine owns the program it was given).  NULL is ignored. */
void ecl_engine_destroy(ecl_engine *e);

/* Replaces the stream used by later calls. */
ecl_status ecl_engine_set_stream(ecl_engine *e, void *cuda_stream);

/* Copy streams for host buffers (the asynchronous enqueueing and event
 * chaining of Sec. 5.1, for the copies of the Buffer proxy of Sec. 4.2).
 * With them set, a run of a program with host buffers issues the copies in
 * on `h2d_stream` and the copies out on `d2h_stream` (NULL = the engine's
 * stream), ordered around the launch by events: the launch waits for the
 * copies in, the copies out wait for the launch, and the next run's copies
 * in wait for this run's launch (its kernel reads the device mirrors) and
 * its launch for this run's copies out.  async != 0: ecl_run returns once
 * everything is enqueued, without waiting; ecl_synchronize (or ecl_stats)
 * waits for the copies out and reports device errors.  So runs of several
 * engines, each with its own host buffers, overlap one engine's copies with
 * another's computation when the host memory is page-locked.  async == 0
 * keeps the synchronous run of Listing 1.  Errors: ECL_ERR_ARG, ECL_ERR_CUDA. */
ecl_status ecl_engine_copy_streams(ecl_engine *e, void *h2d_stream, void *d2h_stream, int async);

/* Time of a run's main kernel, for the Introspector's per-execution timings
 * (Sec. 5.2) and the time measurements of Sec. 7.3.  With two CUDA events
 * set (cudaEvent_t passed as void *, created by the caller with timing,
 * owned by the caller, NULL and NULL to clear), every later run records
 * `begin` on the engine's stream right before the program's main kernel and
 * `end` right after it: a pass before it (the split GEMMs' operand split)
 * or after it (the binomial's greeks pass) falls outside.  The events are
 * not synchronised; read them with cudaEventElapsedTime once the run is
 * complete.  Errors: ECL_ERR_ARG if only one of the two is NULL. */
ecl_status ecl_engine_kernel_events(ecl_engine *e, void *begin, void *end);

/* Global and local work size (Listing 2 "work_items"; Listing 1 sets them
 * one at a time).  gws must be a positive multiple of lws; each kernel
 * also restricts lws (see the kernel list below).  G = gws / lws. */
ecl_status ecl_work_items(ecl_engine *e, uint64_t gws, uint32_t lws);

/* Scheduler and its parameters (Sec. 5.3; see ecl_sched_kind).  The
 * parameters are copied.  Errors: ECL_ERR_SCHED for an unknown kind or
 * out-of-range parameters (checked again at run time against D and G). */
ecl_status ecl_scheduler(ecl_engine *e, ecl_sched_kind kind, const double *params, int nparams);

/* Number of devices D and CTAs per device C (Sec. 4.2 Device module and
 * Listing 2's engine.use(ecl::Device(...), ...): the devices that share
 * the NDRange; Sec. 5.1: one thread drives each device, here a group of
 * C persistent CTAs takes that role).  0 = automatic: for most
 * kernels C = 1 and D = every CTA that fits on the GPU at once; for the
 * GEMM D = 4 groups sharing the SMs.  D*C beyond what is resident at
 * once is allowed (the queue never waits for a CTA that has not started)
 * up to 64 times the resident count (ECL_ERR_SIZE above that). */
ecl_status ecl_workers(ecl_engine *e, int devices, int ctas_per_device);

/* Gives the program to the engine, which owns it from then on (the
 * std::move of Listing 1).  A program already owned by an engine gives
 * ECL_ERR_STATE.  A previous program of the engine is destroyed. */
ecl_status ecl_engine_program(ecl_engine *e, ecl_program *p);

/* Executes the whole NDRange once: validates, plans the packages,
 * then makes ONE launch on the engine's stream (persistent CTAs pulling
 * packages; a plain grid for Static over one device).  With device
 * buffers only, it returns without waiting (use ecl_synchronize).  If the
 * program registered host buffers, inputs are copied to device mirrors
 * before the launch and outputs copied back after it, and the call waits
 * for the stream, so the host containers hold the results on return
 * (the synchronous run of Listing 1).  Errors: ECL_ERR_STATE, ECL_ERR_SIZE, ECL_ERR_BUFFER,
 * ECL_ERR_SCHED, ECL_ERR_CUDA, and ECL_ERR_TIMEOUT reported by the next
 * synchronising call. */
ecl_status ecl_run(ecl_engine *e);

/* Waits for the engine's stream and reports a device-side failure of the
 * last run (ECL_ERR_TIMEOUT when a bounded wait gave up). */
ecl_status ecl_synchronize(ecl_engine *e);

/* Copies up to `cap` package records of the last run into `out` (host
 * memory), in hand-out order, and stores the count in *n (the data the
 * paper's Introspector module extracts from a run, Sec. 5.3's figure of
 * packages per scheduler; Sec. 7.3 derives balance from the devices'
 * finish times).  Synchronises.
 * Monolithic runs have no packages (*n = 0). */
ecl_status ecl_stats(ecl_engine *e, ecl_pkg_stat *out, size_t cap, size_t *n);

/* Copies up to `cap` per-CTA records of the last run (host memory). */
ecl_status ecl_worker_stats(ecl_engine *e, ecl_worker_stat *out, size_t cap, size_t *n);

/* Debug aid: when `counts` (device memory, `n` uint32 entries, n >= G) is
 * set, every run adds 1 to counts[w] for each work-group w it computes,
 * so a caller can check that every work-group ran exactly once.  NULL
 * turns it off.  The caller zeroes and owns the array. */
ecl_status ecl_set_coverage(ecl_engine *e, uint32_t *counts, uint64_t n);

/* Debug and fault-injection knobs (not in the paper; for tests of the
 * failure path, which must not need a GPU fault).
 *   ECL_DEBUG_SPIN_LIMIT  value = polls (about 128 ns apart) a CTA waiting
 *                         for its device's next package makes before it
 *                         gives up with ECL_ERR_TIMEOUT; 0 restores the
 *                         default of 20,000,000.
 *   ECL_DEBUG_WITHHOLD    value != 0: the CTA that fetches a device's next
 *                         package (Dynamic / HGuided with more than one CTA
 *                         per device) takes it but never publishes it, so
 *                         the device's other CTAs wait out the spin limit:
 *                         the run ends with ECL_ERR_TIMEOUT at the next
 *                         synchronising call and the engine stays usable.
 * Errors: ECL_ERR_ARG for an unknown kind or a negative value. */
typedef enum { ECL_DEBUG_SPIN_LIMIT = 1, ECL_DEBUG_WITHHOLD = 2 } ecl_debug_kind;
ecl_status ecl_debug(ecl_engine *e, int kind, int64_t value);

/* Plan facts of the last run: G, the number of packages, D, C and the
 * number of CTAs launched.  Any pointer may be NULL. */
ecl_status ecl_plan_info(const ecl_engine *e, uint64_t *G, uint64_t *packages,
                         uint32_t *devices, uint32_t *ctas_per_device, uint32_t *ctas);

/* The package list a run would use, computed on the host without a GPU
 * (Sec. 5.3 rules; see ecl_sched_kind).  Writes up to `cap` packages as
 * (off[i], len[i]) in work-groups, hand-out order, and the total count in
 * *n; device[i] (may be NULL) is the device of a Static package and
 * 0xffffffff for queue packages.  HGuided with unequal powers is cut on
 * the GPU in the order devices ask; here the requests are simulated in
 * device order 0..D-1, cyclic, and device[i] names the asker.  Errors:
 * ECL_ERR_SCHED (text in errbuf when given), ECL_ERR_SIZE when cap is too
 * small (*n still holds the full count), ECL_ERR_ARG. */
ecl_status ecl_plan(ecl_sched_kind kind, const double *params, int nparams, uint64_t G, uint64_t grain,
                    uint32_t devices, uint64_t *off, uint64_t *len, uint32_t *device, size_t cap,
                    size_t *n, char *errbuf, size_t errlen);

/* Text of the most recent error of the engine ("" when none): the
 * has_errors() / get_errors() lines at the end of Listing 1, as a latched
 * message.  The pointer stays valid until the next failing call,
 * ecl_clear_errors or destroy. */
const char *ecl_last_error(const ecl_engine *e);

/* Number of errors seen since creation or the last clear, and clearing. */
int ecl_error_count(const ecl_engine *e);
void ecl_clear_errors(ecl_engine *e);

/* Number of SMs and the multiple of them the kernel `kernel_name` can keep
 * resident per SM (its persistent CTAs per SM). */
ecl_status ecl_kernel_occupancy(int device_ordinal, const char *kernel_name,
                                int *sms, int *ctas_per_sm);

/* ---------------------------------------------------------------- program */

/* Creates a program bound to one built-in kernel (see the list below): the
 * Program of Sec. 4.2 (inputs, outputs, a kernel and an output pattern)
 * and Listing 1's `ecl::Program program; program.kernel(src, name)`, with
 * the name selecting a compiled kernel instead of OpenCL source.
 * Errors: ECL_ERR_ARG, ECL_ERR_KERNEL (unknown name). */
ecl_status ecl_program_create(ecl_program **p, const char *kernel_name);

/* Frees a program that was NOT given to an engine. */
void ecl_program_destroy(ecl_program *p);

/* Registers an input (resp. output) buffer of `bytes` bytes at `ptr`,
 * host or device memory (the Buffer proxy of Sec. 4.2).  The program does
 * not copy or free it.  A buffer argument must be registered before run. */
ecl_status ecl_program_in(ecl_program *p, void *ptr, size_t bytes);
ecl_status ecl_program_out(ecl_program *p, void *ptr, size_t bytes);

/* Output pattern outs:work_items (Sec. 4.2: the ratio between work-items
 * and output indices, default 1:1; Listing 1 uses 1:lws).  Must equal the
 * kernel's own pattern (listed below); it fixes which slice of each output
 * a package owns. */
ecl_status ecl_program_out_pattern(ecl_program *p, uint32_t outs, uint32_t work_items);

/* Kernel argument `index` (0-based, -1 = the next position after the
 * last one set: the aggregate form of Listing 1).  `value` points at
 * `bytes` bytes: a scalar of the kernel's declared size, or a pointer-sized
 * value holding a buffer address that was registered with
 * ecl_program_in/out (or NULL for an optional output).  Errors:
 * ECL_ERR_ARG (index out of range, size mismatch). */
ecl_status ecl_program_arg(ecl_program *p, int index, const void *value, size_t bytes);

/* Arg::LocalAlloc of Listing 1: reserves `bytes` of shared memory for a
 * local-memory argument.  None of the built-in kernels declares one
 * (their staging memory is fixed by the kernel), so this returns
 * ECL_ERR_ARG naming the kernel. */
ecl_status ecl_program_local(ecl_program *p, int index, size_t bytes);

/* Argument `index` of kernel `kernel_name`: its kind (ECL_ARG_*) and name.
 * ECL_ERR_KERNEL for an unknown kernel, ECL_ERR_ARG past the last one. */
enum { ECL_ARG_BUF_IN = 0, ECL_ARG_BUF_OUT = 1, ECL_ARG_BUF_OUT_OPT = 2,
       ECL_ARG_I32 = 3, ECL_ARG_I64 = 4, ECL_ARG_F32 = 5 };
ecl_status ecl_kernel_arg(const char *kernel_name, int index, int *kind, const char **name);

/* Number of built-in kernels and the name of kernel i (NULL out of range). */
int ecl_kernel_count(void);
const char *ecl_kernel_name(int i);

/* ---------------------------------------------------------------- no allocation
 * Potential energy E = -sum_{i<j} m_i m_j / sqrt(|r_ij|^2 + eps2) of n bodies
 * without allocating any memory.  The paper has no counterpart to this call:
 * it exists for callers that must not call cudaMalloc, such as a process
 * whose device memory is entirely owned by another allocator (a framework
 * pool, a memory-capped serving process) where an allocation behind its back
 * would fail or be counted against it.  The computation is that of the
 * "nbody_energy" program (same kernel, FP32 pair terms, FP64 sums, same
 * result) run as one plain launch without the package queue, so no engine
 * is needed.
 *   pos4        device float4[n] (x, y, z, m), 16-byte aligned
 *   n           1 .. 524288 bodies (ECL_ERR_SIZE beyond: the scratch holds
 *               one FP64 partial per 8 x 64 bodies, 512 KiB in all)
 *   eps2        softening, squared
 *   out_energy  device double[1], 8-byte aligned
 *   cuda_stream stream the work is ordered on (NULL = legacy default)
 * The scratch is a fixed array in the library's device image: every GPU that
 * loads the library holds it (512 KiB + 256 B) until the process exits.  The
 * first call on a device looks its address up (cudaGetSymbolAddress) with
 * that device current; make that first call before any stream capture.
 * The address is kept per device ordinal for the life of the process: it
 * does not survive cudaDeviceReset (or any other teardown of the device's
 * primary context), after which this entry point must not be called again
 * in the same process.
 * Every call on a device shares the one array and each call clears its
 * counter first, so calls whose work overlaps on the GPU (other streams,
 * other host threads) race: order them on one stream.  Asynchronous like
 * ecl_run; errors: ECL_ERR_ARG (NULL or misaligned pointer, n <= 0),
 * ECL_ERR_SIZE, ECL_ERR_CUDA. */
ecl_status ecl_nbody_energy_noalloc(const void *pos4, int32_t n, float eps2, double *out_energy,
                                    void *cuda_stream);

/* ---------------------------------------------------------------- kernels
 * Built-in kernels and their arguments, in order (B = buffer, S = scalar).
 *
 * "mandelbrot"  Sec. 5.3 Fig. 6, Table 2 (8 args, out pattern 4:1)
 *     0 B out uint32[W*H]  1 S int32 W  2 S int32 H  3 S float x0
 *     4 S float y0  5 S float dx  6 S float dy  7 S int32 max_iter
 *   work-item g writes pixels 4g..4g+3 (row-major); gws*4 >= W*H.
 *   Escape count of z <- z^2 + c, c = (x0 + i dx, y0 + j dy), FP32 with
 *   no fused multiply-add (bit-exact against a correctly rounded host).
 *
 * "gaussian"  Table 2 (6 args, out pattern 1:1)
 *     0 B in float[H*W]  1 B weights float[taps]  2 B out float[H*W]
 *     3 S int32 W  4 S int32 H  5 S int32 taps (odd, <= 63)
 *   separable filter, clamp-to-edge borders; work-item g writes pixel g.
 *
 * "nbody"  Listing 2 (7 args, out pattern 1:1)
 *     0 B in_pos float4[n] (x,y,z,m)  1 B in_vel float4[n]  2 S int32 n
 *     3 S float del_t  4 S float esp_sqr  5 B out_pos float4[n]
 *     6 B out_vel float4[n]
 *   a_i = sum_j m_j d_ij / (|d_ij|^2 + esp_sqr)^(3/2), d_ij = r_j - r_i;
 *   r' = r + v dt + a dt^2/2, v' = v + a dt.
 *
 * "nbody_acc"  (4 args, 1:1)  0 B in_pos  1 S int32 n  2 S float esp_sqr
 *     3 B out_acc float4[n] (ax, ay, az, 0)
 *
 * "nbody_energy"  (4 args, work-group partials)  0 B in_pos  1 S int32 n
 *     2 S float esp_sqr  3 B out_energy double[1]
 *   E = -sum_{i<j} m_i m_j / sqrt(|r_ij|^2 + esp_sqr): FP32 pair terms,
 *   FP64 sums; work-group w owns the rows i in [w lws, (w+1) lws).
 *
 * "nbody_adjoint"  (5 args, 1:1)  0 B in_pos  1 S int32 n  2 S float esp_sqr
 *     3 B grad_E float[1] (device scalar dL/dE)  4 B out_grad float4[n]
 *   out_grad_i = dL/dE * (dE/dx_i, dE/dy_i, dE/dz_i, dE/dm_i) with
 *   dE/dr_i = -m_i a_i and dE/dm_i = -sum_{j!=i} m_j / sqrt(r_ij^2+eps2).
 *
 * "nbody_fd"  (8 args, one work-group per sample, lws 1)
 *     0 B in_pos  1 S int32 n  2 S float esp_sqr  3 S float h
 *     4 B body int32[s]  5 B comp int32[s]  6 S int32 s  7 B out double[s]
 *   central difference of E in coordinate comp of body: the perturbed
 *   coordinate is rounded to FP32 and the denominator is the FP32 distance
 *   between the two placements; FP32 terms, the FP64 sum of their
 *   differences (each sample's bodies cut into up to 16 segments, added in
 *   segment order: the result does not depend on the schedule).  A sample
 *   with a body outside [0, n) or a component outside 0..2 gives NaN.
 *
 * "binomial"  Listing 1 workload (9 args, out pattern 1:32, lws 32)
 *     0 B S float[n]  1 B K float[n]  2 B T float[n]  3 B sigma float[n]
 *     4 B steps int32[n] (1..2048; other depths give NaN)  5 S float r  6 S int32 n
 *     7 B price float[n]  8 B greeks float2[n] (delta, vega) or NULL
 *   European call on a Cox-Ross-Rubinstein lattice of steps[o] steps,
 *   backward induction in FP32 by one warp per option (two FP32
 *   instructions per node); with greeks the exact derivatives of the
 *   lattice price with respect to S and sigma, from the lattice's adjoint
 *   weights in closed form (binomial probabilities), in a second, plain
 *   launch on the engine's stream that reads what the lattice kernel left
 *   in the greeks buffer (so greeks hold their final values only once the
 *   run is complete).  Nodes that are
 *   exactly zero (below the strike on the out-of-the-money side) are not
 *   computed.  Inputs: S, K > 0 and T, sigma >= 0; an option whose
 *   out-of-the-money leaves are more than N/2 + 1 (only with sigma or T
 *   negative) gets NaN results.
 *
 * "binomial_full"  (the arguments of "binomial")  the same prices computing
 *   every node of every level: the reference form of "binomial" (identical
 *   prices; greeks from the adjoint lattice, within ~1e-6 of the closed
 *   form).
 *
 * "binomial_batch"  (4 args, out pattern 1:32, lws 32)  many option batches
 *   of uneven size in one NDRange and one persistent launch:
 *     0 B instances ecl_binomial_instance[count] (device, 16-byte aligned)
 *     1 S int32 count  2 S int64 total options  3 S int32 with_greeks
 *   instance i prices options [first_i, first_i + n_i) of the NDRange (first
 *   ascending from 0, sum of n_i = total) from its own arrays; with_greeks = 0
 *   skips delta and vega for the whole batch.  The engine does not
 *   see the arrays the table points to: the caller guarantees them.
 *
 * "mandelbrot_batch"  (3 args, one output pixel block per work-item, lws
 *   256)  many views of uneven size in one NDRange and one persistent launch
 *   (not in the paper: its package model over a concatenated NDRange):
 *     0 B views ecl_mandelbrot_view[count] (device, 16-byte aligned)
 *     1 S int32 count  2 S int64 total work-groups
 *   view i owns work-groups [first_i, first_i + wgs_i) (first ascending from
 *   0) and computes them as "mandelbrot" does its own.  A view with a
 *   misaligned output or no pixels is skipped.  The engine does not see the
 *   arrays the table points to: the caller guarantees them.
 *
 * "gaussian_batch"  (3 args, lws 256 = one 32 x 224 output tile per
 *   work-group)  many images of uneven size, 31 taps each with their own
 *   weights, clamp-to-edge, in one NDRange and one persistent launch (not in
 *   the paper: its package model over a concatenated NDRange of tiles):
 *     0 B images ecl_gaussian_image[count] (device, 16-byte aligned)
 *     1 S int32 count  2 S int64 total tiles
 *   image i owns work-groups [first_i, first_i + tiles_i), tile t at rows
 *   32 (t / ceil(W/224)), columns 224 (t % ceil(W/224)).  An image with a
 *   misaligned output or no pixels is skipped.  The caller guarantees the
 *   arrays the table points to.
 *
 * "gemm_bf16"  (6 args; lws 32768 = one 128 x 256 output tile; the
 *   scheduling unit is two rows of tiles: a CTA computes two vertically
 *   adjacent tiles together)
 *     0 B A bf16[M*K] row-major  1 B Bt bf16[N*K] row-major (B transposed)
 *     2 B C float[M*N] row-major  3 S int32 M  4 S int32 N  5 S int32 K
 *   C = A B, FP32 accumulation in tensor memory (tcgen05).  gws =
 *   ceil(M/128) * ceil(N/256) * 32768; K % 8 == 0.
 *
 * "gemm_split3"  same arguments with A, Bt as float.  Each input is split
 *   into hi = bf16(x) and lo = bf16(x - hi); C = A_hi B_hi + A_hi B_lo +
 *   A_lo B_hi in one FP32 accumulator.  Uses an engine-owned workspace.
 *
 * "gemm_split6"  (7 args; lws 16384 = one 128 x 128 output tile; the
 *   scheduling unit is one row of tiles)  A, Bt, C, M, N, K as "gemm_split3"
 *   (A, Bt float) plus 6 S int32 chunk_k (0 = 1).  Not in the paper: the
 *   compensated GEMM carried to FP32 accuracy.  Each input is split into
 *   x = h + m + l, h = bf16(x), m = bf16(x - h), l = bf16(x - h - m), and
 *   C = hh + (hm + mh + hl + lh + mm): the hh products go into a fresh
 *   tensor-memory accumulator for every chunk_k slices of 64 along K and
 *   are added into FP32 registers (round to nearest) after each chunk; the
 *   five cross products accumulate over the whole K and are added once.
 *   gws = ceil(M/128) * ceil(N/128) * 16384; K % 8 == 0; A and Bt need no
 *   alignment (they are read by the split pass), C 16-byte aligned.  Uses
 *   an engine-owned workspace of 6 bf16 copies (12 * (M + N) * K bytes).
 *
 * "ray"  (11 args, out pattern 1:1; Table 2 gives lws 128)  Sec. 7's Ray
 *   workload as a Whitted tracer (the paper's tracer and scenes are not
 *   available, so the definition is this library's):
 *     0 B scene float[12*spheres + 8*lights]: sphere k = centre x y z,
 *       radius, colour r g b, reflectivity, kd, ks, log2 of the specular
 *       exponent, pad; then light l = position x y z, pad, intensity r g b,
 *       pad
 *     1 S int32 spheres (0..128)  2 S int32 lights (0..16)  3 S int32 width
 *     4 S int32 height  5 S float ambient  6-8 S float background r g b
 *     9 S int32 max_depth (0..64)  10 B out float4[width*height]
 *   Work-item g traces pixel g (row-major) from a camera at the origin
 *   looking down -z (u = (2i+1-W)/H, v = (H-2j-1)/H): nearest sphere hit,
 *   hard shadows from every light, Phong shading, mirror reflections
 *   followed front to back while reflectivity > 0 and depth < max_depth.
 *   out = (r, g, b, rays traced).  FP32 without fused multiply-add: the
 *   result is bit-reproducible on the host.
 *
 * "cast_bf16"  (3 args, 1:1, any lws)  0 B in float[n]  1 B out bf16[n]
 *   2 S int64 n: round to nearest even (the input cast of "gemm_bf16").
 *
 * "fp32_probe"  (4 args, 1:1, lws 256)  0 B out float[gws]  1 S int32 iters
 *   2 F32 m  3 F32 c: not a workload but the measured denominator of the
 *   FP32 rooflines.  Work-item g runs 8 independent chains x <- fma(x, m, c)
 *   of 16*iters steps and writes their sum: 128*iters FFMA per work-item
 *   (m = 0.999, c = 0.001 keep the chains near 1).
 */

#ifdef __cplusplus
}
#endif
#endif /* ECL_H */
