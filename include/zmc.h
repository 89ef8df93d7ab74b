/*
 * zmc.h -- C ABI of the GB300 stratified Monte Carlo integrator.
 *
 * The library implements the method of ZMCintegral (arXiv 1902.07916,
 * Sec. 2.1 and Fig. 1): the integration box is split into k^d equal cells;
 * in every cell the integral is estimated by direct Monte Carlo with n points,
 * independently `num_trials` times (the paper's n1); the cells whose spread
 * over trials is larger than a threshold formed from the mean and standard
 * deviation of all the level's spreads are split again into k^d children, down
 * to a maximal depth; the accepted cells' means are summed into the value and
 * their spreads into the error.  Random numbers are made where they are used
 * (Sec. 2.2), by Philox4x32-10.
 *
 * Conventions for every call:
 *  - Return value: ZMC_OK (0) or one of the ZMC_ERR_* codes below.  On
 *    ZMC_ERR_ARG no output is written.  zmc_last_error(h) then describes the
 *    failure.
 *  - A handle is not thread-safe; distinct handles are independent.
 *  - Pointers documented as "host" are read or written by the CPU only; the
 *    library copies what it keeps.  The library owns all device memory it
 *    allocates for a handle and frees it in zmc_destroy.
 *  - `stream` arguments are cudaStream_t values passed as void*; NULL means
 *    the legacy default stream.  All device work of a call is ordered on it.
 *
 * Readings of the paper used by every entry point (the paper leaves these
 * open): k divisions per dimension; cells numbered row-major with dimension 0
 * fastest; per-cell spread = sample standard deviation over trials; level
 * threshold = mean + sigma_multiplier * population standard deviation of the
 * level's spreads, a cell flagged when strictly larger and never at the last
 * level; error = sqrt(sum over accepted cells of spread^2 / num_trials).
 */
#ifndef ZMC_H
#define ZMC_H

#ifndef __CUDACC_RTC__
#include <stddef.h>
#include <stdint.h>
#endif

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define ZMC_API __attribute__((visibility("default")))
#else
#define ZMC_API
#endif

/* ------------------------------------------------------------ status codes */
#define ZMC_OK 0
#define ZMC_ERR_ARG 1          /* an argument is out of range               */
#define ZMC_ERR_COMPILE 2      /* a user expression failed to compile       */
#define ZMC_ERR_BUDGET 3       /* refinement stopped by max cells / samples */
#define ZMC_ERR_NONFINITE 4    /* the integrand produced NaN or Inf         */
#define ZMC_ERR_OOM 5          /* device memory could not be allocated      */
#define ZMC_ERR_CUDA 6         /* a CUDA runtime call failed                */
#define ZMC_ERR_TIMEOUT 7      /* reserved for a bounded device-side wait;
                                  no kernel of this library waits on another
                                  CTA or kernel, so no call returns it      */
#define ZMC_ERR_NOINTEGRAND 8  /* zmc_set_integrand was never called        */
#define ZMC_ERR_CHECK 9        /* bounds-guarded build only: an index was out
                                  of its buffer; the access was skipped     */

/* ------------------------------------------------------- precision modes */
#define ZMC_FP64 0             /* FP64 uniforms, points, integrand and sums */
#define ZMC_FP32_FP64ACC 1     /* FP32 evaluation, FP32 partial sums over
                                  88 points, FP64 per-thread and warp sums  */
#define ZMC_FP32_KAHAN 2       /* FP32 evaluation, FP32 Kahan / two-sum
                                  accumulation up to the per-cell result     */
/* The FP32 modes draw their points from the FP32 stream (eleven 23-bit
 * uniforms per pair of Philox blocks, see zmc_uniforms), so they sample other
 * points than the FP64 mode does: their results differ from it by Monte Carlo
 * noise as well as by rounding.  The Gaussian integrands ("gauss_norm",
 * "genz_gauss") are evaluated in the log2 domain in the FP32 modes (each
 * thread sums 2^(t - k) against its own reference exponent k, and the sums
 * reach FP64 through ldexp), so values far below FP32's range (1e-38), as a
 * Gaussian of width 0.01 in 9-D gives on cells of width 2/3, keep their
 * spread and steer the refinement as in FP64.  Their relative error grows
 * with the exponent's size and gradient: about 2^-22 (|E| + |grad E| |x|)
 * for exp(E). */

#define ZMC_MAX_DIM 16
#define ZMC_MAX_DEPTH 16
#define ZMC_PLAN_FIELDS 5

typedef struct zmc_ctx* zmc_handle;   /* opaque; owned by the library */

/* Result of one integration.  Arrays are indexed by level - 1. */
typedef struct zmc_result {
    double value;                 /* sum of accepted cell means             */
    double std;                   /* sqrt(sum accepted spread^2 / trials)   */
    int64_t cells_evaluated;      /* cells over all levels run              */
    int64_t samples;              /* points evaluated: sum C_L * n * trials */
    int32_t levels_run;           /* levels actually evaluated (>= 1)       */
    int32_t status;               /* ZMC_OK, ZMC_ERR_BUDGET or _NONFINITE   */
    int64_t cells_per_level[ZMC_MAX_DEPTH];
    int64_t flagged_per_level[ZMC_MAX_DEPTH];   /* cells split further    */
    double theta_per_level[ZMC_MAX_DEPTH];      /* threshold theta_L      */
    double mu_per_level[ZMC_MAX_DEPTH];         /* mean of the spreads    */
    double sigma_per_level[ZMC_MAX_DEPTH];      /* std (ddof 0) of them   */
    /* min over the level's cells of |spread - theta| / theta: how close the
       closest selection decision was to a tie (+inf at the last level). */
    double min_margin_per_level[ZMC_MAX_DEPTH];
    /* the work plan the run used (see zmc_set_work_plan): it fixes the order
       in which every (cell, trial) sum was added up, so passing it back to
       zmc_set_work_plan reproduces the result bit for bit */
    int64_t work_plan[ZMC_PLAN_FIELDS];
} zmc_result;

/*
 * zmc_create -- Sec. 2.1 and Sec. 2.3 (the hyper-parameters).
 *   dim              1 .. ZMC_MAX_DIM
 *   lo, hi           host arrays of `dim` doubles, lo[i] < hi[i], finite;
 *                    copied, the caller keeps ownership
 *   k                divisions per dimension per level, >= 2; k^dim cells
 *                    at level 1 (must be < 2^32), k^depth < 2^32
 *   n                points per cell per trial, >= 2, n*dim < 2^34
 *   num_trials       independent repetitions per cell (n1), 2 .. 1024
 *   depth            maximal partition depth, 1 .. ZMC_MAX_DEPTH
 *   sigma_multiplier m in theta = mu + m*sigma, finite, >= 0
 *   seed             64-bit Philox key (low word, high word)
 * Writes a new handle to *out.  Host-only: no device work happens here.
 * Errors: ZMC_ERR_ARG.
 */
ZMC_API int zmc_create(zmc_handle* out, int dim, const double* lo,
                       const double* hi, int k, int64_t n, int num_trials,
                       int depth, double sigma_multiplier, uint64_t seed);

/*
 * zmc_set_integrand -- the function to integrate (Sec. 3: f1 of Eq. 1 and f2
 * of Eq. 2, plus the Genz test family and user expressions).
 *   name_or_expr  one of
 *     "sin_sum"        sin(x_0 + ... + x_{d-1})                 params: none
 *     "gauss_norm"     (sqrt(2 pi) s)^-d exp(-|x|^2 / (2 s^2))  params: s
 *     "genz_osc"       cos(2 pi u + sum a_i x_i)      params: u, a_0..a_{d-1}
 *     "genz_prodpeak"  prod 1/(a_i^-2 + (x_i-u_i)^2)  params: a_0.., u_0..
 *     "genz_gauss"     exp(-sum a_i^2 (x_i-u_i)^2)    params: a_0.., u_0..
 *     "genz_corner"    (1 + sum a_i x_i)^-(d+1)       params: a_0..a_{d-1}
 *     "constant"       c                              params: c
 *     "linear"         b + sum a_i x_i                params: b, a_0..
 *     "expr:<C expression in x[0..d-1] and p[0..n_params-1]>"
 *                      compiled at run time with NVRTC for this device
 *   params      host array of n_params doubles (copied); may be NULL when
 *               n_params == 0
 * Errors: ZMC_ERR_ARG (unknown name, wrong parameter count, bad values),
 *         ZMC_ERR_COMPILE (expression rejected; the log is in
 *         zmc_last_error), ZMC_ERR_CUDA.
 */
ZMC_API int zmc_set_integrand(zmc_handle h, const char* name_or_expr,
                              const double* params, int n_params);

/* zmc_set_precision -- ZMC_FP64, ZMC_FP32_FP64ACC or ZMC_FP32_KAHAN.
 * The cross-trial statistics, threshold, selection and final sums are FP64
 * in every mode.  Errors: ZMC_ERR_ARG. */
ZMC_API int zmc_set_precision(zmc_handle h, int mode);

/* zmc_set_limits -- refinement budget.  If splitting the flagged cells of a
 * level would make the next level larger than max_cells_per_level cells, or
 * the whole run larger than max_samples points, that level is accepted whole,
 * refinement stops and the result carries status ZMC_ERR_BUDGET.  Device
 * buffers are sized from these limits.  Defaults: 2^24 cells, 2^40 points.
 * Both must be >= the size of level 1.  Errors: ZMC_ERR_ARG. */
ZMC_API int zmc_set_limits(zmc_handle h, int64_t max_cells_per_level,
                           int64_t max_samples);

/*
 * zmc_set_launch -- launch shape of the sampling kernel: `threads` per CTA
 * (64, 128 or 256) and at most `ctas_per_sm` CTAs per SM (0: as many as fit).
 * threads = 0 (the default) lets the library's autotuner choose: on the
 * first run of a (precision, integrand, dimension) it times each candidate
 * shape once on a truncated level 1 of that problem and keeps the fastest
 * for the process (ZMC_TUNE=0 in the environment disables it).  The timing
 * runs go on the handle's own stream once the caller's stream has reached
 * the call (an event, no device-wide synchronisation); when the caller's
 * stream is being captured nothing is timed and the default shape (256
 * threads, as many CTAs as fit) is used for that run.  Results do not
 * depend on the shape: the work units and their order of summation are
 * fixed by the level's size, n and the precision.  Errors: ZMC_ERR_ARG.
 * zmc_launch_shape reports the shape of the last run (threads per CTA, CTAs).
 */
ZMC_API int zmc_set_launch(zmc_handle h, int threads, int ctas_per_sm);
ZMC_API int zmc_launch_shape(zmc_handle h, int* threads, int* grid);

/*
 * zmc_set_work_plan -- how the sampling kernel cuts a level into work units
 * (the paper leaves the GPU work decomposition open; its Numba kernels fix
 * threads per block per experiment, Sec. 3.1-3.2).  Unlike the launch shape
 * the plan decides the order in which each (cell, trial) sum is added up, so
 * results depend on it at rounding level (FP64: about 1e-15 relative; FP32
 * modes: about 1e-7), and every result records the plan it ran with
 * (zmc_result::work_plan).  plan: host array of ZMC_PLAN_FIELDS int64:
 *   [0] target_units          a level is cut into at least this many units
 *                             when its tiles allow, 1 .. 2^18
 *   [1] min_unit_groups       ... but no unit has fewer point groups (of 4
 *                             points in FP64, 11 in the FP32 modes), >= 1:
 *                             "samples per thread" is 1/32 of a unit
 *   [2] lane_tile_groups      tiles of fewer groups always run one per lane
 *   [3] lane_tile_max_groups  tiles of fewer groups run one per lane on ...
 *   [4] lane_tile_min_tiles   ... levels of at least this many tiles, >= 1
 * plan = NULL restores the default, {2^18, 1024, 64, 1024, 2^18}, or the
 * tuned plan when ZMC_TUNE_PLAN is on.  Errors: ZMC_ERR_ARG.
 *
 * zmc_set_tuning -- what the autotuner may choose on a handle's first run:
 * ZMC_TUNE_SHAPE (the default) the launch shape only, which never changes a
 * result; ZMC_TUNE_PLAN also the work plan (lane_tile_min_tiles, then
 * min_unit_groups), timed on the handle's own level 1 when that holds at
 * most 2^31 points (larger levels keep the default), adopted only when at
 * least 2% faster, cached per (kernel, dimension, n, level size) for the
 * process and recorded in the results.  An explicit zmc_set_launch /
 * zmc_set_work_plan wins over the tuner.  Errors: ZMC_ERR_ARG.
 *
 * Persisted choices: with ZMC_TUNE_CACHE=<path> in the environment, every
 * tuned shape and plan is also appended to that file (one JSON object per
 * line, keyed by device name, SM count, compute capability, a hash of the
 * library build, precision, integrand or a hash of the expression, and the
 * problem's dimension -- plus n and level size for a plan), and a later
 * process reads the file before timing anything.  Lines that do not parse or
 * hold values a setter would reject are skipped; a file that cannot be read
 * or written only disables the persistence.
 */
#define ZMC_TUNE_SHAPE 1
#define ZMC_TUNE_PLAN 2
ZMC_API int zmc_set_work_plan(zmc_handle h, const int64_t* plan);
ZMC_API int zmc_set_tuning(zmc_handle h, int flags);

/*
 * zmc_integrate -- run the whole tree search on the current device and
 * return the result in *out (host).  Copies the handle's parameters to the
 * device, enqueues every level on `stream` (replaying a CUDA graph captured
 * on first use), copies the result back and synchronises the stream.  The
 * tree search itself never returns to the host between levels.
 * Returns ZMC_OK, or the result's status (ZMC_ERR_BUDGET,
 * ZMC_ERR_NONFINITE: *out is still filled), or ZMC_ERR_NOINTEGRAND,
 * ZMC_ERR_OOM, ZMC_ERR_CUDA (*out untouched).
 */
ZMC_API int zmc_integrate(zmc_handle h, void* stream, zmc_result* out);

/*
 * zmc_enqueue -- the device half of zmc_integrate: enqueue the tree search on
 * `stream` and return at once; the result stays in device memory until
 * zmc_read_result.  The handle's parameters must already be on the device
 * (they are uploaded here only if a setter ran since the last upload).  The
 * caller must not call a setter, zmc_integrate or zmc_destroy on the handle
 * until the stream has passed this work.
 * Errors: ZMC_ERR_NOINTEGRAND, ZMC_ERR_OOM, ZMC_ERR_CUDA.
 */
ZMC_API int zmc_enqueue(zmc_handle h, void* stream);

/* zmc_read_result -- copy the result of the last zmc_enqueue to *out (host),
 * synchronising `stream` first.  Returns like zmc_integrate. */
ZMC_API int zmc_read_result(zmc_handle h, void* stream, zmc_result* out);

/*
 * zmc_integrate_batch -- many independent integrations in one pass per
 * level: one persistent kernel per level pops (integral, cell, trial) tiles
 * from an atomic work queue, then selection runs per integral.  All handles
 * must use the same precision mode and be on the same device; their
 * integrands must be registry names (not expressions).  outs: host array of
 * `count` results.  Returns ZMC_OK if every integral returned ZMC_OK,
 * otherwise the first non-OK status (each outs[i].status holds its own).
 */
ZMC_API int zmc_integrate_batch(int count, const zmc_handle* hs, void* stream,
                                zmc_result* outs);

/*
 * Tracing, for verification against a reference implementation.
 * zmc_set_trace(h, 1) makes later zmc_integrate calls run level by level
 * with the same kernels and launch shapes, synchronising after every level
 * and keeping a host copy of that level's data.  zmc_trace_level then copies
 * one level (1-based) out; any pointer may be NULL.
 *   cells, flagged   host int64: C_L and the number of cells split further
 *   stats4           host double[4]: mu_L, sigma_L, theta_L, min margin
 *   sums             host double[C_L * num_trials * 2]: (S1, S2) per
 *                    (cell, trial), cell-major
 *   cell_stats       host double[C_L * 2]: (mean, spread) per cell
 *   parents_out      host uint32[flagged * dim]: lattice coordinates (at
 *                    this level) of the split cells, in next-level order
 * Errors: ZMC_ERR_ARG (level not traced).
 */
ZMC_API int zmc_set_trace(zmc_handle h, int on);
ZMC_API int zmc_trace_level(zmc_handle h, int level, int64_t* cells,
                            int64_t* flagged, double* stats4, double* sums,
                            double* cell_stats, uint32_t* parents_out);

/*
 * zmc_philox_words -- the generator the sampling kernel uses, exposed for
 * bit-exact checks.  For b in [0, count) writes the four words of
 * Philox4x32-10(counter = (c0 + b, c1, c2, c3), key = (seed lo, seed hi))
 * to out[4b .. 4b+3].  out: device pointer to 4*count uint32.  Asynchronous
 * on `stream`.  Errors: ZMC_ERR_ARG, ZMC_ERR_CUDA.
 */
ZMC_API int zmc_philox_words(uint64_t seed, uint32_t c0, uint32_t c1,
                             uint32_t c2, uint32_t c3, int64_t count,
                             uint32_t* out, void* stream);

/*
 * zmc_uniforms -- the uniforms the sampling kernel draws, for bit-exact
 * checks of the stream definition (Sec. 2.2: numbers produced where they are
 * used; the generator and layout are this library's choice).  For points
 * [first, first + count) of the stream of (level, slot, trial) under `seed`,
 * writes u into out[(s - first) * dim + i] for every dimension i.
 *   mode ZMC_FP64: dimension i of points 4g..4g+3 are the four 32-bit words
 *     of the Philox4x32-10 block with counter (g*dim + i, trial, slot, level),
 *     u = (w + 1/2) 2^-32;
 *   mode ZMC_FP32_*: dimension i of points 11g..11g+10 come from the pair of
 *     blocks with counters (2(g*dim + i), trial, slot, level) and
 *     (2(g*dim + i) + 1, trial, slot, level), each read as a 128-bit
 *     integer: points 0..4 of the group take the first block's 23-bit fields
 *     (bits 23f .. 23f+22), points 5..9 the second block's, and point 10 the
 *     first block's bits 115..127 below the second block's bits 115..124;
 *     u = (field + 1/2) 2^-23.
 * out: device pointer to count*dim doubles.  Asynchronous on `stream`.
 * Errors: ZMC_ERR_ARG, ZMC_ERR_CUDA.
 */
ZMC_API int zmc_uniforms(uint64_t seed, int level, uint32_t slot, uint32_t trial, int dim,
                         int mode, int64_t first, int64_t count, double* out, void* stream);

/*
 * Instrumentation for measurement.
 * zmc_set_profiling(h, 1): later runs record CUDA events around every
 * level's sampling kernel (inside the captured graph, on the run's stream).
 * zmc_profile(h, eval_ms, levels) then writes, after the stream has passed
 * the run, the sampling kernel's duration per level (host double[depth]) and
 * the number of levels that had cells to *levels.
 * zmc_run_info(h, kernels, h2d_bytes, d2h_bytes): kernels launched by one
 * run (the kernel nodes of the captured graph), and the bytes zmc_integrate
 * copies host->device (the run's parameters) and device->host (the result)
 * per call.  Any pointer may be NULL.  Errors: ZMC_ERR_ARG, ZMC_ERR_CUDA.
 */
ZMC_API int zmc_set_profiling(zmc_handle h, int on);
ZMC_API int zmc_profile(zmc_handle h, double* eval_ms, int* levels);
ZMC_API int zmc_run_info(zmc_handle h, int64_t* kernels, int64_t* h2d_bytes,
                         int64_t* d2h_bytes);

/*
 * zmc_pipe_probe -- measure one instruction kind's throughput on the current
 * GPU (the paper has no counterpart: these are the roofline denominators of
 * the sampling kernel, whose bound is integer work, for which no vendor peak
 * is published).  Launches `blocks` CTAs of `threads` threads (a multiple of
 * 32, at most 256); each thread runs 8 independent chains for `iters` steps:
 *   ZMC_PROBE_IMAD_WIDE    one mad.wide.u32 (32x32 -> 64-bit) per step
 *   ZMC_PROBE_IMAD         one mad.lo.u32
 *   ZMC_PROBE_IMAD_HI      one mad.hi.u32
 *   ZMC_PROBE_HILO_PAIRED  the high and low halves of one 32x32 product (as a
 *                          Philox round needs them) and a three-input XOR
 *   ZMC_PROBE_HILO_SPLIT   the same with the low half's multiplier held in a
 *                          kernel parameter, so the two halves stay separate
 *                          instructions
 *   ZMC_PROBE_LOP3         one three-input XOR (lop3.b32)
 *   ZMC_PROBE_FFMA         one FP32 fma;  ZMC_PROBE_DFMA  one FP64 fma
 *   ZMC_PROBE_PHILOX       one Philox4x32-10 block as the sampling kernel
 *                          forms it (17 wide products, 19 + 2 XORs, a 64-bit
 *                          add)
 *   ZMC_PROBE_PHILOX_SPLIT the same block with split high/low products
 *   sink     device, blocks * threads uint32 out (keeps the work alive)
 *   clocks   device, blocks * 6 int64 out: per CTA, %clock64 before and after
 *            the loop, %globaltimer (ns) before and after, %smid, 0
 * Asynchronous on `stream`.  Errors: ZMC_ERR_ARG, ZMC_ERR_CUDA.
 */
#define ZMC_PROBE_IMAD_WIDE 0
#define ZMC_PROBE_IMAD 1
#define ZMC_PROBE_IMAD_HI 2
#define ZMC_PROBE_HILO_PAIRED 3
#define ZMC_PROBE_HILO_SPLIT 4
#define ZMC_PROBE_LOP3 5
#define ZMC_PROBE_FFMA 6
#define ZMC_PROBE_DFMA 7
#define ZMC_PROBE_PHILOX 8
#define ZMC_PROBE_PHILOX_SPLIT 9
ZMC_API int zmc_pipe_probe(int kind, int64_t iters, int blocks, int threads, uint32_t* sink,
                           int64_t* clocks, void* stream);

/*
 * zmc_level_stats_noalloc -- one tree level's per-cell statistics and
 * threshold (the same arithmetic as the library's own selection step: trial
 * estimates I = volume * S1 / n, per-cell mean and sample spread, and
 * theta = mu + sigma_multiplier * sigma over the cells' spreads) for
 * per-(cell, trial) sums the caller already holds, without allocating any
 * device memory.  The paper has no counterpart; this exists for callers
 * that cannot allocate device memory: applications whose device memory is
 * all owned by their own pool or arena (a framework's caching allocator, a
 * fixed budget carved out at start-up) and that forbid any other allocator,
 * and latency-critical loops that cannot afford the device-wide
 * synchronisation cudaMalloc and cudaFree may imply.
 *   sums         device, cells * trials * 2 doubles: (S1, S2) per (cell,
 *                trial), cell-major (the layout zmc_trace_level returns)
 *   cells        1 .. 1048576 (the bound set by the entry point's scratch)
 *   trials       >= 2;  n >= 1 points per (cell, trial)
 *   volume       the cells' volume;  sigma_multiplier finite, >= 0
 *   cell_stats   device, cells * 2 doubles out: (mean, spread) per cell
 *   level_stats  device, 3 doubles out: (mu, sigma, theta)
 * All outputs are written asynchronously on `stream`.  Scratch: a fixed
 * static device array of about 24 KiB that every GPU using the library holds
 * until the process exits, shared by all calls and keeping the last call's
 * contents (each call clears what must start at zero).  Calls that overlap
 * on the GPU (on different streams, or from different host threads) race on
 * it and must be serialised by the caller.  Every call looks up the array's
 * device address on the current device (cudaGetSymbolAddress, which
 * allocates nothing, so a reset of the device's context leaves no stale
 * address behind); the first call on a device may load the library's device
 * code there, so make it before any stream capture.  Non-finite sums are not
 * reported (unlike zmc_integrate's ZMC_ERR_NONFINITE): a NaN or infinite S1
 * makes that cell's mean and spread, and then mu, sigma and theta, NaN or
 * infinite; callers that need the check test theta with isfinite.
 * Errors: ZMC_ERR_ARG (sizes beyond the bound, NULL pointers, bad values;
 * nothing is launched), ZMC_ERR_CUDA.
 */
ZMC_API int zmc_level_stats_noalloc(const double* sums, int64_t cells, int trials, int64_t n,
                                    double volume, double sigma_multiplier, double* cell_stats,
                                    double* level_stats, void* stream);

/*
 * zmc_check_expression -- compile an expression integrand (the text after
 * "expr:" in zmc_set_integrand; Sec. 3.3 names integrands with condition
 * checks and special functions as a need) for a GPU of compute capability
 * cc_major.cc_minor with NVRTC, without a device and without loading the
 * result: a way to validate expressions ahead of time (and what a host
 * without a GPU can test).
 *   expr         NUL-terminated expression in x[0..dim-1] and p[...]
 *   dim          1..16;  mode  ZMC_FP64 | ZMC_FP32_FP64ACC | ZMC_FP32_KAHAN
 *   log          caller's buffer of log_size bytes (may be NULL when
 *                log_size is 0): the compiler's log or the reason, truncated
 *                and NUL-terminated
 * Errors: ZMC_ERR_ARG (bad sizes or mode, empty expression),
 * ZMC_ERR_COMPILE (NVRTC rejected it, or libnvrtc could not be opened).
 */
ZMC_API int zmc_check_expression(const char* expr, int dim, int mode, int cc_major, int cc_minor,
                                 char* log, size_t log_size);

/* zmc_last_error -- message of the last failed call on h (or of the last
 * failed zmc_create / handle-less call when h is NULL).  Never NULL; valid
 * until the next call on the same handle. */
ZMC_API const char* zmc_last_error(zmc_handle h);

/* zmc_destroy -- free the handle and its device memory.  NULL is accepted. */
ZMC_API int zmc_destroy(zmc_handle h);

#ifdef __cplusplus
}
#endif
#endif /* ZMC_H */
