/*
 * nifty_ls.h -- C-ABI of the GB300 Lomb-Scargle library (method of nifty-ls,
 * Garrison, Foreman-Mackey, Shih & Barnett, arXiv 2409.08090).
 *
 * The library computes the floating-mean, standard-normalised Lomb-Scargle
 * periodogram on the uniform grid f_k = f0 + k df, k = 0 .. nf-1, from the
 * weighted trigonometric sums of Eq. 1 (Sec. 1), evaluated as type-1
 * (nonuniform to uniform) NUFFTs (Eq. 2, Sec. 1): exponential-of-semicircle
 * spreading onto an upsampled fine grid, an FFT of that grid and a diagonal
 * deconvolution (Sec. 1, the finufft paragraph), with width and grid size
 * chosen from the tolerance eps.  Three transforms are taken per series:
 * w^(y - ybar) and w^ at f, w^ at 2f (w_j = 1/dy_j^2, w^ = w / sum w); the
 * sums then give P_k = (YC_tau^2/CC_tau + YS_tau^2/SS_tau)/YY (generalised
 * periodogram, standard normalisation; the paper cites VanderPlas 2018 for it).
 *
 * Memory: every pointer argument may be device memory or host memory (pageable
 * or pinned); the library asks the CUDA runtime which.  Device inputs are read
 * in place and the call returns once the work is queued on the plan's stream.
 * Host inputs are copied into plan-owned device buffers, and a host output is
 * copied back before the call returns (the call then synchronises the stream).
 * All arrays are FP64, contiguous, caller-owned; the plan owns its workspace.
 *
 * Errors: argument errors are returned immediately.  Errors found on the
 * device (a non-finite t/y/dy, dy <= 0, a constant series) are recorded in a
 * per-plan status word that ls_sync() returns; an execution with host output
 * reports them directly.  No entry point aborts, traps or prints.
 *
 * Threading: a plan is not thread-safe; use one plan per host thread or
 * serialise calls.  Plans on different devices are independent.
 */
#ifndef NIFTY_LS_H
#define NIFTY_LS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ls_plan_s *ls_plan_t;

typedef enum {
    LS_OK = 0,
    LS_ERR_ARG = 1,         /* invalid argument or invalid input values          */
    LS_ERR_NOMEM = 2,       /* device or host allocation failed                  */
    LS_ERR_CUDA = 3,        /* a CUDA runtime call failed                        */
    LS_ERR_TIMEOUT = 4,     /* a bounded device-side wait gave up                */
    LS_ERR_DEGENERATE = 5,  /* the weighted variance of y is zero (YY == 0)      */
    LS_ERR_UNSUPPORTED = 6  /* valid request outside what this build implements  */
} ls_status;

/*
 * Normalisation and model (the `norm` argument of the execute calls): one
 * ls_norm value, optionally OR'ed with the model flags below.  These are the
 * options of the Astropy Lomb-Scargle interface that nifty-ls backs (Sec. 1).
 * With chi2 the weighted residual (w = 1/dy^2) of the best sinusoid model at
 * f_k and chi2_ref that of the model without the sinusoid:
 */
typedef enum {
    LS_NORM_STANDARD = 0,   /* 1 - chi2/chi2_ref, in [0, 1]                         */
    LS_NORM_MODEL = 1,      /* chi2_ref/chi2 - 1 = P/(1 - P)                         */
    LS_NORM_LOG = 2,        /* ln(chi2_ref/chi2) = -ln(1 - P) (P >= 1 gives inf/NaN) */
    LS_NORM_PSD = 3         /* (chi2_ref - chi2)/2                                  */
} ls_norm;
/* Model flags.  Default: floating mean (y ~ a cos + b sin + c on centred y).
 * LS_NO_FIT_MEAN: y ~ a cos + b sin, no offset; the transform of w^ at f is
 *   then not needed and is skipped (two transforms per series, not three).
 * LS_NO_CENTER: with LS_NO_FIT_MEAN, y is used as given instead of y - ybar;
 *   ignored with a fitted mean (the offset absorbs the mean). */
#define LS_NO_FIT_MEAN 0x100
#define LS_NO_CENTER 0x200

/* Arithmetic of the spread, the fine-grid FFT and the deconvolution.  In both
 * precisions the phase reduction t*df mod 1, the pre-phase exp(2 pi i fc t),
 * the weighted mean and the final power ratio are FP64. */
typedef enum { LS_FP64 = 0, LS_FP32 = 1 } ls_prec;

/* Parameters a plan chose; filled by ls_plan_describe. */
typedef struct {
    int64_t nf;            /* frequencies the plan was made for               */
    int64_t max_nd;        /* largest series it accepts                       */
    int64_t n;             /* fine-grid size per transform (2,3,5-smooth)     */
    int32_t n1, n2;        /* four-step split n = n1 * n2                     */
    int32_t width;         /* kernel width w (fine-grid cells)                */
    int32_t prec;          /* ls_prec                                         */
    double beta;           /* ES kernel shape parameter                       */
    double eps;            /* tolerance the plan was made for                 */
    double sigma;          /* upsampling factor chosen (n >= sigma nf)        */
    int64_t workspace_bytes;
    int32_t cols_per_block; /* fine-grid columns per pass-A block (bin width)  */
    int32_t fft_max_radix;  /* largest power-of-two radix among the stages of
                               the two sub-FFT schedules (N2 and N1)           */
    int64_t batch_bytes;    /* device bytes the plan holds for batch calls:
                               the lanes' workspaces and the grid classes'
                               tables (workspace_bytes: the single-series
                               workspace and tables)                           */
} ls_plan_info;

/*
 * ls_plan: choose the NUFFT parameters for tolerance eps and nf frequencies
 * (Sec. 1: width and fine-grid size are matched to the user tolerance),
 * allocate the workspace on `device` and build the twiddle and deconvolution
 * tables.  Kernel: exp(beta (sqrt(1 - z^2) - 1)), |z| <= 1; at upsampling 2
 * w = ceil(log10(1/eps)) + 1 cells and beta = 2.30 w (see ls_plan_opts for
 * upsampling 1.5, which ls_plan may pick when it is cheaper).
 *   out      receives the plan handle (NULL on failure).
 *   max_nd   largest number of observations a later execute may pass (>= 2).
 *   nf       number of frequencies (>= 1); executes may use any nf' <= nf.
 *   eps      requested relative tolerance, 1e-14 <= eps <= 1e-1; LS_FP32
 *            needs eps >= 1e-7.
 *   prec     ls_prec.
 *   stream   cudaStream_t the plan launches on (NULL: the legacy default stream).
 * Returns LS_ERR_ARG, LS_ERR_UNSUPPORTED (grid beyond the two-pass FFT's size
 * limit), LS_ERR_NOMEM or LS_ERR_CUDA on failure.  Synchronises the device
 * once (table construction).
 */
ls_status ls_plan(ls_plan_t *out, int64_t max_nd, int64_t nf, double eps, int prec,
                  int device, void *stream);

/* Options of ls_plan_ex (zero-initialise for the defaults). */
typedef struct {
    /* Fine-grid upsampling factor sigma = n / nf: 0 lets the plan choose
     * (the cheaper of 2 and 1.5 by a cost model of grid cells plus kernel
     * evaluations), or exactly 2.0 or 1.5.  Sigma 1.5 needs eps >= 1e-10.
     * The kernel width grows as sigma falls: w = ceil(ln(1/eps) /
     * (pi sqrt(1 - 1/sigma))), beta = 0.976 pi (1 - 1/(2 sigma)) w. */
    double upsampling;
    /* Device memory ls_execute_batch may use for its workspace (fine grids and
     * point records of the series launched together); 0: half of the free
     * memory at the first batch call, at most 8 GiB.  Larger batches are cut
     * into launches that fit. */
    uint64_t batch_workspace_bytes;
    /* Fine-grid columns per pass-A block: the spreader's tile is this many
     * columns of n2 cells, and the bin sort's bins are this many columns wide.
     * 0 lets the plan choose (FP32: the widest of 8, 4, 2 whose two blocks
     * fit an SM; FP64: 2, else 1); 1, 2, 4 or 8 request a width.  A grid that
     * cannot use the request (fewer than two bins, or a block beyond the
     * opt-in shared memory) takes the automatic width; ls_plan_describe
     * reports the width taken.  Batch classes apply the same rule to their
     * own grids. */
    int32_t cols_per_block;
    /* Largest radix of the fine-grid FFT stages (each sub-FFT runs the odd
     * radices 9, 3, 5 first, then powers of two): 16 for radix-16 stages, 8
     * for radix-8 stages (more stages, lighter butterflies), for both
     * sub-FFTs; a pass-A column that would not fit with radix 8 keeps 16.
     * 0 lets the plan choose: radix 8 on the FP64 path; on the FP32 path
     * radix 16 for the columns (N2) and, for the rows (N1), radix 8 where it
     * adds no stage. */
    int32_t fft_max_radix;
} ls_plan_opts;

/* ls_plan with options (opts may be NULL: the defaults). */
ls_status ls_plan_ex(ls_plan_t *out, int64_t max_nd, int64_t nf, double eps, int prec,
                     int device, void *stream, const ls_plan_opts *opts);

/* Replace the stream later calls launch on (NULL: legacy default stream). */
ls_status ls_set_stream(ls_plan_t plan, void *stream);

/*
 * ls_execute: the periodogram of one series.
 *   t, y     nd observation times and values.
 *   dy       nd uncertainties (> 0), or NULL for unit weights.
 *   nd       2 <= nd <= the plan's max_nd.
 *   f0, df   grid f_k = f0 + k df; df > 0; both finite.
 *   nf       1 <= nf <= the plan's nf.
 *   eps      >= the plan's eps (the plan's accuracy is then sufficient).
 *   norm     an ls_norm value OR'ed with model flags (LS_NO_FIT_MEAN,
 *            LS_NO_CENTER); other bits: LS_ERR_UNSUPPORTED.
 *   power    nf outputs (standard normalisation: P_k in [0, 1]).
 * The inputs are taken as exact reals: the phases f t are reduced modulo one
 * cycle exactly, in 128-bit integer arithmetic on the mantissas, so a time
 * offset does not cost accuracy.
 */
ls_status ls_execute(ls_plan_t plan, const double *t, const double *y, const double *dy,
                     int64_t nd, double f0, double df, int64_t nf, double eps, int norm,
                     double *power);

/*
 * ls_execute_sums: as ls_execute, and also writes the six deconvolved sums of
 * Eq. 1 for every frequency, sums[6*k + {0..5}] = (Ch, Sh, C, S, C2, S2) with
 * Ch + i Sh = sum_j w^_j (y_j - ybar) e^{2 pi i f_k t_j},
 * C + i S = sum_j w^_j e^{2 pi i f_k t_j}, C2 + i S2 = sum_j w^_j e^{4 pi i f_k t_j}.
 * `power` may be NULL.  Meant for validating the NUFFT stage.  With
 * LS_NO_FIT_MEAN the transform of w^ at f is skipped and C, S are written as 0;
 * with LS_NO_CENTER, Ch and Sh use y instead of y - ybar.
 */
ls_status ls_execute_sums(ls_plan_t plan, const double *t, const double *y, const double *dy,
                          int64_t nd, double f0, double df, int64_t nf, double eps, int norm,
                          double *power, double *sums);

/*
 * ls_execute_batch: periodograms of nseries independent series (a ragged
 * batch: each series has its own times, values, uncertainties and frequency
 * grid), the many-series workload the paper's batched mode serves (Sec. 2,
 * "Performance").  Series whose frequency counts map to the same fine grid
 * run together: one launch per pipeline stage, the series on the grid's second
 * dimension, within the plan's batch workspace (ls_plan_opts); larger groups
 * are cut into several launches.  The launches are spread over four internal
 * streams (each with a quarter of the workspace) so that small groups overlap
 * on the device; the plan's stream waits for all of them before the call
 * returns, so the call is ordered on it like any other.  The plan supplies precision, tolerance,
 * upsampling, device and stream; its nf and max_nd do not limit the batch.
 *   offsets      host int64[nseries + 1]: series s owns points
 *                offsets[s] .. offsets[s+1]-1 of t, y and dy (>= 2 points).
 *   t, y, dy     device arrays of offsets[nseries] FP64 values (dy may be NULL).
 *   f0, df       host double[nseries]: grid of series s is f0[s] + k df[s].
 *   nf           host int64[nseries] (>= 1).
 *   out_offsets  host int64[nseries]: P_k of series s goes to
 *                power[out_offsets[s] + k], k < nf[s].
 *   eps          >= the plan's eps.  norm: as for ls_execute, for every series.
 *   power        device array.
 * Asynchronous like ls_execute with device buffers; a non-finite value,
 * dy <= 0 or a constant series in any series is reported by ls_sync.
 */
ls_status ls_execute_batch(ls_plan_t plan, int64_t nseries, const int64_t *offsets,
                           const double *t, const double *y, const double *dy, const double *f0,
                           const double *df, const int64_t *nf, const int64_t *out_offsets,
                           double eps, int norm, double *power);

/*
 * ls_execute_batch_shared: periodograms of nseries series observed at the same
 * times with the same uncertainties (a uniform batch, the case the paper's
 * batched mode names, Sec. 2).  The transforms of w^ at f and at 2f depend
 * only on t and dy, so they are taken once for the whole batch; each series
 * adds one transform (w^ (y - ybar) at f).
 *   t, dy        device, nd values each (dy may be NULL: unit weights).
 *   Y            device, nseries x nd values, series s at Y + s nd.
 *   f0, df, nf   the common grid f_k = f0 + k df, k < nf.
 *   power        device, nseries x nf values, series s at power + s nf.
 * Other arguments and the asynchronous behaviour as for ls_execute_batch.
 */
ls_status ls_execute_batch_shared(ls_plan_t plan, int64_t nseries, int64_t nd, const double *t,
                                  const double *Y, const double *dy, double f0, double df,
                                  int64_t nf, double eps, int norm, double *power);

/*
 * Prepared batches: the host work of a batch call done once for a fixed
 * layout, so repeated batches of new values pay only the kernels and a run can
 * be recorded by CUDA stream capture (a graph) and replayed.
 *
 * ls_batch_prepare takes the arguments of ls_execute_batch that fix the
 * layout (offsets, f0, df, nf, out_offsets, eps, norm; host arrays, read
 * during the call only), and ls_batch_prepare_shared those of
 * ls_execute_batch_shared (nseries, nd, f0, df, nf, eps, norm).  Preparation
 * validates the series, groups them by fine grid, builds each grid's tables,
 * splits the groups into launches within the plan's batch workspace budget,
 * allocates the workspaces of those launches and uploads the per-series
 * descriptors; the batch owns all of it (ls_batch_describe reports the
 * bytes).  Synchronous (table construction).
 *
 * ls_batch_run: the periodograms of the prepared layout for the values at t,
 * y, dy (device arrays laid out as for the matching execute call) into power
 * (device).  It enqueues kernels and memsets only (on the plan's stream and
 * its four batch streams, joined back into the plan's stream before it
 * returns): no allocation, no host-device copy, no host synchronisation.
 * Errors and the device status word behave as for ls_execute_batch.  Runs of
 * one batch, and runs and other calls on its plan, must not overlap on the
 * device (they share streams, the status word and, for one batch, its
 * workspaces); the plan must outlive the batch.
 *
 * ls_batch_destroy waits for the plan's streams and frees the batch.  A graph
 * recorded from ls_batch_run must not be replayed after that.  ls_destroy of
 * the plan releases the device memory of batches still prepared on it and
 * leaves their handles inert: ls_batch_run and ls_batch_describe then return
 * LS_ERR_ARG and ls_batch_destroy only frees the handle.
 */
typedef struct ls_batch_s *ls_batch_t;

ls_status ls_batch_prepare(ls_plan_t plan, ls_batch_t *out, int64_t nseries,
                           const int64_t *offsets, const double *f0, const double *df,
                           const int64_t *nf, const int64_t *out_offsets, double eps, int norm);
ls_status ls_batch_prepare_shared(ls_plan_t plan, ls_batch_t *out, int64_t nseries, int64_t nd,
                                  double f0, double df, int64_t nf, double eps, int norm);
ls_status ls_batch_run(ls_batch_t batch, const double *t, const double *y, const double *dy,
                       double *power);
/* Launches and grid classes of the batch, and the device bytes it owns (any
 * output pointer may be NULL). */
ls_status ls_batch_describe(ls_batch_t batch, int64_t *launches, int64_t *classes,
                            int64_t *bytes);
ls_status ls_batch_destroy(ls_batch_t batch);

/* Pipeline kernels this process has enqueued through the library so far
 * (recorded into a graph counts once, at recording; replays do not count):
 * the difference around a call is the number of kernels the call launched. */
ls_status ls_kernel_launches(int64_t *count);

/* Wait for the plan's stream; return and clear the device-side status of every
 * execute since the previous ls_sync (LS_ERR_ARG for invalid values,
 * LS_ERR_DEGENERATE for a constant series, else LS_OK). */
ls_status ls_sync(ls_plan_t plan);

/*
 * Stage timing with CUDA events recorded on the plan's stream around the
 * pipeline's kernels (tracing for roofline measurements).
 * ls_timing_enable(plan, 1) creates the events and starts accumulating; 0
 * destroys them.  Every later execute records one event set (a ring of 64;
 * an older set is drained first when the ring is full).
 * ls_timing_report waits for the recorded sets, writes the summed device
 * time in ms of each stage into ms[0 .. LS_NUM_STAGES-1] and the number of
 * executes into *count, and resets the sums.  Stages, in order:
 *   0 preprocess (weights, mean, phase reduction, point records),
 *   1 bin sort (scan + scatter), 2 pass A (spread + column FFTs),
 *   3 pass B (row FFTs + deconvolution + power).
 */
#define LS_NUM_STAGES 4
ls_status ls_timing_enable(ls_plan_t plan, int enable);
ls_status ls_timing_report(ls_plan_t plan, double *ms, int64_t *count);

/* Fill *info with the plan's parameters and the device bytes it holds. */
ls_status ls_plan_describe(ls_plan_t plan, ls_plan_info *info);

/*
 * ls_plan_reserve_batch: allocate the plan's batch workspaces now -- per
 * stream lane, the per-series arrays and an arena of a quarter of the batch
 * budget (ls_plan_opts.batch_workspace_bytes) -- and create the lane streams,
 * so that later ls_execute_batch / ls_execute_batch_shared calls whose
 * launches fit the budget allocate no device memory and wait for no
 * reallocation.  (A launch holding one series larger than a lane's share
 * still grows that lane's arena.)  Grid-class tables are still built on
 * first use of a class.  ls_plan_describe reports the bytes held
 * (batch_bytes).
 */
ls_status ls_plan_reserve_batch(ls_plan_t plan);

/* Release the plan and its device memory (synchronises its stream). */
ls_status ls_destroy(ls_plan_t plan);

/* Static description of a status code. */
const char *ls_status_str(ls_status s);

/*
 * Host-only queries (no GPU needed), used to check the plan's arithmetic.
 * ls_choose_params: the (w, beta, n, n1, n2, sigma) ls_plan_ex would choose
 * for max_nd observations and the requested upsampling (0: automatic).
 * ls_kernel_ft: phi_hat(k) = int phi(x) e^{i k x} dx of the ES kernel for
 * grid size n, in grid units: (w/2) int_{-1}^{1} psi(z) cos(pi k w z / n) dz,
 * by the same Gauss-Legendre rule the plan uses.
 */
ls_status ls_choose_params(int64_t nf, double eps, int prec, int64_t max_nd, double upsampling,
                           int32_t *width, double *beta, int64_t *n, int32_t *n1, int32_t *n2,
                           double *sigma);
double ls_kernel_ft(double k, int64_t n, int32_t width, double beta);

/*
 * ls_selftest_kernel_eval: runs, on `device`, the double-float evaluation of
 * the ES kernel psi(z) = exp(beta (sqrt(1 - z^2) - 1)) that the FP64 path's
 * spreading uses and the plain FP64 one, at n points evenly spaced on [-1, 1]
 * (2 <= n <= 2^24, 0 < beta < 100), and writes the largest absolute
 * difference to *max_abs_err (psi <= 1, so this is the error relative to the
 * kernel's peak, the scale the spreading error is measured on; near z = +-1
 * the relative error of either evaluation grows with 1/sqrt(1 - z^2)).
 * Synchronous; allocates 16 n bytes.
 */
ls_status ls_selftest_kernel_eval(double beta, int n, int device, double *max_abs_err);

/*
 * ls_selftest_double_assembly: checks, on `device`, the FP32 path's assembly
 * of the double-float power ratio hi + lo into a double on the integer pipe
 * (the power of Sec. 1 is written as FP64) against the FP64 conversions and
 * add it replaces, on n pairs (1 <= n <= 2^32) with |lo| <= ulp(hi)/2 drawn
 * from a counter-based generator seeded by `seed`: values over every exponent
 * and both signs, powers of two, the fast path's exponent bound, ties at the
 * double's rounding position, zero, subnormal and non-finite hi.  Writes the
 * number of pairs whose results differ in any bit to *mismatches (NaN against
 * NaN counts as equal).  Synchronous on the legacy default stream; allocates 8
 * bytes.
 */
ls_status ls_selftest_double_assembly(int64_t n, uint64_t seed, int device, int64_t *mismatches);

/*
 * ls_execute_noalloc: the periodogram of one small series without allocating
 * any memory.  The paper has no counterpart: this entry point exists for
 * callers that cannot allocate device memory -- programs whose device memory
 * belongs to another allocator (a framework's caching allocator) or to a fixed
 * arena, and loops that cannot afford the device-wide synchronisation that
 * cudaMalloc and cudaFree may bring -- and so cannot create an ls_plan.  It
 * runs the ls_execute pipeline on a fixed scratch area of
 * LS_NOALLOC_SCRATCH_BYTES that the library reserves in every GPU's memory
 * when it is loaded and keeps until the process exits.
 *   t, y, dy, power: device pointers (dy may be NULL); nd, f0, df, nf, eps and
 *   prec as for ls_plan/ls_execute (standard normalisation).  The tile width
 *   and FFT schedules are those a plan would choose for the request.
 *   Limits: nd <= LS_NOALLOC_MAX_ND, nf <= LS_NOALLOC_MAX_NF, and the request's
 *   workspace must fit the scratch area; otherwise LS_ERR_UNSUPPORTED and
 *   nothing is launched.  Host pointers: LS_ERR_ARG.
 * The call is synchronous on `stream` (NULL: legacy default stream): it
 * copies a small table from host memory, waits for the stream and returns the
 * device-side status (LS_ERR_ARG for non-finite values or dy <= 0,
 * LS_ERR_DEGENERATE for a constant series).  It therefore cannot be recorded
 * by stream capture.  The first call on a device looks up the scratch area's
 * device address and keeps it for the life of the process; do not call this
 * entry point on a device after cudaDeviceReset.  Every call reuses the same
 * scratch area and clears what must start at zero: calls whose work overlaps
 * on the GPU (other streams or host threads) race on it and must be
 * serialised by the caller.
 */
#define LS_NOALLOC_SCRATCH_BYTES (8u << 20)
#define LS_NOALLOC_MAX_ND 16384
#define LS_NOALLOC_MAX_NF 16384
ls_status ls_execute_noalloc(const double *t, const double *y, const double *dy, int64_t nd,
                             double f0, double df, int64_t nf, double eps, int prec,
                             double *power, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* NIFTY_LS_H */
