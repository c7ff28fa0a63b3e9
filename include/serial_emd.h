/*
 * serial_emd.h -- C ABI of the GB300 Serial-EMD library (libserial_emd.so).
 *
 * Serial-EMD (Zhang et al., arXiv 2106.15319) decomposes a multivariate series
 * or a 2D image by (1) serializing its N signals of length M into one 1D signal
 * of length L = MN + DN - D, joined by D-sample linear-blend transitions
 * (Sec. 3.1-3.2), (2) running 1D empirical mode decomposition on it: extrema,
 * cubic-spline envelopes, mean subtraction and a stop test, repeated per IMF
 * (Sec. 2.1, Eq. 1; EEMD Sec. 2.2), and (3) de-serializing the IMFs back to the
 * input's shape, dropping the transitions (Sec. 3.3).
 *
 * Every step runs in this library's CUDA kernels on one GPU. There is no CPU
 * fallback: when no usable GPU is present the calls return SEMD_ECUDA.
 *
 * Conventions for every entry point:
 *  - Pointers named d_* are device pointers; everything else is host memory.
 *  - Arrays are dense and row-major. An input of shape rows x cols holds its N
 *    signals as rows (SEMD_ORDER_ROWS: M = cols, N = rows; a channels x samples
 *    series or an image read row after row) or as columns (SEMD_ORDER_COLS:
 *    M = rows, N = cols).
 *  - The element type of inputs and IMF outputs follows the plan's precision:
 *    double for SEMD_FP64, float for SEMD_FP32_MIXED. Residues are always double.
 *  - IMF outputs are K x rows x cols (K = max_imfs); slots past the number of
 *    IMFs produced are zero-filled (the paper pads missing IMFs with zeros,
 *    Sec. 4.3, table of IMF counts).
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *  - The caller owns every buffer it passes and keeps it alive until the call's
 *    work has finished on the stream (or, for the server, until poll reports a
 *    final status). The library owns plans, servers and their workspaces.
 *  - No call aborts or exits. Each returns a semd_status; the text of the last
 *    error on a plan or server is returned by serial_emd_last_error().
 */
#ifndef SERIAL_EMD_H
#define SERIAL_EMD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum semd_status {
    SEMD_OK = 0,
    SEMD_PENDING = 1,      /* poll: the request is queued or running */
    SEMD_EINVAL = -1,      /* an argument is out of range or inconsistent */
    SEMD_ENOMEM = -2,      /* a device or host allocation failed */
    SEMD_EBUDGET = -3,     /* the work does not fit the plan's or server's byte budget */
    SEMD_ECUDA = -4,       /* a CUDA call failed (no device, launch error, ...) */
    SEMD_ETIMEOUT = -5,    /* a bounded wait ran out */
    SEMD_ECANCELED = -6,   /* the server was destroyed before the request finished */
    SEMD_EUNSUPPORTED = -7 /* a valid option that the library does not implement */
} semd_status;

typedef enum semd_order { SEMD_ORDER_ROWS = 0, SEMD_ORDER_COLS = 1 } semd_order;
typedef enum semd_stop { SEMD_STOP_FIXED = 0, SEMD_STOP_SD = 1, SEMD_STOP_SNUMBER = 2 } semd_stop;
typedef enum semd_spline_end { SEMD_SPLINE_NATURAL = 0, SEMD_SPLINE_NOT_A_KNOT = 1 } semd_spline_end;
typedef enum semd_boundary { SEMD_BOUNDARY_MIRROR = 0, SEMD_BOUNDARY_ENDPOINTS = 1 } semd_boundary;
typedef enum semd_precision { SEMD_FP64 = 0, SEMD_FP32_MIXED = 1 } semd_precision;

/*
 * Parameters of the method, following the paper's statement of the problem:
 *  rows, cols       shape of one input (the plan's capacity unit, see serial_emd_plan),
 *                   both >= 1, with a serialized length MN + DN - D below 2^30.
 *  order            which axis holds the N signals (see conventions above).
 *  transition_len   D of Sec. 3.2, 0 <= D <= M; -1 selects round(0.2 M), the
 *                   20 % rule of Sec. 4.1. A single signal (N = 1) takes D = 0.
 *  max_imfs         K, 1 <= K <= 32 (Sec. 3.3; the paper caps at 10 in Sec. 4.3).
 *  stop             SEMD_STOP_FIXED: exactly fixed_sifts sifts per IMF (1 to 1000).
 *                   SEMD_STOP_SD: sift until sum (h_prev - h)^2 / sum h_prev^2 <
 *                   sd_threshold (>= 0), at most max_sifts sifts (1 to 1000). Sec. 2.1
 *                   Step 5 leaves the criterion open ("some predefined stopping
 *                   criterion").
 *                   SEMD_STOP_SNUMBER: the S-number rule of the EMD literature: sift
 *                   until s_number consecutive sifts have each left a signal whose
 *                   extrema count (maxima + minima) and zero-crossing count differ by
 *                   at most one, at most max_sifts sifts (1 to 1000).
 *  boundary         envelope end rule (the paper is silent): MIRROR reflects the
 *                   first and last mirror_knots (1 or 2) extrema about the ends;
 *                   ENDPOINTS adds the two end samples as knots.
 *  precision        SEMD_FP64: FP64 end to end. SEMD_FP32_MIXED: sifting in FP32,
 *                   FP64 in the cross-tile spline interface solve, the stop
 *                   reductions, the residue and the EEMD average.
 *  ensemble_trials  <= 1: EMD. > 1: EEMD with that many noise realizations (Sec. 2.2);
 *                   such plans also run CEEMDAN (serial_emd_ceemdan).
 *  noise_rel_std    (>= 0 when ensemble_trials > 1) EEMD beta = noise_rel_std *
 *                   population std of the serialized x;
 *                   CEEMDAN beta_k = noise_rel_std * population std of the residue r_k.
 *  s_number         S of SEMD_STOP_SNUMBER, 1 <= S <= 1000.
 *  spline_end       end conditions of the envelope splines: SEMD_SPLINE_NATURAL (zero
 *                   second derivative at the first and last knot of the sequence,
 *                   boundary knots included) or SEMD_SPLINE_NOT_A_KNOT (continuous third
 *                   derivative at the second and second-to-last knot; sequences of fewer
 *                   than four knots keep natural ends). The paper names the cubic spline
 *                   of standard EMD (Sec. 1) without its end conditions.
 */
typedef struct semd_params {
    int64_t rows;
    int64_t cols;
    int32_t order;
    int32_t transition_len;
    int32_t max_imfs;
    int32_t stop;
    int32_t fixed_sifts;
    int32_t max_sifts;
    double sd_threshold;
    int32_t boundary;
    int32_t mirror_knots;
    int32_t precision;
    int32_t ensemble_trials;
    double noise_rel_std;
    int32_t s_number;
    int32_t spline_end;
} semd_params;

/* Fills p with the defaults: ROWS order, D = -1 (20 % rule), K = 10, fixed 10 sifts,
 * SD threshold 0.2 with at most 50 sifts, S-number 4, MIRROR with 2 knots, natural
 * spline ends, FP32_MIXED, EMD. */
void serial_emd_default_params(semd_params *p);

typedef struct semd_plan_s *semd_plan_t;

/*
 * Creates a plan: validates params and reserves every device workspace up front,
 * so that the decompose calls allocate nothing. Capacity: up to max_batch inputs
 * of at most params->rows x params->cols elements each (for EEMD, one input and
 * ensemble_trials realizations). mem_budget > 0 caps the workspace bytes
 * (SEMD_EBUDGET if it does not fit); 0 means no cap. On success *out owns the
 * plan until serial_emd_destroy. Errors: EINVAL, EBUDGET, ENOMEM, ECUDA.
 */
semd_status serial_emd_plan(const semd_params *params, int max_batch, size_t mem_budget,
                            semd_plan_t *out);

/* Bytes of device workspace the plan holds. */
size_t serial_emd_plan_bytes(semd_plan_t plan);

/*
 * Serial-EMD of one input of the plan's shape (Sec. 3: serialize, EMD or EEMD,
 * de-serialize), enqueued on `stream`.
 *  d_x        input, rows x cols (plan precision).
 *  d_noise    EEMD only: ensemble_trials x L white-noise realizations w^(m)
 *             (plan precision, L = MN + DN - D), or NULL: the library then draws the
 *             noise itself, on the device, from the plan's noise seed
 *             (serial_emd_plan_set_noise_seed): sample p of realization m is word
 *             p mod 4 of the Philox4x32-10 block (Salmon et al., SC 2011) with counter
 *             (p div 4, m, 0, 0) and key (seed low, seed high), mapped from the word u
 *             to (2 (u >> 9) - (2^23 - 1)) * sqrt(3) / 2^23 in FP64: white noise,
 *             uniform with zero mean and unit variance. Ignored for EMD.
 *  d_imfs     output, K x rows x cols (plan precision); for EEMD the trial average.
 *  d_residue  output, rows x cols doubles; may be NULL.
 *  n_imfs     host; if not NULL the call waits for the stream and stores the IMF
 *             count (for EEMD the largest count over the trials). If NULL the call
 *             returns without waiting and serial_emd_plan_counts() gives the counts
 *             after the stream has finished.
 * The plan may not be used by two calls at once. Errors: EINVAL, ECUDA.
 */
semd_status serial_emd_decompose(semd_plan_t plan, const void *d_x, const void *d_noise,
                                 void *d_imfs, double *d_residue, int *n_imfs, void *stream);

/* Seed of the white noise the library draws for EEMD calls that pass no noise (default
 * 0). Takes effect at the next call. Errors: EINVAL (NULL plan). */
semd_status serial_emd_plan_set_noise_seed(semd_plan_t plan, uint64_t seed);

/* One input of a batch: its own shape (within the plan's capacity) and buffers. */
typedef struct semd_instance {
    const void *d_x;   /* rows x cols input (plan precision) */
    int64_t rows;
    int64_t cols;
    void *d_imfs;      /* K x rows x cols output (plan precision) */
    double *d_residue; /* rows x cols doubles, or NULL */
} semd_instance;

/*
 * Serial-EMD of `count` independent inputs of different shapes in one batched run:
 * every pass over the signals covers all inputs at once. Each input's result is
 * bit-identical to decomposing it alone. count <= max_batch and the summed
 * serialized lengths must fit the plan (EBUDGET otherwise). EMD plans only
 * (EINVAL for EEMD plans). n_imfs: host array of `count`, or NULL (see decompose).
 */
semd_status serial_emd_decompose_batch(semd_plan_t plan, int count, const semd_instance *inst,
                                       int *n_imfs, void *stream);

/*
 * Slice-wise standard EMD, the baseline of the paper's experiments (Sec. 4: the standard
 * one-dimensional EMD applied to the input as a collection of one-dimensional slices):
 * each of the `rows` signals of a row-major rows x cols input (plan precision) is
 * decomposed on its own, without serialization or transitions, all in one batched run
 * with the same kernels. d_imfs: K x rows x cols (IMF k of signal i at
 * k*rows*cols + i*cols, zero past the signal's IMF count); d_residue: rows x cols
 * doubles, or NULL; n_imfs: host array of `rows`, or NULL (see decompose). The plan must
 * be an EMD plan whose serialized length holds one signal (cols samples) and whose
 * max_batch is at least `rows`; EBUDGET otherwise, EINVAL for EEMD plans. Results equal
 * those of decompose_batch on the rows taken one by one.
 */
semd_status serial_emd_decompose_slices(semd_plan_t plan, const void *d_x, int64_t rows,
                                        int64_t cols, void *d_imfs, double *d_residue,
                                        int *n_imfs, void *stream);

/*
 * Serial-CEEMDAN of one input of the plan's shape (Sec. 3 with the CEEMDAN of Sec. 2.2,
 * Steps 1-4, as the decomposition), enqueued on `stream`. The plan must be an ensemble
 * plan (ensemble_trials = T >= 2, max_batch 1); EINVAL otherwise. With r_0 the serialized
 * input and E_k(w) the k-th EMD mode of a noise realization w (zero past its mode count;
 * the EMD uses the plan's stop rule and boundary), stage k = 0 .. K-1 runs while r_k has
 * at least one maximum, one minimum and three extrema: beta_k = noise_rel_std * population
 * std of r_k, mode k+1 = the average over the T trials of the first EMD mode of
 * r_k + beta_k w^(m) (k = 0: the first EEMD mode, Step 1) or of r_k + beta_k E_k(w^(m))
 * (k >= 1, Steps 2 and 4), and r_{k+1} = r_k - mode (Step 3), in FP64.
 *  d_x        input, rows x cols (plan precision).
 *  d_noise    T x L white-noise realizations w^(m) (plan precision, L = MN + DN - D).
 *  d_modes    output, K x rows x cols (plan precision), zero past the mode count.
 *  d_residue  output, rows x cols doubles (the final r), or NULL.
 *  n_modes    host; if not NULL the call waits for the stream and stores the mode count;
 *             if NULL, serial_emd_plan_counts() gives it after the stream has finished.
 * Inputs and outputs stay owned by the caller and must stay valid until the stream has
 * finished. The plan may not be used by two calls at once. Errors: EINVAL, ECUDA.
 */
semd_status serial_emd_ceemdan(semd_plan_t plan, const void *d_x, const void *d_noise,
                               void *d_modes, double *d_residue, int *n_modes, void *stream);

/*
 * One realization of the plan's last EEMD call (Sec. 2.2: realization m is the EMD of
 * x + beta w^(m), serialized as in Sec. 3.2), for callers that need the ensemble's spread
 * and not only its average: writes its IMFs de-serialized to d_imfs (K x rows x cols,
 * plan precision, zero past the realization's IMF count) and, if d_residue is not NULL,
 * its residue (rows x cols doubles), enqueued on `stream`. If n_imfs or beta (host) is
 * not NULL the call waits for the stream and stores the realization's IMF count and the
 * beta of that call. The plan must be an ensemble plan whose last call was
 * serial_emd_decompose; trial in [0, ensemble_trials). Errors: EINVAL, ECUDA.
 */
semd_status serial_emd_eemd_trial(semd_plan_t plan, int trial, void *d_imfs, double *d_residue,
                                  int *n_imfs, double *beta, void *stream);

/* After the stream has finished: IMF counts (count entries) and sifts per IMF
 * (count x K entries, may be NULL) of the plan's last decompose call (for a CEEMDAN
 * call: the mode count, and zero sifts). */
semd_status serial_emd_plan_counts(semd_plan_t plan, int count, int *n_imfs, int *sifts);

/*
 * Step-level entry points (Sec. 2.1 Step 1 and Steps 1-4 on an already
 * serialized signal), for unit tests and for callers that sift themselves.
 * serial_emd_extrema: d_h has L elements (plan precision); writes the ascending
 * indices of the maxima to d_tmax and of the minima to d_tmin (int32, capacity L/2+1
 * each) and their counts to the host ints n_max / n_min (waits for the stream).
 * Rule: maximum at k iff h[k-1] < h[k] >= h[k+1], minimum iff h[k-1] > h[k] <=
 * h[k+1], for 1 <= k <= L-2.
 * serial_emd_sift: one sift of d_h into d_out (L elements each); returns through
 * the host pointers the sums (h - h')^2 and h^2. SEMD_EINVAL if either kind of
 * extremum is missing. L must not exceed the plan's serialized length.
 */
semd_status serial_emd_extrema(semd_plan_t plan, const void *d_h, int64_t L, int32_t *d_tmax,
                               int32_t *d_tmin, int64_t *n_max, int64_t *n_min, void *stream);
semd_status serial_emd_sift(semd_plan_t plan, const void *d_h, int64_t L, void *d_out,
                            double *sd_num, double *sd_den, void *stream);

/*
 * Allocation-free form of serial_emd_sift, for callers that cannot reserve device
 * memory at the point where they sift: plug-ins hosted by a framework whose caching
 * allocator owns the device memory (a cudaMalloc of their own would fight it for the
 * same bytes), real-time paths that forbid allocation after start-up, and code that
 * runs under a hard device-memory cap where an allocation could fail mid-stream. The
 * paper has no counterpart; it is a packaging of the same sift.
 * It performs exactly the sift of serial_emd_sift (same kernels, same results) on
 * d_h (L elements of the precision in params->precision) into d_out (L elements),
 * with the envelope rule of params->boundary / params->mirror_knots and the spline
 * end conditions of params->spline_end (each validated as serial_emd_plan validates
 * it; SEMD_EINVAL otherwise); the other fields of params are ignored.
 * The call waits for `stream`: it copies the sums (h - h')^2 and h^2 back to the host
 * pointers and synchronizes the stream before it returns.
 * Scratch: one static device array of about 2.4 MB, compiled into the library, which
 * every GPU that loads the library holds until the process exits; nothing is
 * allocated per call (no cudaMalloc, cudaFree or allocating library routine). L
 * must be in [1, 65536]: a larger L returns SEMD_EINVAL with a message naming the
 * limit. The first call on a device looks up the array's device address and sets
 * kernel attributes for that device; make that first call before any stream capture
 * begins. All calls share the one array and each call clears what it needs, so two
 * calls whose work overlaps on the GPU (different streams or threads) race and give
 * wrong results: serialize them. Errors (EINVAL, ECUDA) are described by
 * serial_emd_last_error(NULL) called on the same host thread: the message of a call
 * without a plan is kept per thread.
 */
semd_status serial_emd_sift_noalloc(const semd_params *params, const void *d_h, int64_t L,
                                    void *d_out, double *sd_num, double *sd_den, void *stream);

/*
 * Execution options of a plan. use_graphs (default 1): a decomposition with a fixed
 * sift count is captured once into a CUDA graph (per batch layout) and replayed on
 * the plan's own stream, joined to the caller's stream by events; the first call for
 * a new layout must not itself be under stream capture. profile (default 0): the
 * pass and reduce kernels are bracketed by CUDA events (graphs are then not used),
 * and serial_emd_plan_stats() reports their summed device time.
 */
semd_status serial_emd_plan_set_options(semd_plan_t plan, int use_graphs, int profile);

/*
 * Tile of the sifting pass kernel: every pass cuts each serialized signal into tiles of
 * `tile` samples (128, 256 or 512; one warp each, tile / 32 samples per lane), and the
 * spline system is partitioned at tile edges. 0 restores the plan's own choice (the
 * tuning table's entry for the plan, else 256). The tile changes rounding only (results
 * agree to the precision's tolerance), and the speed: small tiles spread short signals
 * over more warps, large ones shrink the interface system. Takes effect at the next
 * decompose call. Errors: EINVAL.
 */
semd_status serial_emd_plan_set_tile(semd_plan_t plan, int tile);
/* The plan's current tile (0 for a NULL plan). */
int serial_emd_plan_get_tile(semd_plan_t plan);

/*
 * CTAs per SM of the pass kernel's persistent grid: 0 (the default) keeps as many as fit,
 * n > 0 at most n. Changes speed only. Takes effect at the next call. Errors: EINVAL
 * (outside [0, 64]).
 */
semd_status serial_emd_plan_set_pass_ctas(semd_plan_t plan, int ctas_per_sm);
/* The plan's current setting (0 for a NULL plan). */
int serial_emd_plan_get_pass_ctas(semd_plan_t plan);

/*
 * Variant of the pass kernel. 0 (default, throughput): each warp copies its next tile's
 * signal and interface values into shared memory (asynchronous copies) while the current
 * tile computes; for FP32 with 256-sample tiles it is compiled for four resident CTAs per
 * SM. 1 (latency): no staging, a smaller kernel, for launches with about one tile per
 * warp; for FP32 with 256-sample tiles compiled for three CTAs per SM without register
 * spills. Changes speed only. Errors: EINVAL (not 0 or 1).
 */
semd_status serial_emd_plan_set_pass_variant(semd_plan_t plan, int variant);
int serial_emd_plan_get_pass_variant(semd_plan_t plan);

/* ------------------------------------------------------------------ autotuner */

typedef struct semd_tune_result {
    int32_t tile;        /* chosen tile (samples per warp) */
    int32_t ctas_per_sm; /* chosen CTAs per SM of the pass grid (0: as many as fit) */
    double ms;           /* median device time of one decomposition with the choice */
    double ms_default;   /* the same with the default shape (tile 256, variant 0, all CTAs) */
    int32_t candidates;  /* shapes timed */
    int32_t variant;     /* chosen register budget (see serial_emd_plan_set_pass_variant) */
} semd_tune_result;

/*
 * Times the plan's decomposition of `count` inputs (as serial_emd_decompose_batch takes
 * them; for an ensemble plan one input and its noise, or NULL noise to let the library
 * draw it, as serial_emd_decompose) for every
 * pass-kernel shape: tile 128, 256 or 512, the register budget where the kernel has two,
 * and CTAs per SM of the persistent grid (as many as fit, or fewer). Each shape runs once untimed, then `repeats` times (1..100)
 * with CUDA events on `stream`; the median counts. The fastest shape is kept on the plan
 * and entered in the process-wide tuning table under the plan's key: precision, stop
 * rule, ensemble or not, ceil(log2) of the instance count (trials for an ensemble) and
 * of the longest serialized length. Plans created later with that key start with it.
 * The outputs are overwritten; the call waits for the stream. out may be NULL.
 * Errors: EINVAL, EBUDGET (an input larger than the plan), ECUDA.
 */
semd_status serial_emd_plan_autotune(semd_plan_t plan, int count, const semd_instance *inst,
                                     const void *d_noise, int repeats, semd_tune_result *out,
                                     void *stream);

/* The tuning table's shape for a plan of these params, longest serialized length L and
 * ninst instances: SEMD_OK and *tile, *ctas_per_sm, *variant set, or SEMD_PENDING when the
 * table has no entry. EINVAL for bad arguments. Host only. */
semd_status serial_emd_tune_lookup(const semd_params *params, int64_t L, int ninst, int *tile,
                                   int *ctas_per_sm, int *variant);
/* Empties the tuning table. */
void serial_emd_tune_clear(void);
/* Writes the table as JSON (an "entries" list of flat objects with the key fields,
 * "tile", "ctas_per_sm", "variant" and "ms"). Errors: EINVAL (see
 * serial_emd_tune_last_error). */
semd_status serial_emd_tune_save(const char *path);
/* Merges a file written by serial_emd_tune_save into the table; entries with missing
 * fields or an invalid shape are skipped. Errors: EINVAL (unreadable, no "entries"). */
semd_status serial_emd_tune_load(const char *path);
/* Text of the last save/load error of this thread. */
const char *serial_emd_tune_last_error(void);

/* Statistics of the plan's last decompose call; valid once its stream has finished. */
typedef struct semd_stats {
    int64_t kernel_launches; /* kernels the call ran (inside the graph when used_graph) */
    int64_t pass_launches;   /* profiled pass-kernel launches (0 unless profiling) */
    double pass_ms;          /* their summed device time */
    int64_t reduce_launches; /* profiled interface-solve launches */
    double reduce_ms;
    int64_t sample_sifts;    /* serialized samples x sifts performed */
    int64_t pass_bytes;      /* algorithmic HBM bytes of the pass kernel: per sample, the
                                signal in and out (2w), plus w + 16 for a commit (IMF out,
                                FP64 residue in and out); 8 + w for the first pass */
    int32_t used_graph;
    int32_t _reserved;
} semd_stats;

semd_status serial_emd_plan_stats(semd_plan_t plan, semd_stats *out);

/*
 * Per-launch device times of the plan's last decompose call when it ran with profiling
 * on (serial_emd_plan_set_options): kind 0 the sifting pass launches, kind 1 the interface
 * solves, in launch order, in milliseconds (CUDA events around each launch on its stream).
 * Writes at most cap values to the host array ms (may be NULL) and returns the number of
 * launches of that kind, or -1 for a NULL plan, an unknown kind or cap < 0. Waits for the
 * events. Pass launch i of a fixed-sift-count EMD runs, for i >= 1, IMF (i - 1) / S + 1
 * and sift (i - 1) % S + 1 (S sifts per IMF; the last sift of an IMF also commits it);
 * launch 0 reads the serialized input.
 */
int64_t serial_emd_plan_launch_times(semd_plan_t plan, int kind, float *ms, int64_t cap);

/*
 * Measured fused-multiply-add rate of the current GPU in the arithmetic of `precision`
 * (SEMD_FP64: double, SEMD_FP32_MIXED: float), in GFLOP/s (2 flops per FMA): a probe kernel
 * of independent register-resident FMA chains (iters per chain, e.g. 4096), timed with
 * CUDA events on `stream`; waits for the stream. It is the arithmetic peak against which
 * the plain FP64 form, bound by GB300's narrow FP64 pipe, is reported. Allocates a small
 * output buffer (stream-ordered) and changes no GPU setting. Errors: EINVAL, ECUDA.
 */
semd_status serial_emd_fma_rate(int precision, int iters, double *gflops, void *stream);

/*
 * How the interface solve (the reduced spline system of Sec. 2.1 Step 2, partitioned by
 * tiles) is run on the current GPU for a precision and spline-end rule: instances of
 * *min_tiles to *max_tiles tiles are solved by a thread-block cluster of *cluster CTAs per
 * envelope (distributed shared memory), all others by one CTA per envelope (in shared
 * memory while the system fits there, past *max_tiles with a global-memory scratch).
 * *cluster = 0 (and the range 0..0) when clusters are not used (not-a-knot ends, or a
 * device without clusters of 8 or 16 CTAs). The choice depends on an instance's tile
 * count alone, never on the other instances of a batch. Sets the kernel attributes on the
 * current device. Errors: EINVAL (NULL output, unknown precision or rule), ECUDA.
 */
semd_status serial_emd_interface_solve_shape(int precision, int spline_end, int *cluster,
                                             int64_t *min_tiles, int64_t *max_tiles);

/* Releases a plan and its workspaces (after its work on any stream has finished). */
void serial_emd_destroy(semd_plan_t plan);

/* Text of the last error on a plan; with NULL, of the last failed call without a plan
 * (plan creation, serial_emd_sift_noalloc) on the calling host thread. */
const char *serial_emd_last_error(semd_plan_t plan);

/* ------------------------------------------------------------------ serving */

/*
 * A server decomposes requests of different shapes as they arrive (continuous
 * batching): a host thread admits queued requests whenever slots and the byte
 * budget allow, runs a few passes of the sifting loop over every admitted request at
 * once, and retires requests as they finish, so new ones join while others are on
 * the GPU. Per-request results are identical to decomposing the request alone.
 * Requests of at least 2^21 serialized samples run in a second lane with its own host
 * thread and a lower-priority stream, whose pass launches keep to two CTAs per SM, so
 * that they run beside the small requests' passes instead of lengthening them; that
 * lane holds max(1, max_inflight / 8) requests at a time. Both lanes share the byte
 * budget.
 *  defaults     method parameters; rows/cols give the largest accepted request
 *               (its serialized length must not exceed that of rows x cols).
 *  mem_budget   device bytes the server may hold for request state (> 0).
 *  max_inflight most requests on the GPU at once (>= 1).
 * EEMD is not served (EUNSUPPORTED). Errors: EINVAL, ENOMEM, ECUDA.
 */
typedef struct semd_server_s *semd_server_t;

semd_status serial_emd_server_create(const semd_params *defaults, size_t mem_budget,
                                     int max_inflight, semd_server_t *out);

typedef struct semd_request {
    const void *d_x;   /* rows x cols input (server precision) */
    int64_t rows;
    int64_t cols;
    int32_t order;     /* SEMD_ORDER_ROWS / SEMD_ORDER_COLS */
    int32_t _reserved;
    void *d_imfs;      /* K x rows x cols output (server precision) */
    double *d_residue; /* rows x cols doubles, or NULL */
} semd_request;

typedef struct semd_result {
    int32_t status;     /* SEMD_OK, or the error that ended the request */
    int32_t n_imfs;
    int64_t sifts;      /* total sifts over all IMFs */
    double queue_ms;    /* submit -> admission */
    double run_ms;      /* admission -> outputs written */
} semd_result;

/* Queues a request; *ticket identifies it. EBUDGET if it could never fit. */
semd_status serial_emd_submit(semd_server_t server, const semd_request *req, uint64_t *ticket);

/* Non-blocking: SEMD_PENDING while the request is queued or running; otherwise
 * fills *out (once) and returns SEMD_OK. EINVAL for an unknown ticket. */
semd_status serial_emd_poll(semd_server_t server, uint64_t ticket, semd_result *out);

/* Blocking form of serial_emd_poll with a time limit: waits up to timeout_ms (>= 0) for
 * the request to finish, then fills *out (once) and returns SEMD_OK, or returns
 * SEMD_ETIMEOUT with the request still pending (it may be waited for again). EINVAL for
 * an unknown ticket or a negative limit. */
semd_status serial_emd_wait(semd_server_t server, uint64_t ticket, double timeout_ms,
                            semd_result *out);

/* Stops the server thread; unfinished requests end with SEMD_ECANCELED. */
void serial_emd_server_destroy(semd_server_t server);

const char *serial_emd_server_last_error(semd_server_t server);

#ifdef __cplusplus
}
#endif
#endif /* SERIAL_EMD_H */
