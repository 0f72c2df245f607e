/*
 * mrf.h -- C ABI of the GB300 (sm_103a) MRF dictionary generating and
 * searching (DGS) library.
 *
 * Method: Z. Wang, "MRF-ZOOM: A Fast Dictionary Searching Algorithm for
 * Magnetic Resonance Fingerprinting". A fingerprint is the Bloch-simulated
 * transverse signal of an IR-bSSFP train (Appendix, Eq. A2); a voxel's
 * acquired fingerprint is matched to the dictionary entry of highest complex
 * correlation (Theory, Eq. 1), by brute force over a (T1, T2, df) grid or by
 * the MRF-ZOOM coordinate search (Theory; Methods, Experiment 2).
 *
 * Conventions for every entry point:
 *   - Return value: MRF_OK (0), MRF_PENDING (1, serving only) or a negative
 *     MRF_E_* code. Nothing throws across this boundary. mrf_last_error()
 *     returns a message for the calling thread's most recent failure.
 *   - Units: milliseconds for times and T1/T2, Hz for off-resonance df,
 *     radians for angles.
 *   - Complex data are interleaved (re, im) float32 pairs ("complex64").
 *   - Pointers named *_dev are device pointers on the context's device; the
 *     caller owns them and keeps them alive until the stream reaches the
 *     call. Pointers named *_host are host memory owned by the caller.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream). Calls that
 *     take a stream are asynchronous on it unless stated otherwise.
 *   - Objects returned through `**out` (sequence, dictionary) are owned by the
 *     library and released with the matching *_free call.
 *   - Invalid arguments return MRF_E_INVALID and leave outputs untouched.
 *   - No CPU fallback exists: every computation runs in this library's CUDA
 *     kernels for sm_103a; without a usable device calls return MRF_E_CUDA.
 */
#ifndef MRF_H
#define MRF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    MRF_OK = 0,
    MRF_PENDING = 1,
    MRF_E_INVALID = -1,     /* bad argument, descriptor or state */
    MRF_E_NOMEM = -2,       /* device or host allocation failed */
    MRF_E_BUDGET = -3,      /* would exceed the context's HBM budget */
    MRF_E_TIMEOUT = -4,     /* a bounded wait ran out (host poll or device spin) */
    MRF_E_CUDA = -5,        /* CUDA runtime / driver error */
    MRF_E_NOTFOUND = -6,    /* unknown ticket or handle */
    MRF_E_UNSUPPORTED = -7  /* valid request the library does not implement */
};

typedef enum {
    MRF_F32 = 0,      /* FP32-class: the raw FP32 entries (per-entry scale 1 / ||d||)
                         stored as fp16 (x 2^15) plus e4m3 planes of the values (x 2^8)
                         and of the fp16 residuals (x 2^19); the voxels alike (fp16
                         x 2^12). Each product is the fp16 product plus the two e4m3
                         products of each residual with the other operand (at most
                         about 2^-13 |x_j d_j| per term, rms about 2^-16), the e4m3
                         ones accumulated first. Generated tiles (mrf_match_bruteforce_fused)
                         use bf16 hi + lo with three products (hi.hi + hi.lo + lo.hi). */
    MRF_BF16 = 1,     /* normalised entries rounded to bf16 (nearest even), scale 1 */
    MRF_FP8E4M3 = 2   /* normalised entries scaled to max |value| = 448 per entry,
                         stored as fp8 e4m3 with an fp32 per-entry scale */
} mrf_dtype;

typedef struct mrf_ctx mrf_ctx;
typedef struct mrf_seq mrf_seq;
typedef struct mrf_dict mrf_dict;

/* Thread-local message of the calling thread's last failing call ("" if none). */
const char *mrf_last_error(void);

/* Library version string, e.g. "mrf-gb300 1.0 sm_103a". */
const char *mrf_version(void);

/* Create a context on CUDA device `device`. `hbm_budget_bytes` caps the
 * device memory the library itself allocates for this context (sequences,
 * dictionaries, tables, scratch, serving buffers); 0 means "free memory at
 * creation". The library allocates nothing outside the budget and returns
 * MRF_E_BUDGET instead. Errors: MRF_E_INVALID (no such device, not sm_103),
 * MRF_E_CUDA. */
int mrf_ctx_create(int device, size_t hbm_budget_bytes, mrf_ctx **out);

/* Destroy a context: stops serving, waits for its work, frees everything it owns. */
void mrf_ctx_destroy(mrf_ctx *ctx);

/* Device bytes currently charged to the context's budget, and the budget. */
int mrf_ctx_memory(const mrf_ctx *ctx, size_t *used_bytes, size_t *budget_bytes);

/* Synchronise `stream` and report device-side failures of the context's
 * kernels since the last check: MRF_E_TIMEOUT when a kernel's bounded wait ran
 * out (the kernel returned early, its outputs are invalid, the context stays
 * usable); MRF_E_CUDA when a device-side index check failed (the access was
 * skipped; ZOOM and refinement check their grid points in every build, the
 * bounds-checked build compiled with -DMRF_CHECK checks the dictionary and
 * re-score kernels as well). The flag is cleared on report. Asynchronous entry
 * points report such failures only here. */
int mrf_stream_sync(mrf_ctx *ctx, void *stream);

/* Kernel accounting (no counterpart in the paper; used to measure the
 * kernels against their rooflines). Launch counts are always kept. With
 * profiling enabled, CUDA events are recorded on the launching stream around
 * the dictionary-generation, matcher and ZOOM kernels, and their durations
 * accumulate into the *_ms fields. zoom_* covers a whole on-the-fly ZOOM
 * search (all its kernels); zoomline_* the batched step-3 kernel within it. */
typedef struct {
    uint64_t launches;            /* every kernel this context launched */
    uint64_t dictgen_launches, matcher_launches, zoom_launches;
    double dictgen_ms, matcher_ms, zoom_ms;   /* event-timed launches only */
    uint64_t dictgen_timed, matcher_timed, zoom_timed;
    uint64_t zoomline_launches;
    double zoomline_ms;
    uint64_t zoomline_timed;
    /* work of the batched step-3 kernel, always counted: df positions
     * evaluated (voxel, candidate pairs) and candidates simulated */
    uint64_t zoomline_pairs, zoomline_entries;
    /* the packed on-the-fly ZOOM kernel: warp rounds, candidates simulated,
     * and the most rounds one voxel spent in flight within a launch */
    uint64_t zoom_rounds, zoom_candidates, zoom_max_voxel_rounds;
} mrf_profile;
/* on != 0 starts recording the CUDA events behind the *_ms fields, 0 stops
 * it (launch counts and work counters are kept either way). */
int mrf_profile_enable(mrf_ctx *ctx, int on);
/* Synchronises the device (pending profile events, work counters). reset != 0
 * zeroes all counters. */
int mrf_profile_read(mrf_ctx *ctx, mrf_profile *out, int reset);

/* The FP32 FMA rate this device sustains (the roofline of the on-the-fly
 * Bloch and ZOOM kernels): a kernel of independent FMA chains on every SM,
 * timed with CUDA events, best of three; *tflops = 2 x FMAs / time. Takes a
 * few milliseconds and synchronises the device. */
int mrf_fp32_fma_rate(mrf_ctx *ctx, double *tflops);

/* The dense tensor-core rate of the matcher's MMA shape (the roofline of the
 * BF16 and FP8 brute-force forms): tcgen05.mma kind::f16 (bf16) or
 * kind::f8f6f4 (e4m3), M = 128, N = 256, FP32 accumulation in TMEM, operands
 * resident in 128-byte-swizzled shared memory, one CTA per SM issuing
 * back-to-back MMAs; timed with CUDA events, best of three after a warm-up;
 * *tflops = 2 M N K x MMAs / time. precision: MRF_BF16 or MRF_FP8E4M3. Takes
 * some tens of milliseconds and synchronises the library's stream. Errors:
 * MRF_E_INVALID, MRF_E_CUDA (a wait that timed out is reported by
 * mrf_stream_sync). */
int mrf_mma_rate(mrf_ctx *ctx, int32_t precision, double *tflops);

/* ------------------------------------------------------------------------ */
/* Sequence (Methods: IR-bSSFP train; Appendix: hard RF pulse)              */

/* Acquisition train of n timepoints. For timepoint j the simulator applies
 * the RF pulse, evolves TE_j, samples s_j = Mx + i My, then evolves TR_j -
 * TE_j. A hard pulse (tau_j = 0) is R_z(phi_j) R_x(-alpha_j) R_z(-phi_j)
 * (Appendix, small-beta form). A pulse of duration tau_j > 0 is the
 * Appendix's off-resonant form R_z(phi) R_y(beta) R_x(alpha') R_y(-beta)
 * R_z(-phi) for each candidate's df: beta = atan2(tau dw, alpha) is the angle
 * of the effective field from the x axis and alpha' = -sqrt(alpha^2 + (tau
 * dw)^2) the rotation about it over the pulse, dw = 2 pi df / 1000 rad/ms
 * (the printed arctangent for alpha > 0; the Appendix's Delta-t in alpha' is
 * the pulse duration). No relaxation acts during a pulse; TE_j and TR_j are
 * counted from the pulse. With inversion != 0 an ideal 180 degree pulse about
 * x and inv_delay_ms of free evolution come first. Equilibrium magnetisation
 * M0 = 1. */
typedef struct {
    int32_t n;                   /* timepoints, >= 1 */
    const double *flip_rad;      /* n signed flip angles alpha_j */
    const double *rf_phase_rad;  /* n RF phases phi_j, or NULL for all zero */
    const double *tr_ms;         /* n repetition times, > 0 */
    const double *te_ms;         /* n echo times, 0 <= TE_j <= TR_j */
    int32_t inversion;           /* 0 or 1 */
    double inv_delay_ms;         /* >= 0 */
    const double *pulse_ms;      /* n RF pulse durations tau_j >= 0, or NULL for hard pulses */
} mrf_sequence_desc;

/* Copy a host sequence to the device (FP64 host values; per-timepoint RF
 * rotation coefficients are formed in FP64 on the host and stored as FP32).
 * Synchronous for the upload only: it runs on the library's own stream and
 * does not wait for work queued on the caller's streams. Errors:
 * MRF_E_INVALID (n < 1, non-finite values, TE outside [0, TR], TR <= 0, a
 * negative pulse duration), MRF_E_BUDGET, MRF_E_CUDA.
 * mrf_sequence_free waits for all work on the device, then releases the
 * sequence. mrf_sequence_free_async releases it in the order of `stream`
 * without waiting: every use of the sequence must already be enqueued on
 * that stream (or have finished). */
int mrf_sequence_load(mrf_ctx *ctx, const mrf_sequence_desc *desc, mrf_seq **out);
int mrf_sequence_free(mrf_ctx *ctx, mrf_seq *seq);
int mrf_sequence_free_async(mrf_ctx *ctx, mrf_seq *seq, void *stream);

/* ------------------------------------------------------------------------ */
/* Parameter grid (Theory: ranges R, S, Q of T1, T2, df)                    */

/* Value i of an axis is min + i * step (no cumulative sums). An entry
 * (a, b, c) is valid iff T2_b < T1_a when require_t2_lt_t1 != 0. The linear
 * dictionary index runs over valid entries with T1 outermost, then T2, then
 * df innermost. */
typedef struct {
    double t1_min, t1_step; int32_t n_t1;
    double t2_min, t2_step; int32_t n_t2;
    double df_min, df_step; int32_t n_df;
    int32_t require_t2_lt_t1;
} mrf_grid_desc;

/* Number of valid entries, or a negative MRF_E_INVALID for a bad grid. */
int64_t mrf_grid_count(const mrf_grid_desc *grid);

/* (a, b, c) of linear index `index` (host only). MRF_E_INVALID if out of range. */
int mrf_grid_unravel(const mrf_grid_desc *grid, int64_t index, int32_t *a, int32_t *b, int32_t *c);

/* ------------------------------------------------------------------------ */
/* Fingerprint simulation (Appendix, Eq. A2)                                */

/* Simulate `count` fingerprints for parameter triples t1/t2/df (device
 * float32 arrays, ms / ms / Hz) into out_dev (count x n complex64,
 * row-major, not normalised). One GPU thread per fingerprint, FP32 state.
 * Errors: MRF_E_INVALID, MRF_E_CUDA. */
int mrf_simulate(mrf_ctx *ctx, const mrf_seq *seq, int64_t count, const float *t1_dev,
                 const float *t2_dev, const float *df_dev, void *out_dev, void *stream);

/* ------------------------------------------------------------------------ */
/* Dictionary (Theory: unit-norm entries so that CC is |inner product|)     */

/* Generate the whole grid's dictionary on the device: Bloch recurrence per
 * entry in FP32 and storage in `dtype` (see mrf_dtype) with a per-entry
 * scale such that stored value x scale is the unit-L2-norm entry (Theory:
 * unit-norm entries make CC the inner product). Entry e's row is the
 * interleaved (re, im) signal, zero-padded to `ld` elements. The library owns the dictionary memory,
 * charged to the budget. Runs on `stream`; the dictionary is usable by later
 * work on that stream. Errors: MRF_E_INVALID (bad grid, zero entries),
 * MRF_E_BUDGET, MRF_E_NOMEM, MRF_E_CUDA. */
int mrf_dict_generate(mrf_ctx *ctx, const mrf_seq *seq, const mrf_grid_desc *grid, mrf_dtype dtype,
                      void *stream, mrf_dict **out);
/* mrf_dict_free waits for all work on the device, then releases the
 * dictionary. mrf_dict_free_async releases it in the order of `stream`
 * without waiting: every use of the dictionary (generation, matching, ZOOM)
 * must already be enqueued on that stream (or have finished); the memory
 * returns to the stream-ordered pool. */
int mrf_dict_free(mrf_ctx *ctx, mrf_dict *dict);
int mrf_dict_free_async(mrf_ctx *ctx, mrf_dict *dict, void *stream);

/* Read-only view of a dictionary's device storage (for inspection/tests). */
typedef struct {
    int64_t entries;       /* D, valid grid entries */
    int32_t n;             /* timepoints */
    int32_t ld;            /* row stride in elements of every plane: 2n rounded up to 128, plus
                              64 (BF16) or 128 elements of padding (rows off a power-of-two
                              stride, 1-byte rows on 128-byte lines); entries past 2n are 0 */
    int32_t dtype;         /* mrf_dtype */
    const void *hi_dev;    /* D x ld: fp16 x 2^15 (F32), bf16 (BF16) or e4m3 bytes (FP8) */
    const void *lo_dev;    /* F32 only, else NULL: two D x ld e4m3 planes, the values x 2^8,
                              then the fp16 residuals x 2^19 (value = hi 2^-15 + residual 2^-19) */
    const float *norm_dev; /* D: L2 norm of the un-normalised FP32 signal */
    const float *scale_dev;/* D: per-entry scale, stored value x scale = unit-norm entry
                              (F32: 1 / norm; BF16: 1; FP8: the dequantisation scale) */
    size_t bytes;          /* device bytes charged to the budget */
    int32_t smooth_width;  /* temporal smoothing applied by mrf_dict_smooth (1: none) */
    double smooth_sigma;
} mrf_dict_info;
int mrf_dict_query(const mrf_dict *dict, mrf_dict_info *info);

/* Temporal smoothing (Methods, Experiment 4: 3- and 5-point moving Gaussian
 * smoothing of the fingerprints and of the dictionary). Each sample becomes
 * the weighted mean of the samples within h = (width - 1) / 2 of it, weights
 * exp(-k^2 / (2 sigma^2)) renormalised over the samples that exist at the
 * ends of the timecourse; Re and Im alike. width is 1 (identity), 3 or 5;
 * sigma > 0 in samples (1 is the usual choice).
 *
 * mrf_smooth: in_dev and out_dev are distinct V x n complex64 device arrays
 * (caller-owned), out = smooth(in); runs on `stream`.
 *
 * mrf_dict_smooth: smooths a generated MRF_F32 or MRF_BF16 dictionary's
 * entries in place and renormalises them to unit norm; the stored norms
 * become those of the smoothed un-normalised entries, and the dictionary
 * remembers the smoothing, so that its top-k re-score smooths the
 * re-simulated candidates alike (mrf_match_bruteforce then matches smoothed
 * fingerprints, which the caller smooths with mrf_smooth, against smoothed
 * entries, as in the paper's test of smoothing "both" sides). A dictionary
 * is smoothed at most once. ZOOM on the fly and mrf_refine simulate
 * unsmoothed candidates. Errors: MRF_E_INVALID (width, sigma, aliasing,
 * already smoothed), MRF_E_UNSUPPORTED (FP8 dictionary), MRF_E_CUDA. */
int mrf_smooth(mrf_ctx *ctx, const void *in_dev, void *out_dev, int64_t V, int32_t n, int32_t width, double sigma,
               void *stream);
int mrf_dict_smooth(mrf_ctx *ctx, mrf_dict *dict, int32_t width, double sigma, void *stream);

/* ------------------------------------------------------------------------ */
/* Matching                                                                 */

/* One result per voxel (host or device array of structs, 56 bytes each).
 * Brute force: index/i_* of the best entry by Eq. 1; cc = CC of that entry;
 * m0 = |<x, d>| / ||d||^2 and phase = arg <x, d> on the un-normalised entry
 * d (Theory: proton density from the signal scale); entries_evaluated = D;
 * min_margin = CC gap between the best and the second-best re-scored
 * candidate (-1 when only one candidate is re-scored).
 * ZOOM: the same fields for the final grid point; entries_evaluated counts
 * candidate evaluations of the search and min_margin is the smallest gap
 * between the two best values of any decision it took. */
typedef struct {
    int64_t index;               /* linear dictionary index, -1 if none */
    int32_t i_t1, i_t2, i_df;    /* grid indices (a, b, c) */
    float t1_ms, t2_ms, df_hz;
    float cc;
    float m0;
    float phase;
    int32_t entries_evaluated;
    float min_margin;
} mrf_result;

typedef struct {
    int32_t precision;   /* mrf_dtype; must equal the dictionary's dtype */
    int32_t top_k;       /* candidates kept by the tensor-core pass: 1, 2, 4, 8, 16 or 32 */
    int32_t rescore;     /* 1: re-simulate the top_k in FP32, rank by FP64 CC,
                            ties to the smaller index. 0: keep the tensor-core
                            rank-1 candidate (its cc/m0/phase still come from an
                            FP32 re-simulation with FP64 accumulation). */
} mrf_match_opts;

/* Brute-force DGS for V voxels (fp_dev: V x n complex64, row-major, any
 * scale and phase, n = the dictionary's sequence length). The score matrix is
 * never stored: each voxel's running top_k is kept on chip while the
 * dictionary streams through the tensor cores. The re-score re-simulates
 * with the sequence the dictionary was generated from (the dictionary keeps
 * its own copy). Scratch is taken from the stream-ordered pool and charged
 * to the budget for the call's duration. V = 0 is a no-op. out_dev: V
 * results. Errors: MRF_E_INVALID (dtype mismatch, bad top_k), MRF_E_BUDGET,
 * MRF_E_CUDA; device-side wait failures surface in mrf_stream_sync. */
int mrf_match_bruteforce(mrf_ctx *ctx, const mrf_dict *dict, const void *fp_dev, int64_t V,
                         const mrf_match_opts *opts, mrf_result *out_dev, void *stream);

/* Brute-force DGS over a grid without a resident dictionary (Methods: the
 * search over every grid entry by Eq. 1; for grids whose dictionary does not
 * fit in HBM). The grid's valid entries, in their linear order, are cut into
 * ranges of whole T1 rows of at most chunk_entries entries (0: 8,388,608);
 * each range's dictionary is generated on `stream` in opts->precision,
 * matched as by mrf_match_bruteforce, and released before the next, and the
 * per-voxel answers merge: the higher CC wins, ties to the earlier range
 * (smaller linear index). index and i_t1 refer to the whole grid; min_margin
 * is the gap between the best CC and the best other CC of the ranges' re-
 * scored candidates (-1 if there is none); entries_evaluated is the grid's
 * entry count, saturated at 2^31 - 1. Each range's dictionary is charged to
 * the budget while it lives; the call returns once every range has been
 * queued (the host waits for each range's grid upload, not for the kernels).
 * Errors: MRF_E_INVALID (NULL argument, bad options, a grid without a valid
 * entry, chunk_entries < 0 or smaller than a T1 row's entry count),
 * MRF_E_BUDGET, MRF_E_CUDA. */
int mrf_match_bruteforce_grid(mrf_ctx *ctx, const mrf_seq *seq, const mrf_grid_desc *grid,
                              const mrf_match_opts *opts, int64_t chunk_entries, const void *fp_dev, int64_t V,
                              mrf_result *out_dev, void *stream);

/* Brute force over a grid with no dictionary stored anywhere (the brute-force
 * counterpart of ZOOM's on-the-fly candidates; Theory, brute-force DGS):
 * inside the tensor-core matcher, simulation warps run the Bloch recurrence
 * (FP32, factors on the fly) for each tile of 256 entries and write the raw
 * entries as bf16 (hi + lo for MRF_F32, hi for MRF_BF16) straight into the
 * shared-memory stages the MMAs read, with 1 / ||d|| as each entry's column
 * scale; the top_k lists, their merge and the re-score are those of
 * mrf_match_bruteforce, and so are the results' meaning and layout (index
 * over the grid's valid entries, entries_evaluated = the entry count). Every
 * entry is simulated once per voxel unit (64 voxels for MRF_F32, 128 for
 * MRF_BF16), so it pays for small voxel counts: it needs neither the
 * dictionary's HBM nor its write and read. fp_dev: V x n complex64; out_dev:
 * V results. Errors: MRF_E_INVALID (NULL argument, precision other than
 * MRF_F32 / MRF_BF16, bad top_k or rescore, a grid without a valid entry or
 * with more than 2^31 - 1), MRF_E_BUDGET, MRF_E_CUDA. */
int mrf_match_bruteforce_fused(mrf_ctx *ctx, const mrf_seq *seq, const mrf_grid_desc *grid,
                               const mrf_match_opts *opts, const void *fp_dev, int64_t V, mrf_result *out_dev,
                               void *stream);

/* The tensor-core pass alone: per voxel the top_k (linear index, approximate
 * CC^2 of the normalised pair) in descending order, ties to the smaller
 * index. idx_dev: V x top_k int64, cc2_dev: V x top_k float32. Besides the
 * stored precision, the values carry the FP32 accumulation of the MMAs: at
 * most one unit in the last place of the running sum per MMA, i.e. a CC off by
 * at most sqrt(2) * steps * 2^-23 (steps = 2n/16 bf16 or fp16 MMAs, 2n/32 e4m3
 * ones; MRF_F32 takes both kinds). Measured at n = 1000 (MRF_F32) the values
 * run low by about 1e-5 on average and 2.3e-5 at most. mrf_result CCs never
 * carry this: they come from the FP64-accumulated re-simulation. */
int mrf_match_topk(mrf_ctx *ctx, const mrf_dict *dict, const void *fp_dev, int64_t V, int32_t precision,
                   int32_t top_k, int64_t *idx_dev, float *cc2_dev, void *stream);

/* MRF-ZOOM options (Methods, Experiment 2). Steps are physical (ms / Hz) and
 * are snapped to whole grid steps (round half up, at least 1). */
#define MRF_ZOOM_MAX_LEVELS 16
typedef struct {
    double omega_hz;        /* df pseudo-period; <= 0: 1000 / min_j TR_j (Property II) */
    double t1_init_ms;      /* start of the df search (default 1000) */
    double t2_init_ms;      /* (default 100) */
    double s1a_step_frac;   /* step 1a: coarse df scan step, x omega (6/7) */
    double s1b_half_frac;   /* step 1b: window half-width, x omega (1) */
    double s1b_step_frac;   /* step 1b: window step, x omega (1/20) */
    double s3_half_frac;    /* step 3: finest-step df window half-width, x omega (1/2) */
    int32_t n_s2;           /* step 2: 2D ZOOM levels (200, 100 ms) */
    double s2_t1_ms[MRF_ZOOM_MAX_LEVELS];
    double s2_t2_ms[MRF_ZOOM_MAX_LEVELS];
    int32_t n_s4;           /* step 4: interleaved 1D ZOOMs */
    int32_t s4_param[MRF_ZOOM_MAX_LEVELS];   /* 0: T1, 1: T2 */
    double s4_ms[MRF_ZOOM_MAX_LEVELS];
    /* Spatial-neighbour prior (Methods, Experiment 3), mrf_zoom_search only:
     * prior_chain > 0 searches the V voxels in their given (raster) order as
     * chains of prior_chain consecutive voxels (prior_chain >= V: the paper's
     * single chain through the slice). A chain's first voxel is searched on
     * the whole grid; every later voxel on the grid overlapped with T1p +-
     * prior_t1_ms, T2p +- prior_t2_ms, dfp +- prior_df_hz around the result
     * (T1p, T2p, dfp) of the voxel before it -- the index box |i - i_p| <=
     * floor(half / step), searched as a grid of its own -- starting at (T1p,
     * T2p) when prior_start is 1 (the initial ZOOM centre taken from the
     * neighbouring voxel, Theory) or at t1_init/t2_init clipped into the box
     * when it is 0. Voxels of one chain run one after another; chains run in
     * parallel. Defaults: 0 (off), 1, 3000, 800, 150. */
    int32_t prior_chain;
    int32_t prior_start;
    double prior_t1_ms, prior_t2_ms, prior_df_hz;
} mrf_zoom_opts;

/* Fill `opts` with the schedule of Experiment 2 (T1@100, T2@100, T1@50/20/10,
 * T2@50/20/10 for step 4; final 2D ZOOM at the finest step). */
void mrf_zoom_opts_default(mrf_zoom_opts *opts);

/* MRF-ZOOM for V voxels, every candidate simulated on the fly (no
 * dictionary). fp_dev: V x n complex64. out_dev: V results. The grid may be
 * far larger than any dictionary (it is never materialised). Errors:
 * MRF_E_INVALID, MRF_E_BUDGET, MRF_E_TIMEOUT, MRF_E_CUDA. */
int mrf_zoom_search(mrf_ctx *ctx, const mrf_seq *seq, const mrf_grid_desc *grid, const mrf_zoom_opts *opts,
                    const void *fp_dev, int64_t V, mrf_result *out_dev, void *stream);

/* MRF-ZOOM over a resident dictionary (Methods, Experiment 2: ZOOM "with a
 * full pre-defined dictionary"): the search of mrf_zoom_search on the
 * dictionary's own grid and sequence, each candidate's CC read from the
 * stored normalised entry (one warp streams the row) instead of simulated.
 * The dictionary must be MRF_F32 (FP32-class CC of the stored values) or MRF_BF16 (bf16 CC,
 * decisions may differ from the FP32 search where candidates differ by less
 * than about 1e-3). M0 and phase use the stored entry norms. Errors:
 * MRF_E_INVALID, MRF_E_UNSUPPORTED (FP8 dictionary, or a spatial-neighbour
 * prior in opts), MRF_E_BUDGET, MRF_E_CUDA. */
int mrf_zoom_search_dict(mrf_ctx *ctx, const mrf_dict *dict, const mrf_zoom_opts *opts, const void *fp_dev,
                         int64_t V, mrf_result *out_dev, void *stream);

/* Windowed refinement of per-voxel grid points (Results, Experiment 2: a
 * brute-force search in a small window around a ZOOM answer, here repeated
 * as a hill climb). res_dev holds V results; on entry each voxel's start is
 * (i_t1, i_t2, i_df), and a voxel whose index is < 0 or whose start is not a
 * valid grid point is left unchanged. From the start, the centre is compared
 * with the 26 points of its 3 x 3 x 3 grid neighbourhood (T1 offset outer,
 * then T2, then df, -1 before +1; points off the grid or with T2 >= T1 when
 * the grid requires T2 < T1 are not evaluated) and moves to the best of them
 * when it is strictly better (the first in that order on ties), until the
 * centre wins. CC uses the re-score's arithmetic (FP32 simulation, FP64
 * accumulation). On return the result describes the final point (index,
 * indices, values, cc, m0, phase); entries_evaluated is increased by the
 * points simulated (the start included) and min_margin becomes the smaller
 * of its entry value (when >= 0) and the climb's smallest gap between the
 * two best values of a decision. seq and grid must be those the starting
 * points refer to; fp_dev: V x n complex64. max_moves >= 1 bounds the moves
 * per voxel; a voxel that reaches it keeps its point and raises a device
 * error reported by mrf_stream_sync. Errors: MRF_E_INVALID, MRF_E_BUDGET,
 * MRF_E_CUDA. */
int mrf_refine(mrf_ctx *ctx, const mrf_seq *seq, const mrf_grid_desc *grid, const void *fp_dev, int64_t V,
               int32_t max_moves, mrf_result *res_dev, void *stream);

/* Allocation-free variant of mrf_zoom_search. The paper has no counterpart:
 * it serves callers that cannot let the library allocate device memory
 * during a call -- a framework that already reserved the GPU's memory for
 * its own pool, or a scan loop that must not meet allocation latency or an
 * out-of-memory error mid-run. The call's scratch (grid tables and the voxel
 * work counter) lives in one fixed file-scope device array of
 * MRF_ZOOM_STATIC_SCRATCH_BYTES, present on every GPU that loads the
 * library until the process exits; the call makes no cudaMalloc/cudaFree.
 * The caller still owns fp_dev and out_dev; arguments and results are those
 * of mrf_zoom_search. Limit: the grid's tables must fit the array (about
 * 16 bytes per T1 value plus 4 per T2 and per df value); a larger grid returns
 * MRF_E_INVALID with the needed size. All calls share the array and it keeps
 * the last call's contents: calls that overlap on the GPU race and must be
 * serialised by the caller. The first call on a device looks up the array's
 * address; make it before any stream capture. The spatial-neighbour prior
 * (opts->prior_chain != 0) is refused with MRF_E_UNSUPPORTED. All steps run in one kernel, with the results of
 * mrf_zoom_search bit for bit. */
#define MRF_ZOOM_STATIC_SCRATCH_BYTES (512 * 1024)
int mrf_zoom_search_static(mrf_ctx *ctx, const mrf_seq *seq, const mrf_grid_desc *grid,
                           const mrf_zoom_opts *opts, const void *fp_dev, int64_t V, mrf_result *out_dev,
                           void *stream);

/* ------------------------------------------------------------------------ */
/* Serving: continuous batching of slice requests                           */

typedef enum { MRF_MODE_BRUTE = 0, MRF_MODE_ZOOM = 1 } mrf_mode;

typedef struct {
    int32_t mode;                 /* mrf_mode */
    const mrf_dict *dict;         /* MRF_MODE_BRUTE: resident dictionary */
    mrf_match_opts match;         /* MRF_MODE_BRUTE options */
    const mrf_seq *seq;           /* sequence (both modes) */
    const mrf_grid_desc *grid;    /* MRF_MODE_ZOOM grid (copied at submit) */
    const mrf_zoom_opts *zoom;    /* MRF_MODE_ZOOM options (copied), NULL = default */
    const void *fp_host;          /* V x n complex64, copied at submit */
    int64_t V;
} mrf_request;

typedef struct {
    int32_t max_inflight;         /* launches in flight at once (streams), >= 1 */
    int32_t max_batch_voxels;     /* voxels merged into one launch */
    size_t request_bytes_budget;  /* device bytes for queued+running request buffers;
                                     0 = what remains of the context budget */
} mrf_serve_config;

/* Start the serving loop (a library-owned host thread). */
int mrf_serve_start(mrf_ctx *ctx, const mrf_serve_config *cfg);

/* Enqueue a request; returns immediately with a ticket. The fingerprints are
 * copied, so fp_host may be reused on return. A request whose buffers could
 * never fit the budget returns MRF_E_BUDGET; otherwise it waits for memory.
 * Requests are concatenated into shared launches, so a ZOOM request with a
 * spatial-neighbour prior is refused (MRF_E_UNSUPPORTED).
 * Errors: MRF_E_INVALID, MRF_E_BUDGET, MRF_E_UNSUPPORTED. */
int mrf_serve_submit(mrf_ctx *ctx, const mrf_request *req, uint64_t *ticket);

/* Wait up to timeout_ms (0 = just check) for a ticket. MRF_OK: out_host (V
 * results, caller-owned) is filled and the ticket retired. MRF_PENDING: not
 * done yet (timeout_ms = 0). MRF_E_TIMEOUT: still running after timeout_ms.
 * MRF_E_NOTFOUND: unknown or retired ticket. Never blocks beyond timeout_ms. */
int mrf_serve_poll(mrf_ctx *ctx, uint64_t ticket, int32_t timeout_ms, mrf_result *out_host);

/* Cancel a queued (not yet launched) request; MRF_E_NOTFOUND otherwise. */
int mrf_serve_cancel(mrf_ctx *ctx, uint64_t ticket);

typedef struct {
    uint64_t submitted, admitted, completed, rejected, cancelled, launches;
    uint64_t queued_now, running_now;
    size_t request_bytes_in_use, request_bytes_peak;
} mrf_serve_stats;
/* A snapshot of the serving counters (request counts by fate, shared launches,
 * requests queued and running now, request bytes charged now and at peak).
 * Errors: MRF_E_INVALID (NULL argument or no serving loop started). */
int mrf_serve_get_stats(mrf_ctx *ctx, mrf_serve_stats *stats);

/* Stop accepting work, finish what is admitted, join the thread. */
int mrf_serve_stop(mrf_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* MRF_H */
