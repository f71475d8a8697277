/*
 * snaps.h -- C ABI of libsnaps, the B300 (sm_103a) hot path of SNAPS
 * population outlier detection (Gowanlock et al., arXiv 2405.20176).
 *
 * The library computes, for N objects with F <= 15 features and any set of
 * feature subspaces (bitmasks, Eq. 1), the exact distance similarity
 * self-join (DSSJ, Sec. 3.5) and k-nearest-neighbour self-join (kNNSJ,
 * Sec. 3.6) and the four per-object outlier metrics derived from them
 * (Sec. 3.5.1, 3.6.1; Table 2): eps-neighbour count, mean eps-neighbour
 * distance, kNN in-degree and mean kNN distance, with their rankings.
 *
 * Conventions shared by every entry point
 *  - Every call returns a snaps_status and never aborts the process.  On
 *    failure snaps_last_error() gives a message for the calling thread.
 *  - Pointers are plain host or device pointers; the library tells them
 *    apart with cudaPointerGetAttributes.  Unless a call says otherwise,
 *    input arrays may be host or device memory, and so may outputs.  Device
 *    memory must belong to the call's device (or be managed memory); a
 *    buffer on another GPU is rejected with EINVAL.
 *  - A call makes its context's device current while it runs and restores
 *    the calling thread's previous current device before it returns.  A call
 *    that writes any host output returns only after that output is written
 *    (it synchronises the stream); a call with device outputs only is
 *    asynchronous on `stream`.
 *  - The caller owns every array it passes in.  The library owns contexts
 *    (snaps_ctx) and indexed populations (snaps_pop) and frees them in
 *    snaps_destroy / snaps_release.
 *  - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *    stream).  Device work is ordered on it.
 *  - A subspace mask is a uint16_t with bit j set when feature j belongs to
 *    it.  A valid mask has 2..F bits and no bit >= F.  Masks are always host
 *    arrays.
 *  - Distances are Euclidean over the subspace's features, computed in FP32
 *    in one fixed order: the squared differences are accumulated with fused
 *    multiply-adds from the highest feature index down to the lowest.  Every
 *    neighbour decision uses these bits, so every path (plain,
 *    subspace-batched, grid-indexed, tensor-core filtered) returns the same
 *    eps counts, kNN lists, in-degrees and kNN mean distances; the
 *    tensor-core forms take the mean eps distance from their accumulator
 *    (see snaps_scores).  A point is never its own neighbour.  The eps test is
 *    inclusive, d^2 <= eps^2.  kNN order is by (distance, index).
 *  - Default radius (eps == NULL): eps = 0.05 * sqrt(d) for a d-feature
 *    subspace, i.e. eps^2 = 0.0025 * d rounded once to FP32.
 */
#ifndef SNAPS_H
#define SNAPS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum snaps_status {
    SNAPS_OK = 0,
    SNAPS_EINVAL = 1,    /* an argument is out of range or inconsistent */
    SNAPS_ENOMEM = 2,    /* device allocation failed or would exceed the context's HBM budget */
    SNAPS_EBUSY = 3,     /* the object is in use (e.g. a population with requests in flight) */
    SNAPS_EAGAIN = 4,    /* snaps_poll: the request has not finished within the timeout */
    SNAPS_ETIMEOUT = 5,  /* a bounded device-side wait gave up; the context stays usable */
    SNAPS_ECUDA = 6,     /* the CUDA runtime reported an error */
    SNAPS_ECANCELED = 7  /* the request was cancelled before it ran */
} snaps_status;

#define SNAPS_MAX_FEATURES 15
#define SNAPS_MAX_K 32
#define SNAPS_N_SCORES 4
/* score rows, in this order, in every scores / norm / top output */
#define SNAPS_SCORE_EPS_COUNT 0  /* DSSJ distance-oblivious: eps-neighbour count (Sec. 3.5.1 item 1) */
#define SNAPS_SCORE_EPS_MEAN 1   /* DSSJ distance-aware: mean eps-neighbour distance, 0 if none (item 2) */
#define SNAPS_SCORE_KNN_INDEG 2  /* kNNSJ distance-oblivious: in-degree of the kNN graph (Sec. 3.6.1 item 1) */
#define SNAPS_SCORE_KNN_MEAN 3   /* kNNSJ distance-aware: mean distance to the k neighbours (item 2) */

/* snaps_index flags */
#define SNAPS_NORM_MINMAX 0x1u   /* map every feature onto [0, 1] by its min and max (Sec. 3.3) */
#define SNAPS_NAN_TO_MEAN 0x2u   /* replace NaN by the feature's mean first (Sec. 2.1) */

/* precision argument of snaps_scores / snaps_request: one of the four join
 * forms, optionally OR-ed with one index choice for low-dimensional subspaces */
#define SNAPS_FP32 0u            /* plain FP32 join */
#define SNAPS_TC_F16 1u          /* tensor-core contraction, high/low FP16 parts, exact FP32 recompute near
                                  * eps and the k-th distance */
#define SNAPS_TC_BF16 2u         /* the same with BF16 parts: a 4x wider margin, more recomputes */
#define SNAPS_TC_TF32 3u         /* the same with TF32 parts (kind::tf32, K = 8 per MMA): FP16's margin,
                                  * twice the MMAs and operand bytes */
/* The tensor-core forms join subspaces in blocks of 256 (sorted by
 * dimension), and a block costs about the same however few it carries.  A
 * block is formed only with at least a minimum fill of subspaces: the
 * context's value from snaps_set_tc_min_fill, else snaps_autotune_tc's choice
 * for the population's size class, else SNAPS_TC_MIN_FILL.  Subspaces left
 * over (every one of a request smaller than that) take the plain FP32
 * routes, which return the same counts, kNN lists and in-degrees. */
#define SNAPS_TC_MIN_FILL 128
#define SNAPS_TC_NEVER 257       /* a minimum fill that keeps every subspace off the tensor cores */
#define SNAPS_INDEX_GRID 0x100u  /* subspaces of <= 4 features always take the grid index */
#define SNAPS_INDEX_NONE 0x200u  /* no grid index: every subspace is joined by brute force */
/* Without either index flag, subspaces of <= 4 features take the grid index
 * (sort-by-cell over up to 3 of their features, Sec. 3.8.1) when
 * n >= SNAPS_GRID_AUTO_N.  Its cells are a third of eps wide for two-feature
 * subspaces and eps wide otherwise, unless snaps_autotune recorded another
 * choice.  Every choice gives the same results. */
#define SNAPS_GRID_AUTO_N 65536

typedef struct snaps_ctx snaps_ctx;
typedef struct snaps_pop snaps_pop;

/* Library version as "major.minor.patch"; static storage. */
const char *snaps_version(void);

/* Message describing the calling thread's most recent failure ("" if none);
 * valid until that thread's next snaps_* call. */
const char *snaps_last_error(void);

/* ---- contexts and populations: library plumbing (the paper has no
 * counterpart; it runs one process per subspace, Sec. 3.8) ---- */

/* Create a context on CUDA device `device`.  `hbm_budget_bytes` caps the
 * device memory the context may hold (populations + scratch + in-flight
 * requests); 0 means 90 % of the device's free memory at creation.
 * Errors: EINVAL (bad device or out == NULL), ECUDA. */
snaps_status snaps_create(int device, size_t hbm_budget_bytes, snaps_ctx **out);

/* Finish all queued requests, free everything the context owns.  Populations
 * not yet released are released.  NULL is a no-op.  Errors: none (returns
 * SNAPS_OK). */
snaps_status snaps_destroy(snaps_ctx *ctx);

/* Device memory currently held and the budget, in bytes (either output may
 * be NULL).  Errors: EINVAL (ctx NULL). */
snaps_status snaps_mem_info(const snaps_ctx *ctx, size_t *held, size_t *budget);

/* Index a population: the data set D of Sec. 3.1.
 * feat: n x f float32, row-major, host or device; read before the call
 *   returns (the call synchronises `stream`).
 * flags: SNAPS_NORM_MINMAX and/or SNAPS_NAN_TO_MEAN.  Normalisation takes
 *   each feature's min and max in FP64 and stores (x - min) / (max - min)
 *   computed in FP64 and rounded to FP32; a constant feature becomes 0.
 *   Without SNAPS_NORM_MINMAX the values are used unchanged.
 * Requirements: n >= 2, 1 <= f <= 15, every value finite (NaN allowed only
 *   with SNAPS_NAN_TO_MEAN).
 * Requirements: n <= 2^24 as well.
 * The stored rows are kept in cell order (sorted by a Morton key over the
 * features) so that neighbouring rows are near in feature space; every output
 * of the joins and scores is still indexed by the caller's row order, and the
 * results do not depend on the stored order.
 * The population lives in device memory until snaps_release.
 * Errors: EINVAL, ENOMEM (over budget), ECUDA. */
snaps_status snaps_index(snaps_ctx *ctx, const float *feat, int64_t n, int f,
                         uint32_t flags, void *stream, snaps_pop **out);

/* Release a population and its device memory.  NULL is a no-op.
 * Errors: EBUSY while requests that use it are in flight. */
snaps_status snaps_release(snaps_pop *pop);

/* Size of a population: objects n and features f (host outputs).
 * Errors: EINVAL (pop or an output NULL). */
snaps_status snaps_pop_shape(const snaps_pop *pop, int64_t *n, int *f);

/* Copy the population's stored (normalised) features out as n x f float32
 * row-major into `out` (host or device; caller-owned), in the caller's row
 * order.  Ordered on `stream`; a host `out` is written before the call
 * returns.  Errors: EINVAL (pop or out NULL), ECUDA. */
snaps_status snaps_pop_features(const snaps_pop *pop, float *out, void *stream);

/* kNN self-join (kNNSJ, Sec. 3.6) of every subspace in `masks`.
 * masks: n_masks host uint16 masks.  1 <= k <= min(32, n - 1).
 * idx:  n_masks x n x k int32 (subspace-major, then object, then rank):
 *       the k nearest other objects, nearest first, exact ties by index.
 * dist: same shape, float32 Euclidean distances, or NULL.
 * Errors: EINVAL (bad mask, k, sizes), ENOMEM, ECUDA. */
snaps_status snaps_knn_selfjoin(snaps_pop *pop, const uint16_t *masks, int n_masks,
                                int k, int32_t *idx, float *dist, void *stream);

/* Distance similarity self-join (DSSJ, Sec. 3.5) of every subspace.
 * eps: n_masks host float radii, or NULL for 0.05 * sqrt(d) per subspace.
 * count: n_masks x n int32, #{j != i : d(i, j) <= eps}, or NULL.
 * mean_dist: n_masks x n float32, mean distance to those j (0 when count is
 *   0), or NULL.
 * Errors: EINVAL, ENOMEM, ECUDA. */
snaps_status snaps_eps_selfjoin(snaps_pop *pop, const uint16_t *masks, int n_masks,
                                const float *eps, int32_t *count, float *mean_dist,
                                void *stream);

/* Both joins and the four outlier metrics per object and subspace (Table 2).
 * k, eps: as above.  precision: SNAPS_FP32 (plain FP32 joins), SNAPS_TC_F16,
 *   SNAPS_TC_BF16 or SNAPS_TC_TF32 (the squared-difference x subspace-mask
 *   contraction on the tensor cores, each scaled squared difference split
 *   into a high and a low FP16, BF16 or TF32 part, FP32 accumulation: d^2 to
 *   within 3.9e-6 (FP16, TF32) or 7.4e-6 (BF16) relative.  A candidate within
 *   a margin of 2^-17 (FP16, TF32) or 2^-15 (BF16) of eps^2 or of the k-th
 *   distance is recomputed exactly in FP32, which decides; one clearly inside
 *   eps is counted and its distance taken from the accumulator.  So counts,
 *   kNN lists, in-degrees and kNN means are the plain form's bits, and the
 *   mean eps distance agrees with the plain form's to 2.5e-6 (FP16, TF32) or
 *   4.2e-6 (BF16) relative plus eps / 2^20).  The tensor-core forms need
 *   every feature to span at most 1, which SNAPS_NORM_MINMAX guarantees
 *   (EINVAL otherwise).  Each may be OR-ed with SNAPS_INDEX_GRID or
 *   SNAPS_INDEX_NONE (see their definitions).
 * scores: n_masks x 4 x n float32 raw metrics (rows SNAPS_SCORE_*), or NULL.
 *   Counts and in-degrees are exact integers stored as float.
 * norm:   n_masks x 4 x n float32, each metric mapped onto [0, 1] with
 *   1 = most outlying, from its population min and max (a constant metric
 *   maps to 0; objects without eps-neighbours get 1 for the eps mean
 *   distance and the rest are scaled among themselves), or NULL.  The span
 *   max - min and its reciprocal are taken in FP64; each value is within
 *   half an FP32 ulp (plus 2^-20 ulp) of the FP64 quotient.
 * top:    n_masks x 4 x top_n int32, the first top_n objects of each ranking
 *   (Sec. 3.4, rank 0 = most outlying): counts and in-degrees ascending,
 *   mean distances descending, objects without eps-neighbours first for the
 *   eps mean distance; equal values in index order.  NULL or top_n == 0
 *   skips it; 1 <= top_n <= min(n, 1024) otherwise.
 * Errors: EINVAL, ENOMEM, ECUDA. */
snaps_status snaps_scores(snaps_pop *pop, const uint16_t *masks, int n_masks, int k,
                          const float *eps, uint32_t precision, float *scores,
                          float *norm, int32_t *top, int top_n, void *stream);

/* ---- parameter selection: the over- / underfitting trade-off ---- */

#define SNAPS_SELECT_MAX_GRID 64  /* values per parameter grid */
#define SNAPS_SELECT_MAX_K 4096   /* largest k of a k grid */

/* Select eps and k for every subspace in `masks` as Sec. 3.5.2 (eps, Eq. 2
 * and 3) and Sec. 3.6.2 (k) describe.  For each grid value the population is
 * ranked (Sec. 3.4, as snaps_scores ranks it); U^min_j and U^max_j are the
 * fractions of the top-n objects that the ranking at grid value j shares with
 * the ranking at the smallest and at the largest grid value (Eq. 2); the
 * selected index minimises |U^min_j - U^max_j| (Eq. 3; the smallest such j on
 * ties).  As in Sec. 3.5.3 and 3.6.2, one join per subspace at the largest
 * grid value gives the results at all of them.
 * masks: n_masks host masks.
 * eps grid (used when u_eps or eps_select is non-NULL): n_eps values
 *   (2..SNAPS_SELECT_MAX_GRID) evenly spaced over [eps_min[m], eps_max[m]]
 *   (host arrays, 0 <= eps_min < eps_max): eps_j = eps_min + j (eps_max -
 *   eps_min) / (n_eps - 1), computed in FP64 and rounded to FP32.  Metrics:
 *   0 = eps-neighbour count, 1 = mean eps-neighbour distance.
 * k grid (used when u_k or k_select is non-NULL): n_k (2..64) strictly
 *   ascending values in 1..min(SNAPS_SELECT_MAX_K, n - 1), host array.
 *   Metrics: 0 = kNN in-degree, 1 = mean kNN distance, the latter from an
 *   exact sum of the k_j FP32 distances quantised to 2^-30.
 * top_n: the n of Eq. 2 (the paper uses 1 % of the population), 1..min(n, 1024).
 * Outputs (host or device, caller-owned, any may be NULL):
 *   u_eps:      n_masks x 2 metrics x 2 (0 = U^min, 1 = U^max) x n_eps floats;
 *   eps_select: n_masks x 2 metrics int32, the selected grid index;
 *   u_k, k_select: the same for the k grid.
 * The call synchronises `stream`.
 * Errors: EINVAL (bad masks, grids, top_n, or no output), ENOMEM, ECUDA. */
snaps_status snaps_select(snaps_pop *pop, const uint16_t *masks, int n_masks,
                          const float *eps_min, const float *eps_max, int n_eps,
                          const int32_t *k_grid, int n_k, int top_n,
                          float *u_eps, int32_t *eps_select, float *u_k, int32_t *k_select,
                          void *stream);

/* ---- eps range from selectivity ---- */

#define SNAPS_SELECTIVITY_MAX_SAMPLE 65536
#define SNAPS_SELECTIVITY_MAX_BINS 4096

/* Radii at which the mean number of eps-neighbours per object (itself
 * excluded: the selectivity of Sec. 3.5.3, s = (|A| - |D|) / |D|) reaches
 * each target, estimated from a sample as Sec. 3.5.3 describes: m =
 * min(n_sample, n) objects (original indices floor(s n / m), s < m) against
 * every other object.  eps_mean, the mean of those m (n - 1) distances, bounds
 * the search; they are counted in n_bins bins of width eps_mean / n_bins over
 * [0, eps_mean), and the radius of a target is the first bin edge (b + 1)
 * eps_mean / n_bins at which the cumulative count reaches target * m, or
 * eps_mean when none does.  The paper's grid ends are the targets 0.001 n
 * (eps_min) and 0.15 n (eps_max).  Distances are the library's FP32 ones;
 * eps_mean comes from an exact sum of distances quantised to 2^-20.
 * masks: n_masks host masks.  targets: n_targets (1..32) host doubles in
 *   (0, n - 1], mean neighbours per object.
 * n_sample: 1..SNAPS_SELECTIVITY_MAX_SAMPLE, with n_sample (n - 1) < 2^41;
 *   n_bins: 1..SNAPS_SELECTIVITY_MAX_BINS.
 * Outputs (host or device, caller-owned): eps, n_masks x n_targets floats;
 *   eps_mean, n_masks floats (may be NULL).
 * The call synchronises `stream`.
 * Errors: EINVAL (bad masks, targets, sample or bins; n < 2; eps NULL),
 * ENOMEM, ECUDA. */
snaps_status snaps_eps_selectivity(snaps_pop *pop, const uint16_t *masks, int n_masks,
                                   const double *targets, int n_targets, int n_sample, int n_bins,
                                   float *eps, float *eps_mean, void *stream);

/* ---- autotuning of the index route ---- */

#define SNAPS_TUNE_CELLS 3       /* grid cell widths tried: 1, 1/2 and 1/3 x eps */
#define SNAPS_TUNE_MAX_N 65536   /* larger populations are timed on a sample */

/* One subspace dimension's measurements and choice. */
typedef struct snaps_tune_entry {
    int d;                            /* subspace dimension, 2..4 */
    int grid;                         /* 1: the grid index, 0: brute force */
    float cell_mult;                  /* the grid's cell width in units of eps: 1 / R
                                         (R = 1, 2, 3: a (2R + 1)^D block of cells),
                                         or >= 1 (one cell that wide, a 3^D block) */
    double ms_brute;                  /* ms per subspace, brute force */
    double ms_grid[SNAPS_TUNE_CELLS]; /* ms per subspace, grid at 1, 1/2, 1/3 x eps */
} snaps_tune_entry;

/* Choose how subspaces of 2, 3 and 4 features are joined on populations of
 * this one's size class.  For each dimension d it times two subspaces of d
 * features (the lowest and the highest features) with this k and the default
 * radius: by brute force, and on the grid index (sort-by-cell, Sec. 3.8.1)
 * with cells 1, 1/2 and 1/3 of eps wide, whose search blocks are 3, 5 and 7
 * cells across per index dimension (every neighbour lies within them).  Populations of more than SNAPS_TUNE_MAX_N objects are timed on
 * an evenly strided sample of that many.  The fastest choice is recorded in
 * the context under (floor(log2 n), d, k <= 16 or not).  Calls without an
 * index flag then follow it for the subspaces that are joined on their own:
 * those alone among the requested ones in their 32-subspace chunk, and all of
 * them in the tensor-core forms.  Subspaces that share a chunk keep the
 * built-in rule (the grid from SNAPS_GRID_AUTO_N objects on), because there
 * the subspace-batched join shares its arithmetic and a subspace costs far
 * less than on its own.  SNAPS_INDEX_GRID uses the recorded cell width.  Every
 * route returns the same results; only the time changes.
 * k: 1..min(SNAPS_MAX_K, n - 1).  out: 3 entries (d = 2, 3, 4; host), or NULL.
 * The call synchronises `stream`.
 * Errors: EINVAL, ENOMEM, ECUDA. */
snaps_status snaps_autotune(snaps_pop *pop, int k, snaps_tune_entry *out, void *stream);

/* Measurements and choice of snaps_autotune_tc. */
typedef struct snaps_tc_tune {
    int min_fill;     /* fewest subspaces for which a tensor-core block pays, 1..SNAPS_TC_NEVER */
    double ms_block;  /* one tensor-core block of 256 subspaces of 3..12 features */
    double ms_lone;   /* ms per subspace of the same set joined on its own in plain FP32 */
} snaps_tc_tune;

/* Choose the subspaces-per-block threshold of the tensor-core forms for
 * populations of this one's size class (floor(log2 n)) and this k class.  It
 * times one block of 256 subspaces of 3..12 features (a fixed pseudo-random
 * choice) in `precision` (SNAPS_TC_F16, SNAPS_TC_BF16 or SNAPS_TC_TF32) and 32 of them
 * joined one at a time in plain FP32, on the population or, above
 * SNAPS_TUNE_MAX_N objects, an evenly strided sample of it.  The block pays
 * once it carries more subspaces than its time buys on their own:
 * min_fill = ceil(ms_block / ms_lone), capped at SNAPS_TC_NEVER.  Later
 * tensor-core calls on such populations form blocks only with at least that
 * many subspaces (see SNAPS_TC_MIN_FILL).  The paper has no counterpart.
 * out: host, or NULL.  The call synchronises `stream`.
 * Errors: EINVAL (pop NULL, bad precision or k, fewer than 3 features, a
 * population outside the unit range), ENOMEM, ECUDA. */
snaps_status snaps_autotune_tc(snaps_pop *pop, int k, uint32_t precision, snaps_tc_tune *out, void *stream);

/* Fix the minimum fill of tensor-core blocks for every later call on `ctx`,
 * whatever the population's size: 1 puts every subspace of a tensor-core
 * call on the tensor cores, SNAPS_TC_NEVER none; 0 goes back to the tuned or
 * built-in choice.  Errors: EINVAL (ctx NULL, fill outside 0..SNAPS_TC_NEVER). */
snaps_status snaps_set_tc_min_fill(snaps_ctx *ctx, int fill);

/* Record a choice without timing it, for populations of n's size class and
 * this k class: e->d (2..4), e->grid, e->cell_mult (in (0, 64]; the times are
 * ignored).  Errors: EINVAL. */
snaps_status snaps_autotune_set(snaps_ctx *ctx, int64_t n, int k, const snaps_tune_entry *e);

/* Forget every recorded choice, the tensor-core minimum fills included (the
 * built-in rules apply again; a fill set by snaps_set_tc_min_fill stays).
 * Errors: EINVAL (ctx NULL). */
snaps_status snaps_autotune_clear(snaps_ctx *ctx);

/* ---- serving: continuous batching of scoring requests ---- */

/* Continuous batching is this library's serving layer; the paper schedules
 * whole subspaces across GPUs instead (Sec. 3.8.2).
 *
 * One scoring request: snaps_scores on a resident population.  masks and
 * eps are copied at submit; the outputs (device or host, caller-owned) must
 * stay valid until the request completes. */
typedef struct snaps_request {
    snaps_pop *pop;
    const uint16_t *masks;
    int n_masks;
    int k;
    const float *eps;      /* NULL = default radius */
    uint32_t precision;
    float *scores;         /* may be NULL */
    float *norm;           /* may be NULL */
    int32_t *top;          /* may be NULL */
    int top_n;
} snaps_request;

typedef struct snaps_result {
    snaps_status status;   /* outcome of the request */
    double queue_us;       /* submit -> admitted to a slot */
    double latency_us;     /* submit -> results written */
    int64_t objects_x_subspaces; /* n * n_masks */
} snaps_result;

/* Queue a request.  The context's scheduler admits queued requests in
 * arrival order as soon as a slot and enough of the HBM budget are free, so
 * requests that arrive while others run overlap them on the device.  A
 * request of more than 2e11 candidate-pair evaluations (n (n - 1) x
 * subspaces) runs in parts of its subspace list, each about that much work;
 * a part holds a multiple of 32 subspaces in the FP32 form (one subspace at a
 * time once 32 would exceed 2e11) and a multiple of 256 in the tensor-core
 * forms, whose launches cost a whole 256-subspace block.  Between parts its
 * slot serves the small requests queued behind it (see snaps_serving_stats),
 * so they wait for one part, not for the whole request.
 * Errors: EINVAL (malformed request), ENOMEM (the request alone exceeds the
 * budget). */
snaps_status snaps_submit(snaps_ctx *ctx, const snaps_request *req, uint64_t *ticket);

/* Wait up to timeout_us (0 = just test, < 0 = forever) for a request.
 * Returns SNAPS_OK and fills *out once it has finished (whatever its own
 * status), SNAPS_EAGAIN if it has not, EINVAL for an unknown ticket.  A
 * finished ticket is forgotten after the first successful poll. */
snaps_status snaps_poll(snaps_ctx *ctx, uint64_t ticket, int64_t timeout_us,
                        snaps_result *out);

/* Cancel a request that has not been admitted yet (ECANCELED becomes its
 * status); EBUSY if it is already running or done. */
snaps_status snaps_cancel(snaps_ctx *ctx, uint64_t ticket);

/* Continuous batching: a slot that admits a request whose every subspace is
 * joined on its own (plain form; no 32-subspace chunk with four or more of
 * its subspaces requested; no grid index) and whose work is at most 4e10
 * candidate-pair evaluations (n (n - 1) x subspaces) also admits the requests
 * of that kind queued right behind it, up to 32 and within the HBM budget.
 * Their subspaces are then joined by one launch, each request keeping its own
 * outputs; results are the same as alone.  Counters since the context was
 * created: launches that served two or more requests, and the requests they
 * served (either output may be NULL).  Errors: EINVAL (ctx NULL). */
snaps_status snaps_serving_stats(snaps_ctx *ctx, int64_t *fused_launches, int64_t *fused_requests);

/* Number of requests the scheduler may run at once (default 4, 1..64).
 * Errors: EINVAL (ctx NULL or slots out of range), EBUSY (lowering it after
 * serving has started). */
snaps_status snaps_set_slots(snaps_ctx *ctx, int slots);

/* ---- scoring without device allocation ---- */

#define SNAPS_STATIC_MAX_N 32768       /* objects per allocation-free call */
#define SNAPS_STATIC_MAX_MASKS 32768   /* subspaces per allocation-free call */

/* snaps_scores for callers that cannot let a library allocate device memory
 * -- a process holding a fixed, pre-planned share of a GPU, or code that must
 * not call cudaMalloc / cudaFree because they can synchronise the device.  The
 * paper has no counterpart; this is a deployment convenience.
 * It allocates nothing.  Its working memory -- the normalised population,
 * statistics, the kernels' control block and the subspace plan, about 2.7 MB
 * -- is one static device array inside the library that every GPU which loads
 * the library keeps until the process exits.  Every call looks up that
 * array's device address (cudaGetSymbolAddress, with `device` current).  The
 * first call on a device may make the CUDA driver load the library's device
 * code and, with it, create the array; make that first call before any
 * stream capture.
 * device: CUDA device to run on.  The call makes it current and restores the
 *   calling thread's previous current device before it returns.
 * feat: n x f float32 row-major in device memory, normalised as flags say
 *   (SNAPS_NORM_MINMAX / SNAPS_NAN_TO_MEAN), 2 <= n <= SNAPS_STATIC_MAX_N.
 * masks, n_masks (<= SNAPS_STATIC_MAX_MASKS), k, eps: as for snaps_scores.
 * scores: n_masks x 4 x n float32, device memory (required).
 * top: n_masks x 4 x top_n int32, device memory, or NULL.
 * The call synchronises `stream` before returning.  Every call shares the one
 * array and it keeps the last call's contents (the call clears what must start
 * at zero), so calls whose GPU work overlaps -- on different streams or
 * threads -- race; issue them one after another.  Results equal those of
 * snaps_index + snaps_scores.
 * Errors: EINVAL (sizes beyond the limits, host pointers or memory of another
 * GPU, bad masks / k / eps, non-finite features), ETIMEOUT, ECUDA. */
snaps_status snaps_scores_static(int device, const float *feat, int64_t n, int f,
                                 uint32_t flags, const uint16_t *masks, int n_masks, int k,
                                 const float *eps, float *scores, int32_t *top, int top_n,
                                 void *stream);

/* ---- calibration ---- */

/* Measure on `device` the rate of FP32 (add, compare) pairs -- one pair per
 * (pair, subspace) evaluation is the plain join's algorithmic minimum -- with
 * a dependency-free kernel occupying every SM; writes pairs per second.  The
 * paper has no counterpart: this backs the ALU roofline denominator.
 * Errors: EINVAL (NULL output), ECUDA. */
snaps_status snaps_calibrate_alu(int device, double *evals_per_s);

/* ---- failure detection (library plumbing; the paper has no counterpart) ---- */

/* Every wait of the tensor-core join's pipeline (a tile copy landing, B rows
 * written, an MMA batch done, accumulators read) is bounded: after `spins`
 * tries it gives up, the launch's warps leave in order (each waits for its
 * own copies and MMAs in flight, with the default bound, and tensor memory is
 * freed), and the call returns SNAPS_ETIMEOUT; the context stays usable.
 * spins = 0 restores the default, 2^26 tries, far longer than any healthy
 * copy or MMA takes.  A small value makes the waits give up on purpose, which
 * is how the failure path is tested.  Applies to later calls on `ctx`.
 * Errors: EINVAL (ctx NULL). */
snaps_status snaps_set_wait_limit(snaps_ctx *ctx, unsigned spins);

/* ---- tracing: device time per phase (measurement plumbing; the paper has
 * no counterpart) ---- */

#define SNAPS_PHASE_INDEX 0      /* normalisation kernels of snaps_index */
#define SNAPS_PHASE_JOIN_TREE 1  /* subspace-batched (tree) join kernel */
#define SNAPS_PHASE_JOIN_LANE 2  /* joins of subspaces alone in their 32-subspace chunk
                                  * (the subspace-at-a-time kernel) */
#define SNAPS_PHASE_NORM 3       /* finishing kernel of a call that asks for normalised
                                  * metrics (it also ranks, when top-n lists are asked for) */
#define SNAPS_PHASE_TOP 4        /* finishing kernel of a call that asks for top-n rankings
                                  * alone */
#define SNAPS_PHASE_JOIN_TC 5    /* tensor-core filtered join kernel */
#define SNAPS_PHASE_ORDER 6      /* per-chunk row orders for the subspace-batched join */
#define SNAPS_PHASE_GRID 7       /* grid index builds and grid-indexed joins */
#define SNAPS_PHASE_SELECT 8     /* parameter-selection joins (snaps_select) */
#define SNAPS_N_PHASES 9

/* enable != 0: clear the counters and start recording, around every kernel
 * launch of every later call on this context, a pair of CUDA events on the
 * stream the kernel is launched on.  enable == 0 stops recording.
 * Errors: EINVAL (ctx NULL). */
snaps_status snaps_trace(snaps_ctx *ctx, int enable);

/* Wait for the recorded events, then report per phase the summed device time
 * in milliseconds (ms[SNAPS_N_PHASES]) and the number of kernel launches
 * (launches[SNAPS_N_PHASES]) since tracing was enabled or last read; either
 * array may be NULL.  The counters restart from zero.
 * Errors: EINVAL (ctx NULL), ECUDA (an event failed). */
snaps_status snaps_trace_read(snaps_ctx *ctx, double *ms, int64_t *launches);

/* The subspace-batched join's candidate streams since tracing was last
 * enabled (the context's synchronous calls only): 64-row steps
 * loaded and evaluated, and all steps, the skipped ones -- whose box bound
 * proves every pair fails -- included.  Either output may be NULL.  Waits for
 * the device.  Errors: EINVAL (ctx NULL), ECUDA. */
snaps_status snaps_trace_steps(snaps_ctx *ctx, int64_t *steps_loaded, int64_t *steps_total);

#ifdef __cplusplus
}
#endif

#endif /* SNAPS_H */
