/*
 * boruta.h -- C ABI of the GB300-native GPU Boruta library.
 *
 * The library runs the data-parallel hot path of GPU Boruta (Li et al.,
 * "Novel GPU Boruta algorithms for feature selection from high-dimensional
 * data"): every iteration of Alg. 1 -- shadow features, a random forest fit
 * on the shadow-augmented matrix, per-tree impurity importance (Alg. 2) or
 * out-of-bag permutation importance (Alg. 3), the hit update and the
 * Bonferroni-corrected binomial accept/reject test -- as CUDA kernels for
 * sm_103a.  All entry points use plain pointers and sizes; none takes or
 * returns a framework type.
 *
 * Conventions shared by every entry point:
 *   - Return value: 0 (BORUTA_OK) on success, a negative boruta_status on
 *     error; boruta_last_error() then returns a message (thread-local).
 *     On error, caller-owned outputs are left unspecified.
 *   - Ownership: all pointers are caller-owned.  The library allocates only
 *     its own device workspace, released before boruta_fit returns or by
 *     boruta_session_destroy.
 *   - X is the quantised feature matrix, column-major uint8 bins: column j
 *     starts at X + j*ld (ld >= N bytes, ld and X 16-byte aligned for the
 *     vectorised path; other strides are accepted and use a slower path).
 *     Every bin must be < n_bins.
 *   - y: classification labels as uint8 in [0, n_classes), or regression
 *     targets as int64 fixed point in units of 2^-20.
 *   - Device pointers are accepted unless opts->host_inputs = 1, in which
 *     case X and y are host pointers copied in by the call.
 *   - Work is queued on opts->stream (NULL: the legacy default stream); the
 *     fit calls synchronise that stream once per Boruta iteration.
 *
 * Limits (BORUTA_EINVAL beyond them): 1 <= N < 2^24, 1 <= p < 2^23,
 * 2 <= n_bins <= 256, 1 <= n_classes <= 8, 1 <= n_trees < 2^20,
 * 0 <= max_depth <= 30, 1 <= max_iter <= 126, 0 < alpha.
 * Regression targets must satisfy N * max|y| < 2^62 (BORUTA_EOVERFLOW).
 */
#ifndef BORUTA_GB300_H
#define BORUTA_GB300_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  BORUTA_OK = 0,
  BORUTA_EINVAL = -1,    /* bad argument, size or input value */
  BORUTA_EOVERFLOW = -2, /* an integer bound guard tripped (weights, sums, pools) */
  BORUTA_ETIMEOUT = -3,  /* reserved: no kernel of this library waits on another (no device
                            barrier, no spin), so no call returns it */
  BORUTA_ECUDA = -4,     /* a CUDA runtime call failed */
  BORUTA_ENOMEM = -5     /* device workspace allocation failed */
} boruta_status;

/* task = kind | importance */
#define BORUTA_CLASSIFICATION 0 /* Gini criterion, KL loss for Alg. 3 */
#define BORUTA_REGRESSION 1     /* variance criterion, squared-error loss for Alg. 3 */
#define BORUTA_TREEIMP 0        /* Alg. 2: impurity decrease ("gain x samples") */
#define BORUTA_PERMUT 2         /* Alg. 3 on each tree's out-of-bag rows */

typedef struct {
  int stat;        /* hit statistic: 0 = Z score mean/(sd/sqrt(M)) (default), 1 = mean */
  int precision;   /* per-term arithmetic: 0 = FP64 (default), 1 = FP32; sums are exact either way */
  int tie_break;   /* equal split scores: 0 = lowest feature index (default), 1 = feature drawn first at
                      the node; then the lowest bin */
  int n_classes;   /* classification: 0 = max(y) + 1 */
  double kl_eps;   /* class-probability smoothing in the KL loss; default 1e-7 */
  void* stream;    /* cudaStream_t to run on; NULL = legacy default stream */
  uint32_t job;    /* job id folded into every random stream (batches); default 0 */
  int host_inputs; /* 1: X and y are host pointers, copied to the device inside the call */
  int graph;       /* 1: each iteration is captured into a CUDA graph and replayed through one
                      executable graph, updated in place from iteration to iteration (same
                      results; per-level kernel times are then not recorded) */
  int split_path;  /* larger nodes: 0 = feature-band-sorted groups, in chunks of nodes (default),
                      1 = grouped items only; results are identical */
  int chunk_nodes; /* band path: at most this many larger nodes per chunk (0 = as many as the
                      plan buffers hold, the default); results are identical whatever the value,
                      a small value runs the multi-chunk path on small problems */
  int permut_form; /* Alg. 3 (task with BORUTA_PERMUT): 0 = each tree's out-of-bag rows against
                      that tree's prediction, one importance row per tree (default); 1 = Alg. 3
                      as printed: every row against the forest's prediction (mean over trees of
                      the leaves' class fractions or means), one importance row for the forest,
                      which is then the hit statistic (stat has no effect); its terms are FP64
                      whatever `precision` says */
  int forest_rows; /* permut_form = 1: rows per block of the (row, column) accumulators (0 = as
                      many as fit in about 1 GiB, the default); results are identical */
  int autotune;    /* 1: the first step of a session (of every job of a batch) times its
                      iteration once per histogram tile shape, restoring the state after each,
                      and keeps the fastest: column bytes per feature band (12, 24, 48, 96,
                      192 MiB) x one histogram launch per chunk of nodes or per band, and a
                      single band (no band order), at 8192 row-feature work per group of a
                      larger node, each run also timing every tree level; then the per-level
                      combination (at each level the shape whose level was fastest) at 8192,
                      4096 and 16384.  Results are identical for every shape
                      (boruta_session_tuning and boruta_session_tuning_levels report the
                      timings and the choice).  0 (default): 48 MiB, launches as
                      band_launch says, 8192. */
  int band_launch; /* without autotune: 0 (default) = by level: one histogram launch per feature
                      band (all warps on one band at a time) at the levels where a band holds at
                      least twice as many (node, band) groups as the GPU runs warps at once and
                      that either run in one chunk of nodes or have small groups (estimated
                      rows per node x items per band at most 1/8 of the group work; all
                      counted from the level's largest possible node count), else one per
                      chunk; 1 = one per band at every level; 2 = one per chunk at every
                      level.  Same results. */
} boruta_opts;

/* Host-side, caller-allocated outputs. */
typedef struct {
  int8_t* decision;    /* [p]: 1 accepted, 0 tentative, -1 rejected */
  int32_t* hits;       /* [p]: iterations in which the feature beat the best shadow */
  double* imp_history; /* [max_iter * p]: row t-1 = hit statistic at iteration t, NaN if not in play */
  double* shadow_max;  /* [max_iter]: best shadow statistic per iteration (NaN after the last) */
  int32_t iterations;  /* iterations run */
} boruta_result;

/* Fills opts with the defaults above. */
void boruta_default_opts(boruta_opts* opts);

/*
 * boruta_fit -- the whole of Alg. 1 on one problem.
 *   X        [in]  bins, column-major, column j at X + j*ld (see conventions)
 *   ld       [in]  column stride in bytes, >= N
 *   y        [in]  uint8 labels or int64 fixed-point targets, N entries
 *   N, p     [in]  rows and columns
 *   task     [in]  kind | importance (BORUTA_CLASSIFICATION/REGRESSION | BORUTA_TREEIMP/PERMUT)
 *   n_trees  [in]  trees per forest (M)
 *   max_depth[in]  root has depth 0; nodes at max_depth are leaves
 *   mtry     [in]  features tried per node; 0 = floor(sqrt(p_aug)) (classification) or
 *                  floor(p_aug/3) (regression), recomputed as columns are rejected
 *   n_bins   [in]  number of bins B; split thresholds are bins 0..B-2
 *   max_iter [in]  t_max of Alg. 1
 *   alpha    [in]  significance level before Bonferroni correction
 *   seed     [in]  key of every random stream
 *   opts     [in]  NULL = defaults
 *   out      [out] host buffers sized as documented in boruta_result
 */
int boruta_fit(const uint8_t* X, int64_t ld, const void* y, int64_t N, int64_t p, int task,
               int n_trees, int max_depth, int mtry, int n_bins, int max_iter, double alpha,
               uint64_t seed, const boruta_opts* opts, boruta_result* out);

/*
 * boruta_fit_batch -- many independent problems of uneven size (Alg. 1 on
 * each), run together: every job gets its own CUDA stream and workspace, and
 * the jobs' iterations are enqueued back to back so that their kernels
 * overlap on the GPU; a job drops out when it finishes.  Results are those of
 * boruta_fit on each job with opts->job + j as its job id (the job id keys
 * all of the job's random streams).
 *   jobs[j]  one problem, fields as the boruta_fit arguments of that name;
 *            n_classes overrides opts->n_classes for the job
 *   opts     shared options (NULL = defaults); opts->stream, if given, is
 *            waited on before the jobs start
 *   outs[j]  host result buffers of job j (as boruta_fit's)
 * On error every job's outputs are unspecified and the message names the
 * failing job. */
typedef struct {
  const uint8_t* X;
  int64_t ld;
  const void* y;
  int64_t N, p;
  int task, n_trees, max_depth, mtry, n_bins, max_iter;
  double alpha;
  uint64_t seed;
  int n_classes;
} boruta_job;

int boruta_fit_batch(int n_jobs, const boruta_job* jobs, const boruta_opts* opts, boruta_result* outs);

/*
 * Step-wise batch: boruta_fit_batch one lockstep iteration at a time.
 *   boruta_batch_create   arguments as boruta_fit_batch; the jobs' X and y
 *                         (device pointers) must stay valid until destroy
 *   boruta_batch_step     one iteration of every unfinished job; on return
 *                         the work is complete and opts->stream (if given)
 *                         has waited for it; *running receives the number of
 *                         jobs still unfinished (stepping with none left
 *                         returns BORUTA_EINVAL)
 *   boruta_batch_read     job j's state, as boruta_session_read
 *   boruta_batch_destroy  frees every job's workspace and stream (NULL ok)
 * Errors name the failing job; after an error in step the batch may only be
 * read or destroyed. */
typedef struct boruta_batch boruta_batch;

int boruta_batch_create(int n_jobs, const boruta_job* jobs, const boruta_opts* opts, boruta_batch** out);
int boruta_batch_step(boruta_batch* b, int32_t* running);
/* Up to `iterations` more iterations of every unfinished job, each job
 * advancing on its own as soon as its previous iteration completes (no
 * lockstep barrier); same results as as many boruta_batch_step calls. */
int boruta_batch_run(boruta_batch* b, int iterations, int32_t* running);
int boruta_batch_read(boruta_batch* b, int job, int8_t* decision, int32_t* hits, double* imp_history,
                      double* shadow_max, int32_t* t);
void boruta_batch_destroy(boruta_batch* b);

/* The number of this library's kernels all jobs of the batch have launched
 * since boruta_batch_create (the autotuner's timed iterations included). */
int boruta_batch_kernel_launches(boruta_batch* b, int64_t* kernels);

/*
 * Step-wise interface: the same computation one Boruta iteration at a time
 * (Alg. 1 loop body), for benchmarking, checkpoint/resume and inspection.
 * A session owns its device workspace; X and y must stay valid (device
 * pointers) until boruta_session_destroy.  Not thread-safe per session.
 */
typedef struct boruta_session boruta_session;

int boruta_session_create(const uint8_t* X, int64_t ld, const void* y, int64_t N, int64_t p,
                          int task, int n_trees, int max_depth, int mtry, int n_bins, int max_iter,
                          double alpha, uint64_t seed, const boruta_opts* opts,
                          boruta_session** out);

/* Runs iteration t+1.  *undecided receives the number of undecided features
 * after its test (0 or t == max_iter: the run is finished; stepping a
 * finished session returns BORUTA_EINVAL). */
int boruta_session_step(boruta_session* s, int32_t* undecided);

/* Copies the Boruta state to host buffers (any may be NULL): decision[p],
 * hits[p], imp_history[max_iter*p], shadow_max[max_iter], *t. */
int boruta_session_read(boruta_session* s, int8_t* decision, int32_t* hits, double* imp_history,
                        double* shadow_max, int32_t* t);

/* Restores a state read earlier (resume from a checkpoint): the next step
 * runs iteration t+1 and reproduces the uninterrupted run exactly. */
int boruta_session_write(boruta_session* s, const int8_t* decision, const int32_t* hits,
                         const double* imp_history, const double* shadow_max, int32_t t);

/* Dumps of the last completed iteration, for parity checks.  what:
 *   BORUTA_DUMP_SHADOW   uint8  [n_sha * N]   shadow columns (Alg. 1 X_sha)
 *   BORUTA_DUMP_BOOT     uint32 [M * N]       bootstrap draw counts per tree
 *   BORUTA_DUMP_IMP      double [M * p_aug]   per-tree importance rows ([p_aug], one forest row,
 *                                             with opts->permut_form = 1)
 *   BORUTA_DUMP_STAT     double [p_aug]       hit statistic per augmented column
 *   BORUTA_DUMP_NODES    boruta_node [count]  trees in order, each in (depth, heap) order
 *   BORUTA_DUMP_TREE_PTR int64  [M + 1]       offsets of each tree in the node dump
 *   BORUTA_DUMP_LIVE     int32  [p_live]      original columns in play
 *   BORUTA_DUMP_LEVELS   double [max_depth+1][3]  nodes at each depth, milliseconds
 *                        of the whole split stage at that depth, milliseconds
 *                        of its histogram kernels (0 for the last depth)
 * host must hold capacity bytes; *bytes receives the size needed (pass
 * host = NULL to query).  */
#define BORUTA_DUMP_SHADOW 1
#define BORUTA_DUMP_BOOT 2
#define BORUTA_DUMP_IMP 3
#define BORUTA_DUMP_STAT 4
#define BORUTA_DUMP_NODES 5
#define BORUTA_DUMP_TREE_PTR 6
#define BORUTA_DUMP_LIVE 7
#define BORUTA_DUMP_LEVELS 8
int boruta_session_dump(boruta_session* s, int what, void* host, int64_t capacity, int64_t* bytes);

/* Timing of the last step, from CUDA events on the session's stream (any
 * pointer may be NULL):
 *   hist_ms, hist_bytes  the histogram kernel of the larger nodes (per tree
 *                        level): total milliseconds and the method's
 *                        algorithmic bytes -- one bin per (row, sampled
 *                        feature) pair plus the row's state once per node
 *                        (entry read and rewritten, weight and label: 10 B;
 *                        17 B with the 8-byte regression target)
 *   launches             number of tree levels (histogram-kernel launches)
 *   split_ms, split_bytes the whole split stage of the levels (classify,
 *                        histograms, split records, partition), and its
 *                        algorithmic bytes (bins per (row, feature) pair, row
 *                        state once per node, partition traffic). */
int boruta_session_kernel_stats(boruta_session* s, double* hist_ms, int32_t* launches, double* hist_bytes,
                                double* split_ms, double* split_bytes);

/* The autotuner's measurements (opts->autotune = 1): *n_tried candidates, of
 * which the first `capacity` are written (any pointer may be NULL): the
 * row-feature work per group, the column bytes per band, 1 for one
 * histogram launch per band (0: per chunk), and the milliseconds of the
 * timed iteration; *chosen is the index kept (-1 before the first step or
 * without autotune). */
int boruta_session_tuning(boruta_session* s, int32_t capacity, int32_t* n_tried, uint32_t* group_work,
                          int64_t* band_bytes, int32_t* band_launch, double* ms, int32_t* chosen);

/* Per tree level (max_depth levels, *n_levels; the first `capacity` are
 * written; any pointer may be NULL): the column bytes per band the session
 * uses at that level, the launch mode of its last iteration there (1 per
 * band, 0 per chunk, -1 before the first step), and, when level_ms is given,
 * the autotuner's split-stage milliseconds of each level in each candidate
 * run, row-major [n_tried][capacity] (n_tried from boruta_session_tuning;
 * the caller allocates n_tried * capacity doubles).  In boruta_session_tuning
 * a candidate with band_bytes = band_launch = -1 is the per-level
 * combination. */
int boruta_session_tuning_levels(boruta_session* s, int32_t capacity, int32_t* n_levels, int64_t* band_bytes,
                                 int32_t* band_launch, double* level_ms);

/* The number of this library's kernels the last step launched (the whole
 * iteration: shadows, bootstrap, every level's split kernels, the importance
 * stage, the statistic and the test); 0 before the first step.  A step
 * replayed from a graph launches the same kernels. */
int boruta_session_kernel_launches(boruta_session* s, int64_t* kernels);

/* Timing of the last step's importance stage (Alg. 2 normalisation, or the
 * Alg. 3 tree walks and their reduction), from CUDA events on the session's
 * stream (0 when the step was replayed from a graph), and the number of
 * node visits of the Alg. 3 walks: every node whose split test a walk
 * applied, on the rows' own paths and on the re-walks with a feature's value
 * swapped (0 for TreeImp).  Either pointer may be NULL. */
int boruta_session_importance_stats(boruta_session* s, double* ms, double* node_visits);

void boruta_session_destroy(boruta_session* s);

/* One node of a dumped tree. heap id: root 0, children 2v+1 (left) and 2v+2. */
typedef struct {
  uint64_t heap;
  int32_t depth;
  int32_t feature;  /* augmented column (originals first, then shadows); -1 = leaf */
  int32_t bin;      /* rows with bin <= this go left */
  uint32_t n_rows;  /* distinct in-bag rows at the node */
  uint64_t n;       /* bootstrap-weighted rows */
  int64_t stat[8];  /* weighted class counts, or stat[0] = sum of w*y (regression) */
  double delta;     /* weighted impurity decrease of the split; 0 for leaves */
} boruta_node;

/* ---- device primitives, exposed for parity checks (device pointers) ----
 * boruta_philox: out[4k..4k+3] = Philox4x32-10(ctr[4k..4k+3], key[0..1]) for k < n
 *   (Salmon et al., SC'11), the generator behind every random draw.
 * boruta_perm: out[k] = sigma(idx[k]) for the keyed Feistel permutation of
 *   [0, n_domain) with counter words (w1, w2, w3) -- the Alg. 1 shuffle and
 *   Alg. 3 flush_index construction.
 * boruta_u256_to_double: out[k] = round-to-nearest-even of the 256-bit
 *   integer v[4k..4k+3] (little-endian u64 limbs).
 * boruta_binom_tails: for k < n, p_acc[k] = P(Bin(t[k], 1/2) >= h[k]) and
 *   p_rej[k] = P(Bin(t[k], 1/2) <= h[k]), each rounded once (Alg. 1 test). */
int boruta_philox(const uint32_t* ctr, const uint32_t* key, uint32_t* out, int64_t n, void* stream);
int boruta_perm(uint64_t n_domain, uint64_t seed, uint32_t w1, uint32_t w2, uint32_t w3,
                const uint64_t* idx, uint64_t* out, int64_t count, void* stream);
int boruta_u256_to_double(const uint64_t* v, double* out, int64_t n, void* stream);
int boruta_binom_tails(const int32_t* t, const int32_t* h, double* p_acc, double* p_rej, int64_t n,
                       void* stream);

/* boruta_binom_tails_noalloc -- the same results as boruta_binom_tails,
 * without allocating anything.  The paper has no counterpart: this entry
 * point exists for callers that may not allocate device memory (a host
 * program whose own allocator has reserved the GPU's memory, or a path
 * where cudaMalloc/cudaFree and the device synchronisation they can imply
 * are not allowed).  The binomial table lives in a fixed device array of
 * 258,080 bytes (C(t, k) for t <= 126 and an error word).
 *   t, h   [in]  device int32[n]; t must lie in [0, 126] (else BORUTA_EINVAL,
 *                and the entries with a bad t are written as NaN)
 *   p_acc, p_rej [out] device double[n], as for boruta_binom_tails
 *   stream [in]  cudaStream_t (NULL = legacy default stream); the call waits for it
 * The first call on a device looks up the array's address and fills the
 * table (with that device current).  With CUDA's default lazy module
 * loading that first call is also when the device loads the library's
 * module holding the array, which allocates the array and the module's
 * code: make the first call on each device before the caller's allocator
 * reserves that device's memory, or run with CUDA_MODULE_LOADING=EAGER.
 * Later calls allocate nothing.  No call may be made while its stream is
 * being captured into a CUDA graph (each call copies the error word to
 * pageable host memory and synchronises the stream).  All calls share the
 * array: its error word is cleared at the start of each call, and calls
 * that overlap on the GPU race on it. */
int boruta_binom_tails_noalloc(const int32_t* t, const int32_t* h, double* p_acc, double* p_rej,
                               int64_t n, void* stream);

/* ---- after the run (host computations on host buffers; no GPU work) ----
 *
 * boruta_rank -- Alg. 1's final ranking of a finished run.  The algorithm's
 *   rankdata line is garbled; the reading taken: accepted features rank 1,
 *   tentative ones 2, rejected ones 3, 4, ... in descending order of the
 *   median of their history (the rows 0..iterations-1 of imp_history,
 *   [max_iter][p] as boruta_result holds it, NaN entries -- iterations out of
 *   play -- skipped), equal medians to the lower column index.
 *   decision [in] p values in {-1, 0, 1};  rank [out] int32[p].
 *
 * boruta_select_median -- the selection of the paper's synthetic study, which
 *   ran 20 seeds and selected on the median importance (Sec. 3.1); the
 *   reading taken: per run r, the median of each feature's history and the
 *   median of the run's shadow maxima; median_imp[j] and *median_shadow are
 *   the medians of those over the runs, and selected[j] = 1 when median_imp[j]
 *   > *median_shadow (strict).  Medians skip NaN and take the mean of the two
 *   middle values of an even count.
 *   iterations [in] int32[n_runs]; imp_history [in] [n_runs][max_iter][p];
 *   shadow_max [in] [n_runs][max_iter]; median_imp [out] double[p];
 *   selected [out] int8[p].
 *
 * boruta_fit_seeds -- boruta_fit on one problem for each of n_seeds seeds,
 *   run as independent jobs of one batch (boruta_fit_batch; job j uses
 *   seeds[j] and the job id opts->job + j), then boruta_select_median over
 *   the runs.  outs[j] receives run j (host buffers as boruta_fit's); X and y
 *   as for boruta_fit (device pointers unless opts->host_inputs = 1).
 *
 * All three return BORUTA_EINVAL for bad sizes or NULL buffers. */
int boruta_rank(const int8_t* decision, const double* imp_history, int64_t p, int32_t iterations, int32_t* rank);
int boruta_select_median(int n_runs, int64_t p, int32_t max_iter, const int32_t* iterations,
                         const double* imp_history, const double* shadow_max, double* median_imp,
                         double* median_shadow, int8_t* selected);
int boruta_fit_seeds(const uint8_t* X, int64_t ld, const void* y, int64_t N, int64_t p, int task, int n_trees,
                     int max_depth, int mtry, int n_bins, int max_iter, double alpha, int n_seeds,
                     const uint64_t* seeds, const boruta_opts* opts, boruta_result* outs, double* median_imp,
                     double* median_shadow, int8_t* selected);

/*
 * boruta_quantise -- float features to the uint8 bins the fit consumes (a
 * helper outside the iteration; the paper does not say how features are
 * binned).  bin(x) = min(B-1, floor(B * rank(x) / N)) with rank(x) the number
 * of values of the column strictly below x, so equal values share a bin and
 * -0 equals +0.
 *   X     [in]  device float32, column-major: column j at X + j*ldx, N values
 *   Xb    [out] device uint8 bins, column j at Xb + j*ldb (ldx, ldb >= N)
 *   n_bins      B in [2, 256]; N < 2^24
 *   stream      cudaStream_t (NULL = legacy default); the call waits for it
 * NaN in X returns BORUTA_EINVAL (Xb then unspecified).  Allocates 4 bytes
 * of stream-ordered scratch. */
int boruta_quantise(const float* X, int64_t ldx, int64_t N, int64_t p, int n_bins, uint8_t* Xb, int64_t ldb,
                    void* stream);

/* Message for the last error on this thread ("" if none). */
const char* boruta_last_error(void);

#ifdef __cplusplus
}
#endif
#endif
