/*
 * CPU oracle for GPU Boruta (Li et al., "Novel GPU Boruta algorithms for
 * feature selection from high-dimensional data").
 *
 * TEST INFRASTRUCTURE ONLY.  This library is the plain, slow, obviously
 * correct statement of what the CUDA path computes.  Only the test suite,
 * the smoke check and the benchmark's CPU-baseline leg may load it; the
 * product path never links, imports or calls it.  It shares no source with
 * the CUDA library: its Philox, Feistel permutation, exact integer
 * arithmetic and summation are written here, separately.
 *
 * What it follows:
 *   - Alg. 1 (Boruta outer loop, shadow features, hits, test)
 *   - Alg. 2 (impurity-decrease importance, "gain x samples" per split node,
 *     per-tree normalisation, mean over trees)
 *   - Alg. 3 (permutation importance: one row permutation shared by all
 *     features, loss against the model's own unpermuted prediction),
 *     restricted to each tree's out-of-bag rows
 *   - Sec. 2 text: MSE for regression, KL divergence of predicted class
 *     probabilities for classification
 * and, where the paper is silent (bootstrap, mtry, split criterion, the
 * significance test, random streams), the readings listed in the design
 * notes of the repository.
 */
#ifndef BORUTA_ORACLE_H
#define BORUTA_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ORC_MAX_CLASSES 8
#define ORC_MAX_DEPTH 30

/* Philox counter purposes (high byte of counter word 3). */
#define ORC_P_SHADOW 1u
#define ORC_P_BOOT 2u
#define ORC_P_MTRY 3u
#define ORC_P_PERMUT 4u

/* task = kind | importance */
#define ORC_CLASSIFICATION 0
#define ORC_REGRESSION 1
#define ORC_TREEIMP 0
#define ORC_PERMUT 2

typedef struct {
  const uint8_t* X;     /* column-major bins, column j at X + j*ld */
  int64_t ld;           /* column stride in bytes, >= N */
  const uint8_t* ycls;  /* class labels (classification) or NULL */
  const int64_t* yreg;  /* targets as fixed point, units of 2^-20 (regression) */
  int64_t N, p;
  int task;             /* kind | importance */
  int n_classes;        /* classification only; labels must be < n_classes */
  int n_trees, max_depth, mtry /* 0 = default */, n_bins, max_iter;
  double alpha;
  uint64_t seed;
  uint32_t job;
  int stat;             /* 0 = Z score (mean / (sd / sqrt(M))), 1 = mean */
  double kl_eps;        /* smoothing of class probabilities in the KL loss */
  int tie_break;        /* equal scores: 0 = lowest feature index, 1 = first drawn feature; then lowest bin */
  int permut_form;      /* Alg. 3 rows: 0 = each tree's OOB rows against that tree's prediction,
                           1 = every row against the forest's prediction (the printed algorithm;
                           one importance per column, which is then the hit statistic) */
} orc_problem;

/* One tree node, as dumped for parity checks.  Trees are listed in
 * (depth, heap id) order; heap id: root 0, children 2v+1 (left), 2v+2. */
typedef struct {
  uint64_t heap;
  int32_t depth;
  int32_t feature;      /* augmented column index, -1 for a leaf */
  int32_t bin;          /* split: bin <= threshold goes left */
  uint32_t n_rows;      /* distinct in-bag rows reaching the node */
  uint64_t n;           /* bootstrap-weighted row count */
  int64_t stat[ORC_MAX_CLASSES]; /* weighted class counts, or stat[0] = sum w*y */
  double delta;         /* weighted impurity decrease of the split (0 for leaves) */
} orc_node;

/* ---- random streams ---- */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
uint32_t orc_fmix32(uint32_t x);
/* sigma(idx[k]) for the keyed Feistel permutation of [0, n). */
void orc_perm(uint64_t n, uint64_t seed, uint32_t w1, uint32_t w2, uint32_t w3,
              const uint64_t* idx, uint64_t* out, int64_t count);
void orc_bootstrap(uint64_t seed, uint32_t job, int t, int tree, int64_t N, uint32_t* counts);
void orc_mtry(uint64_t seed, uint32_t job, int t, int tree, uint32_t heap, int64_t p_aug,
              int mtry, uint32_t* feats);
int64_t orc_default_mtry(int task, int64_t p_aug);
int64_t orc_shadow_count(int64_t p_live);
/* Shadow matrix of iteration t: n_sha columns of N bytes each. */
void orc_shadow(const orc_problem* P, int t, const int32_t* live, int64_t p_live,
                uint8_t* Xsha);
/* Alg. 3 flush_index of iteration t: pi[i] for i in [0, N). */
void orc_permut_table(const orc_problem* P, int t, uint64_t* pi);

/* ---- exact arithmetic (test hooks) ---- */
/* sign of a1*b1 - a2*b2 for 256-bit a and 256-bit b (little-endian u64 limbs);
 * returns 2 if a product overflows 256 bits. */
int orc_cmp_products(const uint64_t a1[4], const uint64_t b1[4],
                     const uint64_t a2[4], const uint64_t b2[4]);
double orc_u256_to_double(const uint64_t a[4]);
double orc_exact_sum(const double* x, int64_t n);
void orc_binom_tails(int t, int h, double* p_acc, double* p_rej,
                     uint64_t upper[2], uint64_t lower[2]);

/* Best split of one explicit node (for brute-force checks).
 *   bins: nrows x nf, row-major; weights w[nrows]; labels / targets y.
 *   feats: candidate feature indices into [0, nf); among equal scores the
 *   feature listed first wins, then the lowest bin.
 * Returns 1 and fills feature/bin/delta if a split with delta > 0 exists. */
int orc_node_split(int task, int n_classes, int n_bins, int64_t nrows, int64_t nf,
                   const uint8_t* bins, const uint32_t* w, const uint8_t* ycls,
                   const int64_t* yreg, const int32_t* feats, int nfeats,
                   int32_t* feature, int32_t* bin, double* delta);

/* ---- one tree of one iteration ----
 * live[p_live]: the original columns in play (ascending); Xsha from orc_shadow.
 * Writes up to cap nodes ((depth, heap) order), the tree's TreeImp row
 * (normalised, p_aug doubles) and/or its OOB permutation-importance row. */
int orc_tree(const orc_problem* P, int t, const int32_t* live, int64_t p_live,
             const uint8_t* Xsha, int tree, orc_node* nodes, int64_t cap,
             int64_t* n_nodes, double* imp_treeimp, double* imp_permut);

/* ---- Alg. 3 as printed: all N rows, the forest's averaged prediction ----
 * imp[p_aug]: mean over rows of the loss between the forest's prediction and
 * its prediction with column f read at flush_index (see forest.c). */
int orc_forest_permut(const orc_problem* P, int t, const int32_t* live, int64_t p_live,
                      const uint8_t* Xsha, double* imp);

/* ---- the test of Alg. 1 alone ----
 * state[p] (1 accepted, 0 undecided, -1 rejected) is updated in place from
 * the hit counts after iteration t. */
void orc_decide(int t, double alpha, int64_t p, const int32_t* hits, int8_t* state);

/* ---- one Boruta iteration (Alg. 1 loop body) ----
 * state/hits are updated in place; hist_row[p] receives the hit statistic of
 * each live feature (NaN otherwise); imp (n_trees x p_aug) and s (p_aug) are
 * optional dumps (with permut_form = 1, imp holds one row of p_aug). */
int orc_iteration(const orc_problem* P, int t, int8_t* state, int32_t* hits,
                  double* hist_row, double* shadow_max, double* imp, double* s,
                  int64_t* p_aug_out);

/* ---- after the run ----
 * orc_rank: Alg. 1's final ranking (its rankdata line is garbled; reading):
 *   accepted 1, undecided 2, rejected 3, 4, ... by descending median of the
 *   feature's history (iterations 1..iterations of imp_history, [max_iter][p],
 *   NaN entries skipped), equal medians to the lower index.
 * orc_select_median: the multi-seed selection of the paper's synthetic study
 *   (20 runs, "the median importance as the basis for the final selection";
 *   reading): per run r, m_rj = median of feature j's history and m_r = median
 *   of the run's shadow maxima; med_imp[j] = median over runs of m_rj,
 *   *med_shadow = median over runs of m_r; selected[j] = med_imp[j] >
 *   *med_shadow.  imp_history is [n_runs][max_iter][p], shadow_max
 *   [n_runs][max_iter]; medians of an even count take the mean of the two
 *   middle values. */
void orc_rank(int64_t p, int32_t iterations, const int8_t* decision, const double* imp_history,
              int32_t* rank);
void orc_select_median(int n_runs, int64_t p, int32_t max_iter, const int32_t* iterations,
                       const double* imp_history, const double* shadow_max, double* med_imp,
                       double* med_shadow, int8_t* selected);

/* ---- the whole run ---- */
int orc_boruta(const orc_problem* P, int8_t* decision, int32_t* hits,
               double* imp_history, double* shadow_max, int32_t* iterations);

#ifdef __cplusplus
}
#endif
#endif
