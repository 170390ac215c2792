/*
 * Oracle random forest, TreeImp and OOB permutation importance.
 * TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * One tree (the forest fit of Alg. 1, "M <- fit([X_cur || X_sha], y)", with
 * cuML's silent defaults read as Breiman's forest):
 *   - bootstrap: N draws with replacement; a row's weight is its draw count;
 *   - each node tries the mtry features of its own feature sample;
 *   - candidate split (f, b): rows with bin <= b go left, b in [0, B-2],
 *     valid if both sides have positive weight;
 *   - criterion, maximised exactly over integers:
 *       classification (Gini):  A_L/n_L + A_R/n_R,  A = sum_k c_k^2
 *       regression (variance):  S_L^2/n_L + S_R^2/n_R,  S = sum w*y
 *     ties go to the lowest feature index (or, with tie_break = 1, to the
 *     feature drawn first in the node's sample), then to the lowest bin;
 *   - a node is a leaf at depth max_depth, when no candidate is valid, or
 *     when the best split does not decrease impurity (delta <= 0).
 *
 * delta, "gain x samples" of Alg. 2 (CalcNodeImp), is the weighted impurity
 * decrease n_P*I_P - n_L*I_L - n_R*I_R, which for both criteria equals
 *   score(split) - score(parent),  score(parent) = A_P/n_P  or  S_P^2/n_P.
 * It is formed exactly as num/den and rounded as RN(num) / RN(den).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "exact.h"

typedef struct {
  uint64_t n;
  uint64_t cnt[ORC_MAX_CLASSES];
  int64_t S;
} stats_t;

typedef struct {
  int kind; /* ORC_CLASSIFICATION or ORC_REGRESSION */
  int C, B;
  const uint8_t* ycls;
  const int64_t* yreg;
  const uint8_t* const* col; /* column pointers, indexed by row id */
} data_t;

static void stats_add_row(stats_t* s, const data_t* d, uint32_t row, uint64_t w) {
  s->n += w;
  if (d->kind == ORC_CLASSIFICATION)
    s->cnt[d->ycls[row]] += w;
  else
    s->S += (int64_t)w * d->yreg[row];
}

static void stats_sub(stats_t* r, const stats_t* a, const stats_t* b, int C) {
  r->n = a->n - b->n;
  for (int k = 0; k < C; k++) r->cnt[k] = a->cnt[k] - b->cnt[k];
  r->S = a->S - b->S;
}

/* A = sum_k c_k^2 (classification) or S^2 (regression) */
static u256 sq_term(const stats_t* s, const data_t* d) {
  if (d->kind == ORC_CLASSIFICATION) {
    unsigned __int128 A = 0;
    for (int k = 0; k < d->C; k++) A += (unsigned __int128)s->cnt[k] * s->cnt[k];
    return u256_from_u128(A);
  }
  uint64_t m = s->S < 0 ? (uint64_t)0 - (uint64_t)s->S : (uint64_t)s->S;
  return u256_from_u128((unsigned __int128)m * m);
}

/* split score as num/den: (A_L n_R + A_R n_L) / (n_L n_R) */
static void split_score(const stats_t* L, const stats_t* R, const data_t* d, u256* num,
                        u256* den, int* of) {
  u256 aL = sq_term(L, d), aR = sq_term(R, d);
  u256 t1 = u256_mul(aL, u256_from_u64(R->n), of);
  u256 t2 = u256_mul(aR, u256_from_u64(L->n), of);
  *num = u256_add(t1, t2);
  *den = u256_mul(u256_from_u64(L->n), u256_from_u64(R->n), of);
}

/* x1/y1 > x2/y2 for positive denominators */
static int frac_gt(u256 x1, u256 y1, u256 x2, u256 y2, int* of) {
  return u256_cmp(u256_mul(x1, y2, of), u256_mul(x2, y1, of)) > 0;
}

typedef struct {
  int found;
  int32_t f, b;
  stats_t left;
  u256 num, den;
} best_t;

static int cmp_u32(const void* a, const void* b) {
  uint32_t x = *(const uint32_t*)a, y = *(const uint32_t*)b;
  return (x > y) - (x < y);
}

/* Exhaustive search over the node's candidate splits, features in the
 * given order; the first of equal scores is kept. */
static void node_search(const data_t* d, const uint32_t* rows, const uint32_t* w, int64_t nrows,
                        const stats_t* parent, const uint32_t* feats, int nfeats,
                        best_t* best, int* of) {
  stats_t* hist = (stats_t*)malloc(sizeof(stats_t) * (size_t)d->B);
  best->found = 0;
  for (int fi = 0; fi < nfeats; fi++) {
    uint32_t f = feats[fi];
    memset(hist, 0, sizeof(stats_t) * (size_t)d->B);
    for (int64_t r = 0; r < nrows; r++) stats_add_row(&hist[d->col[f][rows[r]]], d, rows[r], w[r]);
    stats_t left;
    memset(&left, 0, sizeof left);
    for (int b = 0; b + 1 < d->B; b++) {
      left.n += hist[b].n;
      for (int k = 0; k < d->C; k++) left.cnt[k] += hist[b].cnt[k];
      left.S += hist[b].S;
      if (left.n == 0 || left.n == parent->n) continue;
      stats_t right;
      stats_sub(&right, parent, &left, d->C);
      u256 num, den;
      split_score(&left, &right, d, &num, &den, of);
      if (!best->found || frac_gt(num, den, best->num, best->den, of)) {
        best->found = 1;
        best->f = (int32_t)f;
        best->b = b;
        best->left = left;
        best->num = num;
        best->den = den;
      }
    }
  }
  free(hist);
}

/* delta = num/den - parent_score, exactly; returns 0 if delta <= 0 */
static int split_delta(const best_t* bs, const stats_t* parent, const data_t* d, double* delta,
                       int* of) {
  u256 pnum = sq_term(parent, d);
  u256 pden = u256_from_u64(parent->n);
  u256 lhs = u256_mul(bs->num, pden, of);
  u256 rhs = u256_mul(pnum, bs->den, of);
  if (u256_cmp(lhs, rhs) <= 0) return 0;
  u256 dnum = u256_sub(lhs, rhs);
  u256 dden = u256_mul(bs->den, pden, of);
  *delta = u256_to_double(dnum) / u256_to_double(dden);
  return 1;
}

int orc_node_split(int task, int n_classes, int n_bins, int64_t nrows, int64_t nf,
                   const uint8_t* bins, const uint32_t* w, const uint8_t* ycls,
                   const int64_t* yreg, const int32_t* feats, int nfeats, int32_t* feature,
                   int32_t* bin, double* delta) {
  uint8_t** cols = (uint8_t**)malloc(sizeof(uint8_t*) * (size_t)nf);
  for (int64_t f = 0; f < nf; f++) {
    cols[f] = (uint8_t*)malloc((size_t)nrows);
    for (int64_t r = 0; r < nrows; r++) cols[f][r] = bins[r * nf + f];
  }
  data_t d = {task & 1, n_classes, n_bins, ycls, yreg, (const uint8_t* const*)cols};
  uint32_t* rows = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)nrows);
  stats_t parent;
  memset(&parent, 0, sizeof parent);
  for (int64_t r = 0; r < nrows; r++) {
    rows[r] = (uint32_t)r;
    stats_add_row(&parent, &d, (uint32_t)r, w[r]);
  }
  uint32_t* fs = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(nfeats > 0 ? nfeats : 1));
  for (int k = 0; k < nfeats; k++) fs[k] = (uint32_t)feats[k];
  best_t bs;
  int of = 0;
  node_search(&d, rows, w, nrows, &parent, fs, nfeats, &bs, &of);
  int ok = 0;
  if (bs.found && parent.n > 0) ok = split_delta(&bs, &parent, &d, delta, &of);
  if (ok) {
    *feature = bs.f;
    *bin = bs.b;
  }
  for (int64_t f = 0; f < nf; f++) free(cols[f]);
  free(cols);
  free(rows);
  free(fs);
  return of ? -2 : ok;
}

/* ---------------- one tree ---------------- */

typedef struct {
  const orc_problem* P;
  data_t d;
  int t, tree, D, mtry;
  int64_t p_aug;
  orc_node* nodes; /* pre-order (DFS) as built */
  int64_t* left;
  int64_t* right;
  int64_t n, cap;
  int of;
  int err;
} tree_t;

static int64_t grow(tree_t* T, uint64_t heap, int depth, const uint32_t* rows, const uint32_t* w,
                    int64_t nrows) {
  if (T->n >= T->cap) {
    T->err = 1;
    return -1;
  }
  stats_t st;
  memset(&st, 0, sizeof st);
  for (int64_t r = 0; r < nrows; r++) stats_add_row(&st, &T->d, rows[r], w[r]);
  int64_t idx = T->n++;
  orc_node* nd = &T->nodes[idx];
  memset(nd, 0, sizeof *nd);
  nd->heap = heap;
  nd->depth = depth;
  nd->feature = -1;
  nd->n_rows = (uint32_t)nrows;
  nd->n = st.n;
  if (T->d.kind == ORC_CLASSIFICATION)
    for (int k = 0; k < T->d.C; k++) nd->stat[k] = (int64_t)st.cnt[k];
  else
    nd->stat[0] = st.S;
  T->left[idx] = T->right[idx] = -1;
  if (depth >= T->D || nrows < 1) return idx;

  uint32_t* feats = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)T->mtry);
  orc_mtry(T->P->seed, T->P->job, T->t, T->tree, (uint32_t)heap, T->p_aug, T->mtry, feats);
  if (T->P->tie_break == 0) qsort(feats, (size_t)T->mtry, sizeof(uint32_t), cmp_u32);
  best_t bs;
  node_search(&T->d, rows, w, nrows, &st, feats, T->mtry, &bs, &T->of);
  free(feats);
  double delta = 0.0;
  if (!bs.found || !split_delta(&bs, &st, &T->d, &delta, &T->of)) return idx;

  nd->feature = bs.f;
  nd->bin = bs.b;
  nd->delta = delta;
  uint32_t* lr = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)nrows * 2);
  uint32_t* lw = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)nrows * 2);
  int64_t nl = 0, nr = 0;
  for (int64_t r = 0; r < nrows; r++) /* left rows first, in order */
    if (T->d.col[bs.f][rows[r]] <= bs.b) {
      lr[nl] = rows[r];
      lw[nl] = w[r];
      nl++;
    }
  for (int64_t r = 0; r < nrows; r++)
    if (T->d.col[bs.f][rows[r]] > bs.b) {
      lr[nl + nr] = rows[r];
      lw[nl + nr] = w[r];
      nr++;
    }
  int64_t li = grow(T, 2 * heap + 1, depth + 1, lr, lw, nl);
  int64_t ri = grow(T, 2 * heap + 2, depth + 1, lr + nl, lw + nl, nr);
  T->left[idx] = li;
  T->right[idx] = ri;
  free(lr);
  free(lw);
  return idx;
}

/* leaf reached by row `row`; if f >= 0, column f reads row `prow` instead */
static int64_t predict(const tree_t* T, uint32_t row, int64_t f, uint32_t prow) {
  int64_t k = 0;
  while (T->nodes[k].feature >= 0) {
    int32_t g = T->nodes[k].feature;
    uint8_t v = (g == f) ? T->d.col[g][prow] : T->d.col[g][row];
    k = (v <= T->nodes[k].bin) ? T->left[k] : T->right[k];
  }
  return k;
}

/* Loss between the unpermuted prediction (leaf q) and the permuted one
 * (leaf q2), Sec. 2 / Alg. 3 LossFunction:
 *   regression:     squared difference of the leaf means (real units)
 *   classification: KL(P_q || P_q2) over the leaves' smoothed class
 *                   fractions, P~_k = (c_k/n + eps) / (1 + C*eps). */
static double loss(const tree_t* T, int64_t q, int64_t q2) {
  const orc_node* a = &T->nodes[q];
  const orc_node* b = &T->nodes[q2];
  if (T->d.kind == ORC_REGRESSION) {
    double mu_a = (double)a->stat[0] / (double)a->n;
    double mu_b = (double)b->stat[0] / (double)b->n;
    double diff = (mu_a - mu_b) * 0x1p-20;
    return diff * diff;
  }
  double eps = T->P->kl_eps;
  double norm = 1.0 + (double)T->d.C * eps;
  double kl = 0.0;
  for (int k = 0; k < T->d.C; k++) {
    double pa = ((double)a->stat[k] / (double)a->n + eps) / norm;
    double pb = ((double)b->stat[k] / (double)b->n + eps) / norm;
    kl += pa * log(pa / pb);
  }
  return kl;
}

typedef struct {
  int32_t f;
  int64_t order;
  double v;
} fd_t;

static int cmp_fd(const void* a, const void* b) {
  const fd_t* x = (const fd_t*)a;
  const fd_t* y = (const fd_t*)b;
  if (x->f != y->f) return (x->f > y->f) - (x->f < y->f);
  return (x->order > y->order) - (x->order < y->order);
}

static int cmp_node_level(const void* a, const void* b) {
  const orc_node* x = (const orc_node*)a;
  const orc_node* y = (const orc_node*)b;
  if (x->depth != y->depth) return (x->depth > y->depth) - (x->depth < y->depth);
  return (x->heap > y->heap) - (x->heap < y->heap);
}

/* Column pointers of the augmented matrix [X_cur || X_sha]. */
static const uint8_t** aug_columns(const orc_problem* P, const int32_t* live, int64_t p_live,
                                   const uint8_t* Xsha, int64_t* p_aug) {
  int64_t n_sha = orc_shadow_count(p_live);
  *p_aug = p_live + n_sha;
  const uint8_t** col = (const uint8_t**)malloc(sizeof(uint8_t*) * (size_t)*p_aug);
  for (int64_t a = 0; a < p_live; a++) col[a] = P->X + (int64_t)live[a] * P->ld;
  for (int64_t c = 0; c < n_sha; c++) col[p_live + c] = Xsha + c * P->N;
  return col;
}

/* Fits tree `tree` of iteration t: bootstrap (counts into cnt[N]), then the
 * recursive growth from the root.  Returns 0, or -1 / -2 (pool / 256-bit
 * bound); the caller frees the tree with tree_free. */
static int tree_fit(tree_t* T, const orc_problem* P, int t, int tree, const uint8_t** col,
                    int64_t p_aug, uint32_t* cnt) {
  int64_t N = P->N;
  memset(T, 0, sizeof *T);
  T->P = P;
  T->d.kind = P->task & 1;
  T->d.C = (T->d.kind == ORC_CLASSIFICATION) ? P->n_classes : 1;
  T->d.B = P->n_bins;
  T->d.ycls = P->ycls;
  T->d.yreg = P->yreg;
  T->d.col = col;
  T->t = t;
  T->tree = tree;
  T->D = P->max_depth;
  T->p_aug = p_aug;
  T->mtry = (int)(P->mtry > 0 ? (P->mtry < p_aug ? P->mtry : p_aug)
                              : orc_default_mtry(P->task, p_aug));
  T->cap = 2 * N + 1;
  T->nodes = (orc_node*)malloc(sizeof(orc_node) * (size_t)T->cap);
  T->left = (int64_t*)malloc(sizeof(int64_t) * (size_t)T->cap);
  T->right = (int64_t*)malloc(sizeof(int64_t) * (size_t)T->cap);

  /* bootstrap: in-bag rows ascending with their draw counts */
  orc_bootstrap(P->seed, P->job, t, tree, N, cnt);
  uint32_t* rows = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)N);
  uint32_t* w = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)N);
  int64_t nin = 0;
  for (int64_t i = 0; i < N; i++)
    if (cnt[i]) {
      rows[nin] = (uint32_t)i;
      w[nin] = cnt[i];
      nin++;
    }
  grow(T, 0, 0, rows, w, nin);
  free(rows);
  free(w);
  return T->err ? -1 : (T->of ? -2 : 0);
}

static void tree_free(tree_t* T) {
  free(T->nodes);
  free(T->left);
  free(T->right);
}

int orc_tree(const orc_problem* P, int t, const int32_t* live, int64_t p_live,
             const uint8_t* Xsha, int tree, orc_node* nodes_out, int64_t cap, int64_t* n_nodes,
             double* imp_treeimp, double* imp_permut) {
  int64_t N = P->N;
  int64_t p_aug;
  const uint8_t** col = aug_columns(P, live, p_live, Xsha, &p_aug);
  tree_t T;
  uint32_t* cnt = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)N);
  int rc = tree_fit(&T, P, t, tree, col, p_aug, cnt);

  /* Alg. 2: per tree, gain x samples summed per feature, then divided by
   * the tree's total.  Sums are exact, rounded once. */
  if (rc == 0 && imp_treeimp) {
    fd_t* fd = (fd_t*)malloc(sizeof(fd_t) * (size_t)(T.n + 1));
    int64_t m = 0;
    for (int64_t k = 0; k < T.n; k++) /* pre-order, the order CalcNodeImp visits */
      if (T.nodes[k].feature >= 0) {
        fd[m].f = T.nodes[k].feature;
        fd[m].order = k;
        fd[m].v = T.nodes[k].delta;
        m++;
      }
    qsort(fd, (size_t)m, sizeof(fd_t), cmp_fd);
    double* g = (double*)calloc((size_t)p_aug, sizeof(double));
    double* vals = (double*)malloc(sizeof(double) * (size_t)(m + 1));
    for (int64_t a = 0; a < m;) {
      int64_t b = a;
      while (b < m && fd[b].f == fd[a].f) {
        vals[b - a] = fd[b].v;
        b++;
      }
      g[fd[a].f] = exact_sum(vals, b - a, 1);
      a = b;
    }
    double tot = exact_sum(g, p_aug, 1);
    for (int64_t j = 0; j < p_aug; j++) imp_treeimp[j] = tot > 0.0 ? g[j] / tot : 0.0;
    free(g);
    free(vals);
    free(fd);
  }

  /* Alg. 3 over the tree's out-of-bag rows: for every feature, swap in
   * the column value of row flush_index[i] and compare the prediction
   * with the tree's own unpermuted prediction. */
  if (rc == 0 && imp_permut) {
    uint64_t* pi = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)N);
    orc_permut_table(P, t, pi);
    int64_t n_oob = 0;
    uint32_t* oob = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(N + 1));
    for (int64_t i = 0; i < N; i++)
      if (cnt[i] == 0) oob[n_oob++] = (uint32_t)i;
    int64_t* base = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n_oob + 1));
    for (int64_t r = 0; r < n_oob; r++) base[r] = predict(&T, oob[r], -1, 0);
    double* L = (double*)malloc(sizeof(double) * (size_t)(n_oob + 1));
    for (int64_t f = 0; f < p_aug; f++) {
      for (int64_t r = 0; r < n_oob; r++) {
        int64_t q2 = predict(&T, oob[r], f, (uint32_t)pi[oob[r]]);
        L[r] = loss(&T, base[r], q2);
      }
      imp_permut[f] = n_oob > 0 ? exact_sum(L, n_oob, 1) / (double)n_oob : 0.0;
    }
    free(L);
    free(base);
    free(oob);
    free(pi);
  }

  if (rc == 0 && nodes_out) {
    if (T.n > cap) {
      rc = -1;
    } else {
      memcpy(nodes_out, T.nodes, sizeof(orc_node) * (size_t)T.n);
      qsort(nodes_out, (size_t)T.n, sizeof(orc_node), cmp_node_level);
    }
  }
  if (n_nodes) *n_nodes = T.n;
  free(cnt);
  tree_free(&T);
  free(col);
  return rc;
}

/* ---------------- Alg. 3 as printed: every row, the forest's prediction ----------------
 *
 * The model is the whole forest: its prediction for a row is the mean over
 * the M trees of the leaf's value -- the class fractions c_k/n of the leaf
 * (predicted class probabilities) or the leaf mean S/n (regression, units of
 * 2^-20).  y_gpu is the forest's prediction for every row of
 * [X_cur || X_sha]; for each augmented column f, that column is replaced by
 * its values at flush_index (one permutation of the N rows per iteration,
 * shared by all columns), every row is predicted again, and imp[f] is the
 * mean over the N rows of the loss between the two predictions: the squared
 * difference in real units (regression), or KL(P~_base || P~_perm) of the
 * smoothed class probabilities P~_k = (P_k + eps) / (1 + C eps).
 * Each mean over trees is the exact sum of the per-tree doubles rounded
 * once, then divided by M; the mean over rows is exact, rounded once. */

static double leaf_value(const tree_t* T, int64_t q, int k) {
  const orc_node* nd = &T->nodes[q];
  return (double)nd->stat[k] / (double)nd->n;
}

static double forest_loss(const orc_problem* P, int kind, int C, const double* a, const double* b) {
  if (kind == ORC_REGRESSION) {
    double diff = (a[0] - b[0]) * 0x1p-20;
    return diff * diff;
  }
  double eps = P->kl_eps;
  double norm = 1.0 + (double)C * eps;
  double kl = 0.0;
  for (int k = 0; k < C; k++) {
    double pa = (a[k] + eps) / norm;
    double pb = (b[k] + eps) / norm;
    kl += pa * log(pa / pb);
  }
  return kl;
}

int orc_forest_permut(const orc_problem* P, int t, const int32_t* live, int64_t p_live,
                      const uint8_t* Xsha, double* imp) {
  int64_t N = P->N, M = P->n_trees;
  int64_t p_aug;
  const uint8_t** col = aug_columns(P, live, p_live, Xsha, &p_aug);
  tree_t* T = (tree_t*)calloc((size_t)M, sizeof(tree_t));
  uint32_t* cnt = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)N);
  int rc = 0;
  int64_t built = 0;
  for (; built < M && rc == 0; built++) rc = tree_fit(&T[built], P, t, (int)built, col, p_aug, cnt);
  free(cnt);
  if (rc == 0) {
    int kind = P->task & 1;
    int K = kind == ORC_CLASSIFICATION ? P->n_classes : 1;
    uint64_t* pi = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)N);
    orc_permut_table(P, t, pi);
    double* vals = (double*)malloc(sizeof(double) * (size_t)M);
    double* base = (double*)malloc(sizeof(double) * (size_t)(N * K));
    double* perm = (double*)malloc(sizeof(double) * (size_t)K);
    double* L = (double*)malloc(sizeof(double) * (size_t)N);
    int64_t* leaf = (int64_t*)malloc(sizeof(int64_t) * (size_t)M);
    for (int64_t i = 0; i < N; i++) { /* y_gpu: the forest's own prediction */
      for (int64_t tau = 0; tau < M; tau++) leaf[tau] = predict(&T[tau], (uint32_t)i, -1, 0);
      for (int k = 0; k < K; k++) {
        for (int64_t tau = 0; tau < M; tau++) vals[tau] = leaf_value(&T[tau], leaf[tau], k);
        base[i * K + k] = exact_sum(vals, M, 1) / (double)M;
      }
    }
    for (int64_t f = 0; f < p_aug; f++) {
      for (int64_t i = 0; i < N; i++) { /* column f read at flush_index[i] */
        for (int64_t tau = 0; tau < M; tau++) leaf[tau] = predict(&T[tau], (uint32_t)i, f, (uint32_t)pi[i]);
        for (int k = 0; k < K; k++) {
          for (int64_t tau = 0; tau < M; tau++) vals[tau] = leaf_value(&T[tau], leaf[tau], k);
          perm[k] = exact_sum(vals, M, 1) / (double)M;
        }
        L[i] = forest_loss(P, kind, K, base + i * K, perm);
      }
      imp[f] = exact_sum(L, N, 1) / (double)N;
    }
    free(pi);
    free(vals);
    free(base);
    free(perm);
    free(L);
    free(leaf);
  }
  for (int64_t tau = 0; tau < built; tau++) tree_free(&T[tau]);
  free(T);
  free(col);
  return rc;
}
