/*
 * Oracle Boruta loop (Alg. 1).  TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * Per iteration t = 1, 2, ...:
 *   X_cur = columns with state >= 0 (undecided and accepted), in order;
 *   X_sha = shuffled copies of X_cur, doubled until >= 5 columns;
 *   fit a forest on [X_cur || X_sha]; per-tree importance rows (Alg. 2 or
 *   the OOB form of Alg. 3), or one row for the whole forest (Alg. 3 as
 *   printed, permut_form = 1: that row is the hit statistic s);
 *   hit statistic per augmented column over the trees (FP64):
 *       mean_j = (sum_tau imp[tau][j]) / M
 *       sd_j   = sqrt(sum_tau (imp[tau][j] - mean_j)^2 / (M - 1))   (0 if M = 1)
 *       Z_j    = mean_j / (sd_j / sqrt(M)); if sd_j = 0: 0 when mean_j = 0, else +inf
 *     s_j = Z_j (Kursa's statistic) or mean_j (the paper's Imp);
 *   hit += 1[s_j > max over shadow columns of s]  (strict, Alg. 1);
 *   test(state, hit, t): for each undecided feature, with m = number of
 *   undecided features before the test,
 *       P_acc = P(Bin(t, 1/2) >= hit), P_rej = P(Bin(t, 1/2) <= hit),
 *       accept if P_acc < alpha/m, else reject if P_rej < alpha/m (Bonferroni).
 * The loop ends when no feature is undecided or t = max_iter.
 * All sums over trees are exact and rounded once.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "exact.h"

/* test(state, hit, t) of Alg. 1: two one-sided binomial tests at 1/2 with
 * Bonferroni's correction over the m features undecided before the test
 * (m is fixed before any feature of this test is decided); accept is tried
 * before reject; both comparisons are strict. */
void orc_decide(int t, double alpha, int64_t p, const int32_t* hits, int8_t* state) {
  int64_t m = 0;
  for (int64_t j = 0; j < p; j++) m += state[j] == 0;
  if (m == 0) return;
  double thr = alpha / (double)m;
  for (int64_t j = 0; j < p; j++) {
    if (state[j] != 0) continue;
    unsigned __int128 up, lo;
    binom_tails(t, hits[j], &up, &lo);
    double p_acc = ldexp(u128_to_double(up), -t);
    double p_rej = ldexp(u128_to_double(lo), -t);
    if (p_acc < thr)
      state[j] = 1;
    else if (p_rej < thr)
      state[j] = -1;
  }
}

int orc_iteration(const orc_problem* P, int t, int8_t* state, int32_t* hits, double* hist_row,
                  double* shadow_max, double* imp_out, double* s_out, int64_t* p_aug_out) {
  int64_t p = P->p, M = P->n_trees;
  int32_t* live = (int32_t*)malloc(sizeof(int32_t) * (size_t)p);
  int64_t p_live = 0;
  for (int64_t j = 0; j < p; j++)
    if (state[j] >= 0) live[p_live++] = (int32_t)j;
  int64_t n_sha = orc_shadow_count(p_live);
  int64_t p_aug = p_live + n_sha;
  if (p_aug_out) *p_aug_out = p_aug;
  uint8_t* Xsha = (uint8_t*)malloc((size_t)(n_sha * P->N + 1));
  orc_shadow(P, t, live, p_live, Xsha);

  int permut = (P->task & ORC_PERMUT) != 0;
  int forest = permut && P->permut_form == 1; /* Alg. 3 as printed: one importance row */
  double* imp = (double*)malloc(sizeof(double) * (size_t)(M * p_aug));
  int rc = 0;
  if (forest) {
    rc = orc_forest_permut(P, t, live, p_live, Xsha, imp);
    M = 1; /* the statistic is that row itself */
  } else {
    for (int64_t tau = 0; tau < M && rc == 0; tau++) {
      double* row = imp + tau * p_aug;
      rc = orc_tree(P, t, live, p_live, Xsha, (int)tau, NULL, 0, NULL, permut ? NULL : row,
                    permut ? row : NULL);
    }
  }
  free(Xsha);
  if (rc) {
    free(imp);
    free(live);
    return rc;
  }

  double* s = (double*)malloc(sizeof(double) * (size_t)p_aug);
  double* sq = (double*)malloc(sizeof(double) * (size_t)M);
  for (int64_t j = 0; j < p_aug; j++) {
    double mean = exact_sum(imp + j, M, p_aug) / (double)M;
    double sd = 0.0;
    if (M > 1) {
      for (int64_t tau = 0; tau < M; tau++) {
        double dlt = imp[tau * p_aug + j] - mean;
        sq[tau] = dlt * dlt;
      }
      sd = sqrt(exact_sum(sq, M, 1) / (double)(M - 1));
    }
    double z;
    if (sd == 0.0)
      z = (mean == 0.0) ? 0.0 : INFINITY;
    else
      z = mean / (sd / sqrt((double)M));
    s[j] = (P->stat == 1 || forest) ? mean : z;
  }
  free(sq);

  double smax = -INFINITY;
  for (int64_t c = p_live; c < p_aug; c++)
    if (s[c] > smax) smax = s[c];
  *shadow_max = smax;
  for (int64_t j = 0; j < p; j++) hist_row[j] = NAN;
  for (int64_t a = 0; a < p_live; a++) {
    int32_t j = live[a];
    hist_row[j] = s[a];
    if (s[a] > smax) hits[j] += 1;
  }

  orc_decide(t, P->alpha, p, hits, state);

  if (imp_out) memcpy(imp_out, imp, sizeof(double) * (size_t)(M * p_aug));
  if (s_out) memcpy(s_out, s, sizeof(double) * (size_t)p_aug);
  free(s);
  free(imp);
  free(live);
  return 0;
}

static int validate(const orc_problem* P) {
  if (P->N < 1 || P->p < 1 || P->ld < P->N) return -1;
  if (P->n_trees < 1 || P->max_depth < 0 || P->max_depth > ORC_MAX_DEPTH) return -1;
  if (P->n_bins < 2 || P->n_bins > 256 || P->max_iter < 1 || P->max_iter > 126) return -1;
  if (!(P->alpha > 0.0)) return -1;
  if ((P->task & 1) == ORC_CLASSIFICATION) {
    if (P->n_classes < 1 || P->n_classes > ORC_MAX_CLASSES || !P->ycls) return -1;
    for (int64_t i = 0; i < P->N; i++)
      if (P->ycls[i] >= P->n_classes) return -1;
  } else {
    if (!P->yreg) return -1;
    /* |sum of w*y| must stay below 2^62 for any node */
    uint64_t mx = 0;
    for (int64_t i = 0; i < P->N; i++) {
      int64_t v = P->yreg[i];
      uint64_t a = v < 0 ? (uint64_t)0 - (uint64_t)v : (uint64_t)v;
      if (a > mx) mx = a;
    }
    if (mx && (unsigned __int128)mx * (uint64_t)P->N >= ((unsigned __int128)1 << 62)) return -2;
  }
  for (int64_t j = 0; j < P->p; j++)
    for (int64_t i = 0; i < P->N; i++)
      if (P->X[j * P->ld + i] >= P->n_bins) return -1;
  return 0;
}

int orc_boruta(const orc_problem* P, int8_t* decision, int32_t* hits, double* imp_history,
               double* shadow_max, int32_t* iterations) {
  int rc = validate(P);
  if (rc) return rc;
  int64_t p = P->p;
  for (int64_t j = 0; j < p; j++) {
    decision[j] = 0;
    hits[j] = 0;
  }
  for (int64_t k = 0; k < (int64_t)P->max_iter * p; k++) imp_history[k] = NAN;
  for (int k = 0; k < P->max_iter; k++) shadow_max[k] = NAN;
  int t = 0;
  while (t < P->max_iter) {
    int64_t undecided = 0;
    for (int64_t j = 0; j < p; j++) undecided += decision[j] == 0;
    if (undecided == 0) break;
    t += 1;
    rc = orc_iteration(P, t, decision, hits, imp_history + (int64_t)(t - 1) * p,
                       shadow_max + (t - 1), NULL, NULL, NULL);
    if (rc) return rc;
  }
  *iterations = t;
  return 0;
}

/* ---------------- after the loop ---------------- */

static int cmp_double(const void* a, const void* b) {
  double x = *(const double*)a, y = *(const double*)b;
  return (x > y) - (x < y);
}

/* median of the non-NaN values among x[0], x[stride], ...; NaN if none
 * (mean of the two middle values for an even count) */
static double median_of(const double* x, int64_t n, int64_t stride, double* buf) {
  int64_t m = 0;
  for (int64_t k = 0; k < n; k++)
    if (!isnan(x[k * stride])) buf[m++] = x[k * stride];
  if (m == 0) return NAN;
  qsort(buf, (size_t)m, sizeof(double), cmp_double);
  return (m & 1) ? buf[m / 2] : (buf[m / 2 - 1] + buf[m / 2]) / 2.0;
}

void orc_rank(int64_t p, int32_t iterations, const int8_t* decision, const double* imp_history,
              int32_t* rank) {
  double* buf = (double*)malloc(sizeof(double) * (size_t)(iterations + 1));
  double* med = (double*)malloc(sizeof(double) * (size_t)p);
  int64_t* rej = (int64_t*)malloc(sizeof(int64_t) * (size_t)p);
  int64_t nr = 0;
  for (int64_t j = 0; j < p; j++) {
    rank[j] = decision[j] == 1 ? 1 : 2;
    if (decision[j] == -1) {
      med[j] = median_of(imp_history + j, iterations, p, buf);
      rej[nr++] = j;
    }
  }
  /* rejected: 3, 4, ... by descending median (a NaN median last), ties to the lower index;
   * a plain insertion sort of the rejected columns */
  for (int64_t a = 1; a < nr; a++) {
    int64_t j = rej[a], b = a;
    while (b > 0) {
      int64_t i = rej[b - 1];
      int before = isnan(med[i]) ? 0 : (isnan(med[j]) ? 1 : (med[i] > med[j] || (med[i] == med[j] && i < j)));
      if (before) break;
      rej[b] = rej[b - 1];
      b--;
    }
    rej[b] = j;
  }
  for (int64_t a = 0; a < nr; a++) rank[rej[a]] = (int32_t)(3 + a);
  free(buf);
  free(med);
  free(rej);
}

void orc_select_median(int n_runs, int64_t p, int32_t max_iter, const int32_t* iterations,
                       const double* imp_history, const double* shadow_max, double* med_imp,
                       double* med_shadow, int8_t* selected) {
  if (n_runs < 1 || max_iter < 1) return;
  double* buf = (double*)malloc(sizeof(double) * (size_t)(max_iter + n_runs + 1));
  double* per_run = (double*)malloc(sizeof(double) * (size_t)n_runs);
  for (int64_t j = 0; j < p; j++) {
    for (int r = 0; r < n_runs; r++)
      per_run[r] = median_of(imp_history + (int64_t)r * max_iter * p + j, iterations[r], p, buf);
    med_imp[j] = median_of(per_run, n_runs, 1, buf);
  }
  for (int r = 0; r < n_runs; r++)
    per_run[r] = median_of(shadow_max + (int64_t)r * max_iter, iterations[r], 1, buf);
  *med_shadow = median_of(per_run, n_runs, 1, buf);
  for (int64_t j = 0; j < p; j++) selected[j] = med_imp[j] > *med_shadow;
  free(buf);
  free(per_run);
}
