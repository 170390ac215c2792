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
