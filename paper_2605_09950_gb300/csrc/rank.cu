// After the Boruta loop: Alg. 1's final ranking, the median selection over
// runs with different seeds (the paper's synthetic study), and the batched
// driver that runs those seeds as independent jobs on the GPU.
//
// Ranking (Alg. 1's rankdata line is garbled; the reading taken): accepted
// features rank 1, tentative ones 2, rejected ones 3, 4, ... in descending
// order of the median of their history (the iterations they were in play),
// equal medians to the lower column index.
//
// Median selection (the paper ran 20 seeds and selected on the median
// importance; the reading taken): per run, the median of each feature's
// history and the median of the run's shadow maxima; over runs, the median
// of each; a feature is selected when its median is strictly above the
// shadows' median.  Medians skip NaN entries (iterations a feature was out
// of play) and take the mean of the two middle values of an even count.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <vector>

#include "boruta.h"

int boruta_record_error(int code, const char* msg);  // api.cu: records the message

namespace {

// median of the non-NaN values x[0], x[stride], ..., x[(n-1)*stride]; NaN if none
double median_skip_nan(const double* x, int64_t n, int64_t stride, std::vector<double>& buf) {
  buf.clear();
  for (int64_t k = 0; k < n; ++k) {
    const double v = x[k * stride];
    if (!std::isnan(v)) buf.push_back(v);
  }
  if (buf.empty()) return std::nan("");
  std::sort(buf.begin(), buf.end());
  const size_t m = buf.size();
  return (m % 2) ? buf[m / 2] : (buf[m / 2 - 1] + buf[m / 2]) / 2.0;
}

}  // namespace

extern "C" int boruta_rank(const int8_t* decision, const double* imp_history, int64_t p, int32_t iterations,
                           int32_t* rank) {
  if (p < 0 || iterations < 0 || (p > 0 && (!decision || !rank || (iterations > 0 && !imp_history))))
    return boruta_record_error(BORUTA_EINVAL, "boruta_rank: bad arguments");
  std::vector<double> buf, med(static_cast<size_t>(p), 0.0);
  std::vector<int64_t> rejected;
  for (int64_t j = 0; j < p; ++j) {
    if (decision[j] < -1 || decision[j] > 1)
      return boruta_record_error(BORUTA_EINVAL, "boruta_rank: decision values are -1, 0, 1");
    rank[j] = decision[j] == 1 ? 1 : 2;
    if (decision[j] == -1) {
      med[j] = median_skip_nan(imp_history + j, iterations, p, buf);
      rejected.push_back(j);
    }
  }
  // descending median, a NaN median last; stable on the ascending column order
  std::stable_sort(rejected.begin(), rejected.end(), [&](int64_t a, int64_t b) {
    if (std::isnan(med[a])) return false;
    if (std::isnan(med[b])) return true;
    return med[a] > med[b];
  });
  for (size_t r = 0; r < rejected.size(); ++r) rank[rejected[r]] = static_cast<int32_t>(3 + r);
  return BORUTA_OK;
}

extern "C" int boruta_select_median(int n_runs, int64_t p, int32_t max_iter, const int32_t* iterations,
                                    const double* imp_history, const double* shadow_max, double* median_imp,
                                    double* median_shadow, int8_t* selected) {
  if (n_runs < 1 || p < 0 || max_iter < 1 || !iterations || !imp_history || !shadow_max || !median_shadow ||
      (p > 0 && (!median_imp || !selected)))
    return boruta_record_error(BORUTA_EINVAL, "boruta_select_median: bad arguments");
  for (int r = 0; r < n_runs; ++r)
    if (iterations[r] < 0 || iterations[r] > max_iter)
      return boruta_record_error(BORUTA_EINVAL, "boruta_select_median: a run's iterations exceed max_iter");
  std::vector<double> buf, per_run(static_cast<size_t>(n_runs));
  for (int r = 0; r < n_runs; ++r)
    per_run[r] = median_skip_nan(shadow_max + static_cast<int64_t>(r) * max_iter, iterations[r], 1, buf);
  *median_shadow = median_skip_nan(per_run.data(), n_runs, 1, buf);
  for (int64_t j = 0; j < p; ++j) {
    for (int r = 0; r < n_runs; ++r)
      per_run[r] = median_skip_nan(imp_history + static_cast<int64_t>(r) * max_iter * p + j, iterations[r], p, buf);
    median_imp[j] = median_skip_nan(per_run.data(), n_runs, 1, buf);
    selected[j] = median_imp[j] > *median_shadow ? 1 : 0;
  }
  return BORUTA_OK;
}

extern "C" int boruta_fit_seeds(const uint8_t* X, int64_t ld, const void* y, int64_t N, int64_t p, int task,
                                int n_trees, int max_depth, int mtry, int n_bins, int max_iter, double alpha,
                                int n_seeds, const uint64_t* seeds, const boruta_opts* opts, boruta_result* outs,
                                double* median_imp, double* median_shadow, int8_t* selected) {
  if (n_seeds < 1 || !seeds || !outs || !median_shadow || (p > 0 && (!median_imp || !selected)))
    return boruta_record_error(BORUTA_EINVAL, "boruta_fit_seeds: bad arguments");
  if (max_iter < 1 || p < 1) return boruta_record_error(BORUTA_EINVAL, "boruta_fit_seeds: bad sizes");
  std::vector<boruta_job> jobs(static_cast<size_t>(n_seeds));
  for (int r = 0; r < n_seeds; ++r)
    jobs[r] = boruta_job{X, ld, y, N, p, task, n_trees, max_depth, mtry, n_bins, max_iter, alpha, seeds[r],
                         opts ? opts->n_classes : 0};
  int rc = boruta_fit_batch(n_seeds, jobs.data(), opts, outs);
  if (rc) return rc;
  // the runs' histories, contiguous
  std::vector<double> hist(static_cast<size_t>(n_seeds) * max_iter * p), smax(static_cast<size_t>(n_seeds) * max_iter);
  std::vector<int32_t> its(static_cast<size_t>(n_seeds));
  for (int r = 0; r < n_seeds; ++r) {
    std::copy(outs[r].imp_history, outs[r].imp_history + static_cast<int64_t>(max_iter) * p,
              hist.begin() + static_cast<int64_t>(r) * max_iter * p);
    std::copy(outs[r].shadow_max, outs[r].shadow_max + max_iter, smax.begin() + static_cast<int64_t>(r) * max_iter);
    its[r] = outs[r].iterations;
  }
  return boruta_select_median(n_seeds, p, max_iter, its.data(), hist.data(), smax.data(), median_imp, median_shadow,
                              selected);
}
