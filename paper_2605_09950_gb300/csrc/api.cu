// C ABI of the GPU Boruta library: argument checks, device workspace, the
// per-iteration launch sequence (Alg. 1 loop body) and result transfer.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

#include "boruta.h"
#include "engine.cuh"

using namespace bgb;

namespace {

thread_local std::string g_error;

int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_error = buf;
  return code;
}

#define CK(call)                                                                          \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess) return fail(BORUTA_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

int64_t shadow_count(int64_t p_live) {
  int64_t n = p_live;
  if (n <= 0) return 0;
  while (n < 5) n *= 2;
  return n;
}

int64_t isqrt(int64_t v) {
  int64_t r = static_cast<int64_t>(std::sqrt(static_cast<double>(v)));
  while (r * r > v) --r;
  while ((r + 1) * (r + 1) <= v) ++r;
  return r;
}

}  // namespace

// error reporting for noalloc.cu (same thread-local message as every entry point)
int boruta_noalloc_fail(int code, const char* msg) { return fail(code, "%s", msg); }
int boruta_record_error(int code, const char* msg) { return fail(code, "%s", msg); }

struct boruta_session {
  Dev d{};
  cudaStream_t st = nullptr;
  int64_t p = 0, N = 0;
  int task = 0, mtry_opt = 0, max_iter = 0, t = 0, split_path = 0, chunk_nodes = 0;
  // histogram tile shape: column bytes per feature band and row x feature
  // work per group; opts.autotune times the candidates on the first step
  int64_t band_bytes = kBandBytes;
  // histogram launches: 0 = per feature band at the levels where a band
  // holds at least twice as many groups as the GPU runs warps at once (else
  // per chunk), 1 = per band, 2 = per chunk (opts.band_launch)
  int band_policy = 0;
  // per tree level (empty: band_bytes and band_policy at every level)
  std::vector<int64_t> lvl_bb;
  std::vector<int32_t> lvl_bl;
  std::vector<int32_t> used_bw, used_bl;  // band width (columns) and launch mode of each level, last iteration
  bool autotune = false, tuned = false;
  std::vector<uint32_t> tune_gw;
  std::vector<int64_t> tune_bb;  // -1: the per-level combination
  std::vector<int32_t> tune_bl;
  std::vector<double> tune_ms;
  std::vector<std::vector<double>> tune_lvl_ms;  // per candidate: split-stage ms of each level
  int tune_chosen = -1;
  int pending_t = 0;  // iteration enqueued and not yet finished
  bool graph = false;                   // iterations replayed through an instantiated CUDA graph
  cudaStream_t gst = nullptr;           // capture stream of the graph
  cudaGraphExec_t gexec = nullptr;      // the graph of the last iteration, updated in place
  int graph_builds = 0, graph_updates = 0;
  bool own_stream = false;
  unsigned long long* counters_h = nullptr;  // pinned copy of the device counters
  bool finished = false;
  std::vector<void*> dev_allocs;
  std::vector<int8_t> state_h;
  // pinned staging
  uint32_t* status_h = nullptr;
  int8_t* state_pin = nullptr;
  int32_t* live_pin = nullptr;
  // device per-iteration arrays
  int32_t* live_d = nullptr;
  uint8_t* X_owned = nullptr;
  void* y_owned = nullptr;
  // launch geometry
  int sms = 0, split_grid = 0, small_grid = 0, tree_grid = 0, permut_grid = 0, walk_grid = 0;
  size_t split_smem = 0;
  // second stream for the small-node kernel, and its fork/join events
  cudaStream_t st2 = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr;
  // split-kernel timing of the last step
  std::vector<cudaEvent_t> ev;
  double split_ms = 0.0;
  std::vector<double> level_ms, level_hist_ms;
  int split_launches = 0;
  int64_t iter_kernels = 0;   // kernels the last enqueued iteration launched
  int64_t total_kernels = 0;  // kernels launched since the session was created
  double split_bytes = 0.0;
  std::vector<cudaEvent_t> hev;  // around the histogram kernel of each level
  double hist_ms = 0.0, hist_bytes = 0.0;
  cudaEvent_t iev[2] = {nullptr, nullptr};  // around the importance stage (Alg. 2 or 3)
  double imp_ms = 0.0, imp_visits = 0.0;

  template <typename T>
  int alloc(T** p, size_t count) {
    void* q = nullptr;
    if (count == 0) count = 1;
    cudaError_t e = cudaMalloc(&q, count * sizeof(T));
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(BORUTA_ENOMEM, "device allocation of %zu bytes failed: %s", count * sizeof(T),
                  cudaGetErrorString(e));
    }
    dev_allocs.push_back(q);
    *p = static_cast<T*>(q);
    return 0;
  }

  ~boruta_session() {
    if (st) cudaStreamSynchronize(st);
    for (void* q : dev_allocs) cudaFree(q);
    for (cudaEvent_t e : ev) cudaEventDestroy(e);
    for (cudaEvent_t e : hev) cudaEventDestroy(e);
    for (cudaEvent_t e : iev)
      if (e) cudaEventDestroy(e);
    if (st2) {
      cudaStreamSynchronize(st2);
      cudaStreamDestroy(st2);
    }
    if (gexec) cudaGraphExecDestroy(gexec);
    if (gst) cudaStreamDestroy(gst);
    if (fork) cudaEventDestroy(fork);
    if (join) cudaEventDestroy(join);
    if (status_h) cudaFreeHost(status_h);
    if (counters_h) cudaFreeHost(counters_h);
    if (own_stream && st) cudaStreamDestroy(st);
    if (state_pin) cudaFreeHost(state_pin);
    if (live_pin) cudaFreeHost(live_pin);
  }
};

static int check_args(const uint8_t* X, int64_t ld, const void* y, int64_t N, int64_t p, int task,
                      int n_trees, int max_depth, int mtry, int n_bins, int max_iter, double alpha,
                      const boruta_opts* o) {
  if (!X || !y) return fail(BORUTA_EINVAL, "X and y must not be NULL");
  if (N < 1 || N >= (1 << 24)) return fail(BORUTA_EINVAL, "N = %lld outside [1, 2^24)", (long long)N);
  if (p < 1 || p >= (1 << 23)) return fail(BORUTA_EINVAL, "p = %lld outside [1, 2^23)", (long long)p);
  if (ld < N) return fail(BORUTA_EINVAL, "ld = %lld < N", (long long)ld);
  if (task < 0 || task > 3) return fail(BORUTA_EINVAL, "task = %d is not kind | importance", task);
  if (n_trees < 1 || n_trees >= (1 << 20)) return fail(BORUTA_EINVAL, "n_trees = %d", n_trees);
  if (max_depth < 0 || max_depth > kMaxDepth) return fail(BORUTA_EINVAL, "max_depth = %d", max_depth);
  if (n_bins < 2 || n_bins > 256) return fail(BORUTA_EINVAL, "n_bins = %d outside [2, 256]", n_bins);
  if (max_iter < 1 || max_iter > kMaxIterations)
    return fail(BORUTA_EINVAL, "max_iter = %d outside [1, %d]", max_iter, kMaxIterations);
  if (!(alpha > 0.0)) return fail(BORUTA_EINVAL, "alpha must be positive");
  if (mtry < 0) return fail(BORUTA_EINVAL, "mtry = %d", mtry);
  if (o->n_classes < 0 || o->n_classes > kMaxClasses)
    return fail(BORUTA_EINVAL, "n_classes = %d outside [0, 8]", o->n_classes);
  if (o->split_path < 0 || o->split_path > 1) return fail(BORUTA_EINVAL, "opts: split_path takes 0 or 1");
  if (o->chunk_nodes < 0) return fail(BORUTA_EINVAL, "opts: chunk_nodes must not be negative");
  if (o->permut_form < 0 || o->permut_form > 1) return fail(BORUTA_EINVAL, "opts: permut_form takes 0 or 1");
  if (o->forest_rows < 0) return fail(BORUTA_EINVAL, "opts: forest_rows must not be negative");
  if (o->autotune < 0 || o->autotune > 1) return fail(BORUTA_EINVAL, "opts: autotune takes 0 or 1");
  if (o->band_launch < 0 || o->band_launch > 2) return fail(BORUTA_EINVAL, "opts: band_launch takes 0, 1 or 2");
  if (o->permut_form == 1 && !(task & BORUTA_PERMUT))
    return fail(BORUTA_EINVAL, "opts: permut_form = 1 is a form of Alg. 3 (task needs BORUTA_PERMUT)");
  if (o->precision < 0 || o->precision > 1 || o->tie_break < 0 || o->tie_break > 1 || o->stat < 0 ||
      o->stat > 1)
    return fail(BORUTA_EINVAL, "opts: precision, tie_break and stat take 0 or 1");
  if (!(o->kl_eps > 0.0)) return fail(BORUTA_EINVAL, "kl_eps must be positive");
  return 0;
}

extern "C" {

void boruta_default_opts(boruta_opts* o) {
  std::memset(o, 0, sizeof *o);
  o->kl_eps = 1e-7;
}

const char* boruta_last_error(void) { return g_error.c_str(); }

static int session_init(boruta_session* s, const uint8_t* X, int64_t ld, const void* y, int64_t N,
                        int64_t p, int task, int n_trees, int max_depth, int mtry, int n_bins,
                        int max_iter, double alpha, uint64_t seed, const boruta_opts* o) {
  int rc;
  s->st = static_cast<cudaStream_t>(o->stream);
  s->p = p;
  s->N = N;
  s->task = task;
  s->mtry_opt = mtry;
  s->split_path = o->split_path;
  s->chunk_nodes = o->chunk_nodes;
  s->autotune = o->autotune != 0;
  s->graph = o->graph != 0;
  s->max_iter = max_iter;
  Dev& d = s->d;
  const bool reg = (task & 1) != 0;
  d.kind = reg ? 1 : 0;
  d.permut = (task & BORUTA_PERMUT) ? 1 : 0;
  d.N = static_cast<int32_t>(N);
  d.ldN = static_cast<int32_t>((N + 15) / 16 * 16);
  d.p = static_cast<int32_t>(p);
  d.B = n_bins;
  d.D = max_depth;
  d.M = n_trees;
  d.max_iter = max_iter;
  d.precision = o->precision;
  d.group_work = kGroupWork;
  s->band_policy = o->band_launch;
  d.band_launch = 0;
  d.permut_form = d.permut ? o->permut_form : 0;
  d.tie_break = o->tie_break;
  d.stat = o->stat;
  d.seed = seed;
  d.job = o->job;
  d.kl_eps = o->kl_eps;
  d.alpha = alpha;

  const size_t ybytes = reg ? sizeof(int64_t) : sizeof(uint8_t);
  if (o->host_inputs) {
    if ((rc = s->alloc(&s->X_owned, static_cast<size_t>(ld) * p))) return rc;
    CK(cudaMemcpyAsync(s->X_owned, X, static_cast<size_t>(ld) * p, cudaMemcpyHostToDevice, s->st));
    uint8_t* yb = nullptr;
    if ((rc = s->alloc(&yb, ybytes * N))) return rc;
    CK(cudaMemcpyAsync(yb, y, ybytes * N, cudaMemcpyHostToDevice, s->st));
    s->y_owned = yb;
    d.X = s->X_owned;
    y = yb;
  } else {
    d.X = X;
  }
  d.ld = ld;
  d.ycls = reg ? nullptr : static_cast<const uint8_t*>(y);
  d.yreg = reg ? static_cast<const int64_t*>(y) : nullptr;

  const int64_t p_aug_max = p + shadow_count(p);
  const int64_t n_sha_max = shadow_count(p);
  // node pool: per tree at most min(2^l, N) nodes at depth l
  uint64_t per_tree = 0;
  for (int l = 0; l <= max_depth; ++l) per_tree += std::min<uint64_t>(1ull << l, static_cast<uint64_t>(N));
  uint64_t cap = per_tree * static_cast<uint64_t>(n_trees);
  if (cap > 0xFFFFFFF0ull) cap = 0xFFFFFFF0ull;
  d.cap = static_cast<uint32_t>(cap);
  const int Cmax = kMaxClasses;

  if ((rc = s->alloc(&s->live_d, p))) return rc;
  d.live = s->live_d;
  (void)n_sha_max;
  if ((rc = s->alloc(&d.Xaug, static_cast<size_t>(p_aug_max) * d.ldN))) return rc;
  const size_t MN = static_cast<size_t>(n_trees) * N;
  if ((rc = s->alloc(&d.bootcnt, MN))) return rc;
  if ((rc = s->alloc(&d.rows[0], MN))) return rc;
  if ((rc = s->alloc(&d.rows[1], MN))) return rc;
  if ((rc = s->alloc(&d.oob, MN))) return rc;
  if ((rc = s->alloc(&d.oob_cnt, n_trees))) return rc;
  if (d.permut && (rc = s->alloc(&d.piv, static_cast<size_t>(N)))) return rc;
  // the row-major copy of Xaug: the small-node split reads a row's sampled
  // columns from it, and the Alg. 3 walks a row's path
  if ((rc = s->alloc(&d.Xrow, static_cast<size_t>(N) * ((p_aug_max + 15) / 16 * 16)))) return rc;
  const size_t P = cap;
  if ((rc = s->alloc(&d.nd_tree, P))) return rc;
  if ((rc = s->alloc(&d.nd_heap, P))) return rc;
  if ((rc = s->alloc(&d.nd_seg, P))) return rc;
  if ((rc = s->alloc(&d.nd_len, P))) return rc;
  if ((rc = s->alloc(&d.nd_n, P))) return rc;
  if ((rc = s->alloc(&d.nd_split, P))) return rc;
  if ((rc = s->alloc(&d.nd_child, P))) return rc;
  if (d.permut && (rc = s->alloc(&d.nd_sc, P))) return rc;
  if ((rc = s->alloc(&d.nd_delta, P))) return rc;
  if ((rc = s->alloc(&d.nd_lrows, P))) return rc;
  if ((rc = s->alloc(&d.nd_ln, P))) return rc;
  if (reg) {
    if ((rc = s->alloc(&d.nd_S, P))) return rc;
    if ((rc = s->alloc(&d.nd_lS, P))) return rc;
  }
  if ((rc = s->alloc(&d.lvl_off, max_depth + 2))) return rc;
  if ((rc = s->alloc(&d.lvl_cnt, max_depth + 2))) return rc;
  if ((rc = s->alloc(&d.work, max_depth + 2))) return rc;
  if ((rc = s->alloc(&d.chunk, kScanBlocks))) return rc;
  if ((rc = s->alloc(&d.acc, static_cast<size_t>(n_trees) * p_aug_max * kCsaLimbs))) return rc;
  if ((rc = s->alloc(&d.imp, static_cast<size_t>(n_trees) * p_aug_max))) return rc;
  if ((rc = s->alloc(&d.s, p_aug_max))) return rc;
  if ((rc = s->alloc(&d.state, p))) return rc;
  if ((rc = s->alloc(&d.hits, p))) return rc;
  if ((rc = s->alloc(&d.hist, static_cast<size_t>(max_iter) * p))) return rc;
  if ((rc = s->alloc(&d.smax, max_iter))) return rc;
  if ((rc = s->alloc(&d.status, 4))) return rc;
  if ((rc = s->alloc(&d.counters, 4))) return rc;
  u128* pascal = nullptr;
  if ((rc = s->alloc(&pascal, 127 * 127))) return rc;
  d.pascal = pascal;

  CK(cudaHostAlloc(&s->status_h, 4 * sizeof(uint32_t), cudaHostAllocDefault));
  CK(cudaHostAlloc(reinterpret_cast<void**>(&s->counters_h), 4 * sizeof(unsigned long long), cudaHostAllocDefault));
  CK(cudaHostAlloc(&s->state_pin, p, cudaHostAllocDefault));
  CK(cudaHostAlloc(&s->live_pin, p * sizeof(int32_t), cudaHostAllocDefault));

  // binomial coefficients C(t, k), t, k <= 126, by Pascal's rule (exact)
  std::vector<u128> tri(127 * 127, 0);
  tri[0] = 1;
  for (int t = 1; t <= 126; ++t) {
    tri[t * 127] = 1;
    for (int k = 1; k <= t; ++k) tri[t * 127 + k] = tri[(t - 1) * 127 + k - 1] + tri[(t - 1) * 127 + k];
  }
  CK(cudaMemcpyAsync(pascal, tri.data(), tri.size() * sizeof(u128), cudaMemcpyHostToDevice, s->st));

  // state: all undecided, history NaN
  CK(cudaMemsetAsync(d.state, 0, p, s->st));
  CK(cudaMemsetAsync(d.hits, 0, p * sizeof(int32_t), s->st));
  std::vector<double> nan_hist(static_cast<size_t>(max_iter) * p, std::nan(""));
  CK(cudaMemcpyAsync(d.hist, nan_hist.data(), nan_hist.size() * sizeof(double), cudaMemcpyHostToDevice, s->st));
  CK(cudaMemcpyAsync(d.smax, nan_hist.data(), max_iter * sizeof(double), cudaMemcpyHostToDevice, s->st));
  CK(cudaMemsetAsync(d.status, 0, 4 * sizeof(uint32_t), s->st));
  CK(cudaMemsetAsync(d.counters, 0, 4 * sizeof(unsigned long long), s->st));

  // input validation on the device
  d.C = 1;
  launch_validate(d, s->st);
  CK(cudaGetLastError());
  unsigned long long maxy = 0;
  CK(cudaMemcpyAsync(s->status_h, d.status, 4 * sizeof(uint32_t), cudaMemcpyDeviceToHost, s->st));
  CK(cudaMemcpyAsync(&maxy, d.counters + 1, sizeof maxy, cudaMemcpyDeviceToHost, s->st));
  CK(cudaStreamSynchronize(s->st));
  if (s->status_h[0] & kErrInput)
    return fail(BORUTA_EINVAL, "input has a bin >= n_bins (%d) or a label >= 8", n_bins);
  // Bins above the largest one present are empty in every node: a threshold
  // there sends every row left and is never valid, so the fit only needs
  // histograms up to the largest bin (same trees, smaller histograms and
  // scans; e.g. genotype columns declared with 256 bins use 3).
  d.B = std::max(2, std::min(n_bins, static_cast<int>(s->status_h[3]) + 1));
  if (reg) {
    d.C = 1;
    if (maxy && static_cast<double>(maxy) * static_cast<double>(N) >= 4611686018427387904.0)
      return fail(BORUTA_EOVERFLOW, "N * max|y| must stay below 2^62");
  } else {
    const int seen = static_cast<int>(s->status_h[2]) + 1;
    if (o->n_classes == 0) {
      d.C = seen;
    } else {
      if (seen > o->n_classes) return fail(BORUTA_EINVAL, "label %d >= n_classes %d", seen - 1, o->n_classes);
      d.C = o->n_classes;
    }
  }
  if (!reg) {
    if ((rc = s->alloc(&d.nd_cnt, P * d.C))) return rc;
    if ((rc = s->alloc(&d.nd_lcnt, P * d.C))) return rc;
  }
  // larger nodes of one level: at most N/33 per tree (each has > 32 rows)
  const size_t big_cap = static_cast<size_t>(n_trees) * (static_cast<size_t>(N) / 33 + 1);
  if ((rc = s->alloc(&d.big, big_cap))) return rc;
  uint8_t* ninfo = nullptr;
  if ((rc = s->alloc(&ninfo, big_cap * ninfo_bytes(split_variant(d.kind, d.C))))) return rc;
  d.ninfo = ninfo;
  // nodes of one level: at most min(2^D, N) per tree
  const size_t level_cap = std::min<size_t>(
      cap, static_cast<size_t>(n_trees) * std::min<uint64_t>(1ull << max_depth, static_cast<uint64_t>(N)));
  if ((rc = s->alloc(&d.small, level_cap))) return rc;
  if ((rc = s->alloc(&d.nsmall, max_depth + 2))) return rc;
  if ((rc = s->alloc(&d.ntiny, max_depth + 2))) return rc;
  if ((rc = s->alloc(&d.micro, level_cap))) return rc;
  if ((rc = s->alloc(&d.nmicro, max_depth + 2))) return rc;
  d.small_cap = static_cast<uint32_t>(level_cap);
  uint8_t* cand = nullptr;
  if ((rc = s->alloc(&cand, big_cap * kItemsPerNode * cand_bytes(split_variant(d.kind, d.C))))) return rc;
  d.cand = cand;
  // feature-band plan buffers: one item per (larger node, draw slot)
  {
    const int64_t mtry_max = mtry > 0 ? std::min<int64_t>(mtry, p_aug_max)
                                      : std::max<int64_t>(1, reg ? p_aug_max / 3 : isqrt(p_aug_max));
    uint64_t cap_items = static_cast<uint64_t>(big_cap) * static_cast<uint64_t>(mtry_max);
    if (cap_items > kMaxItems) cap_items = kMaxItems;
    d.item_cap = cap_items;
    if ((rc = s->alloc(&d.items_u, cap_items))) return rc;
    if ((rc = s->alloc(&d.items_s, cap_items))) return rc;
    if ((rc = s->alloc(&d.items_b, cap_items))) return rc;
    uint8_t* fb = nullptr;
    if ((rc = s->alloc(&fb, cap_items * packed_bytes(split_variant(d.kind, d.C))))) return rc;
    d.fbest = fb;
    if ((rc = s->alloc(&d.band_cnt, kMaxBands + 1))) return rc;
  }
  (void)Cmax;
  if (d.permut_form == 1) {
    // Alg. 3 as printed: per row the exact base sums; per block of rows the
    // exact (row, column) deltas, blocks sized to about 1 GiB
    const int64_t K = reg ? 1 : d.C;
    const int64_t per_row = p_aug_max * K * kCsaLimbs * static_cast<int64_t>(sizeof(long long));
    d.frows = static_cast<uint32_t>(std::max<int64_t>(1, std::min<int64_t>(N, (int64_t{1} << 30) / per_row)));
    if (o->forest_rows > 0) d.frows = std::min<uint32_t>(d.frows, static_cast<uint32_t>(o->forest_rows));
    if ((rc = s->alloc(&d.fbase, static_cast<size_t>(N) * K * kCsaLimbs))) return rc;
    if ((rc = s->alloc(&d.fbase_mean, static_cast<size_t>(N) * K))) return rc;
    if ((rc = s->alloc(&d.facc, static_cast<size_t>(d.frows) * p_aug_max * K * kCsaLimbs))) return rc;
    CK(cudaMemsetAsync(d.facc, 0, static_cast<size_t>(d.frows) * p_aug_max * K * kCsaLimbs * sizeof(long long),
                       s->st));
  }
  CK(cudaMemsetAsync(d.status, 0, 4 * sizeof(uint32_t), s->st));

  // launch geometry
  int dev = 0;
  CK(cudaGetDevice(&dev));
  CK(cudaDeviceGetAttribute(&s->sms, cudaDevAttrMultiProcessorCount, dev));
  s->split_smem = split_smem_bytes(d.kind, d.C, d.B);
  const void* kptr[4];
  int nk = 0;
  const int variant = split_variant(d.kind, d.C);
  split_kernel_ptrs(variant, kptr, &nk);
  // The limit is a property of the kernel, shared by every session in the
  // process: set it to what the variant can need at most (its largest class
  // count, 256 bins) so that no session lowers it below another's launches.
  const size_t smem_cap = std::max(s->split_smem, split_smem_bytes(d.kind, variant_classes(variant), 256));
  for (int i = 0; i < nk; ++i)
    CK(cudaFuncSetAttribute(kptr[i], cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem_cap)));
  int per_sm = 0;
  CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kptr[1], kSplitThreads, s->split_smem));
  if (per_sm < 1) return fail(BORUTA_EINVAL, "split kernel does not fit on an SM");
  s->split_grid = per_sm * s->sms;
  // warp-per-node kernels: as many blocks as the GPU holds at once (they
  // loop over their nodes), so no partial last wave
  int small_per_sm = 0;
  CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&small_per_sm, small_kernel_ptr(variant), 256, 0));
  s->small_grid = std::max(1, std::min(8, small_per_sm)) * s->sms;
  s->tree_grid = std::min(n_trees, 8 * s->sms);
  s->permut_grid = 16 * s->sms;
  int walk_per_sm = 0;
  CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&walk_per_sm, permut_kernel_ptr(d.precision), 128,
                                                   permut_smem_bytes(max_depth)));
  s->walk_grid = std::max(1, walk_per_sm) * s->sms;
  s->ev.resize(2 * (max_depth + 1));
  for (auto& e : s->ev) CK(cudaEventCreate(&e));
  s->hev.resize(2 * (max_depth + 1));
  for (auto& e : s->hev) CK(cudaEventCreate(&e));
  for (auto& e : s->iev) CK(cudaEventCreate(&e));
  CK(cudaStreamCreateWithFlags(&s->st2, cudaStreamNonBlocking));
  if (s->graph) CK(cudaStreamCreateWithFlags(&s->gst, cudaStreamNonBlocking));
  CK(cudaEventCreateWithFlags(&s->fork, cudaEventDisableTiming));
  CK(cudaEventCreateWithFlags(&s->join, cudaEventDisableTiming));
  s->state_h.assign(p, 0);
  return 0;
}

int boruta_session_create(const uint8_t* X, int64_t ld, const void* y, int64_t N, int64_t p, int task,
                          int n_trees, int max_depth, int mtry, int n_bins, int max_iter, double alpha,
                          uint64_t seed, const boruta_opts* opts, boruta_session** out) {
  if (!out) return fail(BORUTA_EINVAL, "out must not be NULL");
  *out = nullptr;
  boruta_opts o;
  if (opts)
    o = *opts;
  else
    boruta_default_opts(&o);
  int rc = check_args(X, ld, y, N, p, task, n_trees, max_depth, mtry, n_bins, max_iter, alpha, &o);
  if (rc) return rc;
  boruta_session* s = new boruta_session();
  rc = session_init(s, X, ld, y, N, p, task, n_trees, max_depth, mtry, n_bins, max_iter, alpha, seed, &o);
  if (rc) {
    std::string msg = g_error;
    delete s;
    g_error = msg;
    return rc;
  }
  *out = s;
  return 0;
}

// Enqueues iteration t on the session's stream (or records it, when the
// stream is being captured into a graph), with the copies of its status,
// state and counters into pinned host memory; does not wait.
static int enqueue_iteration(boruta_session* s, int t, cudaStream_t st) {
  Dev& d = s->d;
  const bool timed = !s->graph;
  // X_cur: undecided and accepted columns, in order
  int32_t p_live = 0;
  for (int64_t j = 0; j < s->p; ++j)
    if (s->state_h[j] >= 0) s->live_pin[p_live++] = static_cast<int32_t>(j);
  const int64_t n_sha = shadow_count(p_live);
  const int64_t p_aug = p_live + n_sha;
  d.t = t;
  d.p_live = p_live;
  d.n_sha = static_cast<int32_t>(n_sha);
  d.p_aug = static_cast<int32_t>(p_aug);
  int64_t m = s->mtry_opt > 0 ? std::min<int64_t>(s->mtry_opt, p_aug)
                              : (d.kind ? p_aug / 3 : isqrt(p_aug));
  d.mtry = static_cast<int32_t>(std::max<int64_t>(m, 1));
  d.ldP = static_cast<int32_t>((p_aug + 15) / 16 * 16);
  // feature bands: ~kBandBytes of columns each, at most kMaxBands; the packed
  // item holds a 14-bit slot and a 22-bit feature
  d.band_w = 0;
  d.nbands = 0;
  d.chunk0 = 0;
  d.chunk_cap = static_cast<uint32_t>(std::min<uint64_t>(d.item_cap / static_cast<uint64_t>(d.mtry), 1u << 26));
  if (s->chunk_nodes > 0) d.chunk_cap = std::min<uint32_t>(d.chunk_cap, static_cast<uint32_t>(s->chunk_nodes));
  const bool band_ok = s->split_path == 0 && d.chunk_cap > 0 && d.mtry < (1 << 14) && p_aug < (1 << 22);
  // the band width and launch mode of a level (big: its larger nodes, at
  // most; level -1: the iteration's defaults)
  auto set_band = [&](Dev& dl, int level, uint64_t big) {
    dl.band_w = 0;
    dl.nbands = 0;
    dl.band_launch = 0;
    if (!band_ok) return;
    const bool per_level = level >= 0 && level < static_cast<int>(s->lvl_bb.size());
    const int64_t bb = per_level ? s->lvl_bb[level] : s->band_bytes;
    int64_t w = std::max<int64_t>(1, bb / d.ldN);
    w = std::max<int64_t>(w, (p_aug + kMaxBands - 1) / kMaxBands);
    w = std::min<int64_t>(w, p_aug);  // one band at most holds every column
    dl.band_w = static_cast<int32_t>(w);
    dl.nbands = static_cast<int32_t>((p_aug + w - 1) / w);
    if (per_level) {
      dl.band_launch = s->lvl_bl[level];
    } else if (s->band_policy == 1) {
      dl.band_launch = 1;
    } else if (s->band_policy == 0 && level >= 0) {
      // All warps on one band at a time pays once a band's groups fill the
      // GPU twice over (with fewer, the launches of the bands run part-empty).
      // Over several chunks it multiplies the launches, each ending in a tail
      // as long as its longest group, so there it is kept to levels whose
      // groups are small (estimated rows per node x the node's items per
      // band, at most the group work): measured faster on the deep levels of
      // the N=1e6 multiclass workload (groups of ~60), slower on those of the
      // SNP workload (groups of thousands).
      const uint64_t groups_per_band = big * static_cast<uint64_t>(d.mtry) / static_cast<uint64_t>(dl.nbands);
      const uint64_t resident = static_cast<uint64_t>(s->split_grid) * (kSplitThreads / 32);
      const bool one_chunk = big <= static_cast<uint64_t>(d.chunk_cap);
      const uint64_t width = std::max<uint64_t>(1, big / static_cast<uint64_t>(d.M));  // nodes per tree, at most
      const uint64_t rows = static_cast<uint64_t>(d.N) * 632 / 1000 / width;          // in-bag rows per node, about
      const uint64_t per_band = std::max<uint64_t>(1, static_cast<uint64_t>(d.mtry) / static_cast<uint64_t>(dl.nbands));
      const uint64_t group = std::min<uint64_t>(rows * per_band, d.group_work);
      const bool small_groups = group * 8 <= d.group_work;
      dl.band_launch = (groups_per_band >= 2 * resident && (one_chunk || small_groups)) ? 1 : 0;
    }
  };
  set_band(d, -1, 0);

  CK(cudaMemcpyAsync(s->live_d, s->live_pin, p_live * sizeof(int32_t), cudaMemcpyHostToDevice, st));
  CK(cudaMemsetAsync(d.bootcnt, 0, static_cast<size_t>(d.M) * d.N * sizeof(uint32_t), st));
  CK(cudaMemsetAsync(d.acc, 0, static_cast<size_t>(d.M) * p_aug * kCsaLimbs * sizeof(long long), st));
  CK(cudaMemsetAsync(d.work, 0, (d.D + 2) * sizeof(uint32_t), st));
  CK(cudaMemsetAsync(d.nsmall, 0, (d.D + 2) * sizeof(uint32_t), st));
  CK(cudaMemsetAsync(d.ntiny, 0, (d.D + 2) * sizeof(uint32_t), st));
  CK(cudaMemsetAsync(d.nmicro, 0, (d.D + 2) * sizeof(uint32_t), st));
  CK(cudaMemsetAsync(d.lvl_cnt, 0, (d.D + 2) * sizeof(uint32_t), st));
  CK(cudaMemsetAsync(d.counters, 0, 4 * sizeof(unsigned long long), st));

#define CK_LAUNCH(what)                                                                          \
  do {                                                                                           \
    cudaError_t e_ = cudaGetLastError();                                                         \
    if (e_ != cudaSuccess) return fail(BORUTA_ECUDA, "launching %s: %s", what, cudaGetErrorString(e_)); \
  } while (0)
  CK_LAUNCH("(before the iteration)");
  int64_t nk = 0;  // kernels launched by this iteration
  nk += launch_gather_live(d, st);
  CK_LAUNCH("k_gather_live");
  nk += launch_shadow(d, st);
  CK_LAUNCH("k_shadow");
  nk += launch_bootstrap(d, s->tree_grid, st);
  CK_LAUNCH("bootstrap kernels");
  nk += launch_transpose(d, s->permut_grid, st);
  CK_LAUNCH("k_transpose_rows");
  for (int level = 0; level < d.D; ++level) {
    // grids sized to what the level can hold (every split kernel loops over
    // its work, so any grid is correct): at most M * min(2^level, N) nodes, of
    // which at most M * min(2^level, N/33) have more than 32 rows
    const uint64_t width = 1ull << level;
    const uint64_t nodes = static_cast<uint64_t>(d.M) * std::min<uint64_t>(width, static_cast<uint64_t>(d.N));
    const uint64_t big = static_cast<uint64_t>(d.M) * std::min<uint64_t>(width, static_cast<uint64_t>(d.N) / 33);
    const uint64_t groups = big * static_cast<uint64_t>(d.mtry);  // work items of the larger nodes, at most
    const int gs = static_cast<int>(std::min<uint64_t>(s->small_grid, (nodes + 7) / 8));
    const int gi = static_cast<int>(std::min<uint64_t>(s->split_grid, std::max<uint64_t>(1, (groups + 7) / 8)));
    if (timed) CK(cudaEventRecord(s->ev[2 * level], st));
    Dev dl = d;
    set_band(dl, level, big);
    if (s->used_bw.size() != static_cast<size_t>(d.D)) {
      s->used_bw.assign(d.D, 0);
      s->used_bl.assign(d.D, 0);
    }
    s->used_bw[level] = dl.band_w;
    s->used_bl[level] = dl.band_launch;
    nk += launch_split(dl, level, std::max(gs, 1), gi, big, s->split_smem, st, s->st2, s->fork, s->join,
                       timed ? s->hev[2 * level] : nullptr, timed ? s->hev[2 * level + 1] : nullptr);
    CK_LAUNCH("split kernels");
    if (timed) CK(cudaEventRecord(s->ev[2 * level + 1], st));
    nk += launch_children(d, level, st);
    CK_LAUNCH("next-level kernels");
  }
  if (timed) CK(cudaEventRecord(s->iev[0], st));
  if (d.permut_form == 1)
    nk += launch_forest_permut(d, s->permut_grid, st);
  else if (d.permut)
    nk += launch_permut(d, s->permut_grid, s->walk_grid, st);
  else
    nk += launch_treeimp(d, s->tree_grid, st);
  CK_LAUNCH("importance kernels");
  if (timed) CK(cudaEventRecord(s->iev[1], st));
  if (d.permut_form == 1) {  // one importance row for the forest: it is the hit statistic
    Dev d1 = d;
    d1.M = 1;
    d1.stat = 1;
    nk += launch_stats_decide(d1, st);
  } else {
    nk += launch_stats_decide(d, st);
  }
  CK_LAUNCH("k_stats / k_decide");
  s->iter_kernels = nk;
  s->total_kernels += nk;
  CK(cudaMemcpyAsync(s->status_h, d.status, 4 * sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(s->state_pin, d.state, s->p, cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(s->counters_h, d.counters, 4 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
  return 0;
}

static int step_finish(boruta_session* s, int32_t* undecided);

// Histogram tile shape by measurement: the next iteration is run once per
// candidate, timed with CUDA events, and the state is restored after each
// run.  First the column bytes per feature band (12, 24, 48, 96, 192 MiB) x
// one histogram launch per chunk or per band, and a single band (no band
// order), at 8192 row-feature work per group; each run also times every
// tree level.  Then the per-level combination -- at each level the shape
// whose level was fastest -- at 8192, 4096 and 16384 work per group.  The
// fastest run is kept.  The candidates give identical results (the shape
// decides only which warp does which part of the same sums, and when).
static int tune_tiles(boruta_session* s) {
  struct Shape {
    uint32_t gw;
    int64_t bb;  // -1: per level (lvl_bb, lvl_bl)
    int32_t bl;
  };
  const int64_t p = s->p, T = s->max_iter;
  std::vector<int8_t> dec(p);
  std::vector<int32_t> hits(p);
  std::vector<double> hist(static_cast<size_t>(T * p)), smax(T);
  int32_t t0 = 0;
  int rc = boruta_session_read(s, dec.data(), hits.data(), hist.data(), smax.data(), &t0);
  if (rc) return rc;
  cudaEvent_t e[2];
  CK(cudaEventCreate(&e[0]));
  CK(cudaEventCreate(&e[1]));
  s->tune_gw.clear();
  s->tune_bb.clear();
  s->tune_bl.clear();
  s->tune_ms.clear();
  s->tune_lvl_ms.clear();
  const bool graph = s->graph;
  s->graph = false;  // level events need stream launches
  const int policy0 = s->band_policy;
  std::vector<int64_t> comb_bb;
  std::vector<int32_t> comb_bl;
  auto run = [&](const Shape& sh) -> int {
    s->d.group_work = sh.gw;
    if (sh.bb < 0) {
      s->lvl_bb = comb_bb;
      s->lvl_bl = comb_bl;
      s->band_policy = policy0;
    } else {
      s->lvl_bb.clear();
      s->lvl_bl.clear();
      s->band_bytes = sh.bb;
      s->band_policy = sh.bl ? 1 : 2;
    }
    CK(cudaEventRecord(e[0], s->st));
    int r = enqueue_iteration(s, t0 + 1, s->st);
    if (!r) {
      s->pending_t = t0 + 1;
      CK(cudaEventRecord(e[1], s->st));
      r = step_finish(s, nullptr);
    }
    float ms = 0.f;
    if (!r) CK(cudaEventElapsedTime(&ms, e[0], e[1]));
    if (!r) r = boruta_session_write(s, dec.data(), hits.data(), hist.data(), smax.data(), t0);
    if (!r) {
      s->tune_gw.push_back(sh.gw);
      s->tune_bb.push_back(sh.bb);
      s->tune_bl.push_back(sh.bb < 0 ? -1 : sh.bl);
      s->tune_ms.push_back(ms);
      s->tune_lvl_ms.push_back(s->level_ms);
    }
    return r;
  };
  auto best_index = [&]() {
    size_t b = 0;
    for (size_t i = 1; i < s->tune_ms.size(); ++i)
      if (s->tune_ms[i] < s->tune_ms[b]) b = i;
    return b;
  };
  for (int64_t bb : {int64_t{12} << 20, int64_t{24} << 20, int64_t{48} << 20, int64_t{96} << 20,
                     int64_t{192} << 20, int64_t{1} << 40})
    for (int32_t bl : {0, 1})
      if (!rc && !(bl == 1 && bb > (int64_t{192} << 20))) rc = run(Shape{kGroupWork, bb, bl});
  const size_t uniform = rc ? 0 : s->tune_ms.size();
  if (!rc) {
    // per level: the shape of the uniform run whose level was fastest
    const int D = s->d.D;
    comb_bb.assign(D, kBandBytes);
    comb_bl.assign(D, 0);
    for (int l = 0; l < D; ++l) {
      size_t b = 0;
      for (size_t i = 1; i < uniform; ++i)
        if (s->tune_lvl_ms[i].size() > static_cast<size_t>(l) && s->tune_lvl_ms[i][l] < s->tune_lvl_ms[b][l]) b = i;
      comb_bb[l] = s->tune_bb[b];
      comb_bl[l] = s->tune_bl[b];
    }
    for (uint32_t gw : {kGroupWork, 4096u, 16384u})
      if (!rc) rc = run(Shape{gw, -1, 0});
  }
  cudaEventDestroy(e[0]);
  cudaEventDestroy(e[1]);
  s->graph = graph;
  if (rc) return rc;
  const size_t best = best_index();
  s->d.group_work = s->tune_gw[best];
  if (s->tune_bb[best] < 0) {
    s->lvl_bb = comb_bb;
    s->lvl_bl = comb_bl;
    s->band_policy = policy0;
  } else {
    s->lvl_bb.clear();
    s->lvl_bl.clear();
    s->band_bytes = s->tune_bb[best];
    s->band_policy = s->tune_bl[best] ? 1 : 2;
  }
  s->tune_chosen = static_cast<int>(best);
  return 0;
}

static int step_launch(boruta_session* s) {
  if (!s) return fail(BORUTA_EINVAL, "session is NULL");
  if (s->finished) return fail(BORUTA_EINVAL, "the run is finished (no undecided feature or t = max_iter)");
  if (s->pending_t) return fail(BORUTA_EINVAL, "an iteration is already in flight");
  if (s->autotune && !s->tuned) {
    s->tuned = true;
    const int rc = tune_tiles(s);
    if (rc) return rc;
  }
  const int t = s->t + 1;
  if (!s->graph) {
    const int rc = enqueue_iteration(s, t, s->st);
    if (rc) return rc;
  } else {
    // The iteration is captured (on the session's own capture stream: the
    // caller's may be the legacy default stream, which cannot be captured)
    // into a graph; the executable graph of the previous iteration is updated
    // in place (kernel arguments, grids and copy sizes change with t and the
    // live columns) and replayed on the caller's stream, or built again when
    // the update is refused (the launch sequence changed).
    CK(cudaStreamBeginCapture(s->gst, cudaStreamCaptureModeThreadLocal));
    const int rc = enqueue_iteration(s, t, s->gst);
    cudaGraph_t g = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(s->gst, &g);
    if (rc) {
      if (g) cudaGraphDestroy(g);
      return rc;
    }
    if (ec != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      return fail(BORUTA_ECUDA, "graph capture: %s", cudaGetErrorString(ec));
    }
    bool updated = false;
    if (s->gexec) {
      cudaGraphExecUpdateResultInfo info;
      updated = cudaGraphExecUpdate(s->gexec, g, &info) == cudaSuccess;
      if (!updated) {
        cudaGetLastError();
        cudaGraphExecDestroy(s->gexec);
        s->gexec = nullptr;
      }
    }
    if (!updated) {
      const cudaError_t ei = cudaGraphInstantiate(&s->gexec, g, 0);
      if (ei != cudaSuccess) {
        cudaGraphDestroy(g);
        s->gexec = nullptr;
        return fail(BORUTA_ECUDA, "graph instantiation: %s", cudaGetErrorString(ei));
      }
      ++s->graph_builds;
    } else {
      ++s->graph_updates;
    }
    cudaGraphDestroy(g);
    CK(cudaGraphLaunch(s->gexec, s->st));
  }
  s->pending_t = t;
  return 0;
}

// Waits for the iteration enqueued by step_launch and takes its results.
static int step_finish(boruta_session* s, int32_t* undecided) {
  Dev& d = s->d;
  const int t = s->pending_t;
  s->pending_t = 0;
  CK(cudaStreamSynchronize(s->st));
  const unsigned long long* bytes = s->counters_h;
  const uint32_t err = s->status_h[0];
  if (err) {
    s->finished = true;
    if (err & kErrPool) return fail(BORUTA_EOVERFLOW, "node pool capacity (%u) exceeded", d.cap);
    if (err & kErrWeight) return fail(BORUTA_EOVERFLOW, "a bootstrap count exceeded 255");
    if (err & kErrAcc) return fail(BORUTA_EOVERFLOW, "an importance term left the exact accumulator range");
    return fail(BORUTA_EINVAL, "device reported error flags 0x%x", err);
  }
  s->split_ms = 0.0;
  s->hist_ms = 0.0;
  s->level_ms.assign(d.D + 1, 0.0);
  s->level_hist_ms.assign(d.D + 1, 0.0);
  for (int level = 0; level < d.D && !s->graph; ++level) {  // graph replays carry no level events
    float ms = 0.f, hms = 0.f;
    CK(cudaEventElapsedTime(&ms, s->ev[2 * level], s->ev[2 * level + 1]));
    CK(cudaEventElapsedTime(&hms, s->hev[2 * level], s->hev[2 * level + 1]));
    s->split_ms += ms;
    s->hist_ms += hms;
    s->level_ms[level] = ms;
    s->level_hist_ms[level] = hms;
  }
  s->split_launches = d.D;
  s->split_bytes = static_cast<double>(bytes[0]);
  s->hist_bytes = static_cast<double>(bytes[2]);
  s->imp_ms = 0.0;
  if (!s->graph) {
    float ims = 0.f;
    CK(cudaEventElapsedTime(&ims, s->iev[0], s->iev[1]));
    s->imp_ms = ims;
  }
  s->imp_visits = static_cast<double>(bytes[3]);
  std::memcpy(s->state_h.data(), s->state_pin, s->p);
  s->t = t;
  const int32_t und = static_cast<int32_t>(s->status_h[1]);
  s->finished = und == 0 || t >= s->max_iter;
  if (undecided) *undecided = und;
  return 0;
}

int boruta_session_step(boruta_session* s, int32_t* undecided) {
  int rc = step_launch(s);
  if (rc) return rc;
  return step_finish(s, undecided);
}

int boruta_session_read(boruta_session* s, int8_t* decision, int32_t* hits, double* imp_history,
                        double* shadow_max, int32_t* t) {
  if (!s) return fail(BORUTA_EINVAL, "session is NULL");
  const Dev& d = s->d;
  if (decision) CK(cudaMemcpyAsync(decision, d.state, s->p, cudaMemcpyDeviceToHost, s->st));
  if (hits) CK(cudaMemcpyAsync(hits, d.hits, s->p * sizeof(int32_t), cudaMemcpyDeviceToHost, s->st));
  if (imp_history)
    CK(cudaMemcpyAsync(imp_history, d.hist, static_cast<size_t>(s->max_iter) * s->p * sizeof(double),
                       cudaMemcpyDeviceToHost, s->st));
  if (shadow_max)
    CK(cudaMemcpyAsync(shadow_max, d.smax, s->max_iter * sizeof(double), cudaMemcpyDeviceToHost, s->st));
  CK(cudaStreamSynchronize(s->st));
  if (t) *t = s->t;
  return 0;
}

int boruta_session_write(boruta_session* s, const int8_t* decision, const int32_t* hits,
                         const double* imp_history, const double* shadow_max, int32_t t) {
  if (!s || !decision || !hits || !imp_history || !shadow_max)
    return fail(BORUTA_EINVAL, "session and all state buffers are required");
  if (t < 0 || t > s->max_iter) return fail(BORUTA_EINVAL, "t = %d outside [0, max_iter]", t);
  const Dev& d = s->d;
  int64_t und = 0;
  for (int64_t j = 0; j < s->p; ++j) {
    if (decision[j] < -1 || decision[j] > 1) return fail(BORUTA_EINVAL, "decision values are -1, 0, 1");
    und += decision[j] == 0;
  }
  CK(cudaMemcpyAsync(d.state, decision, s->p, cudaMemcpyHostToDevice, s->st));
  CK(cudaMemcpyAsync(d.hits, hits, s->p * sizeof(int32_t), cudaMemcpyHostToDevice, s->st));
  CK(cudaMemcpyAsync(d.hist, imp_history, static_cast<size_t>(s->max_iter) * s->p * sizeof(double),
                     cudaMemcpyHostToDevice, s->st));
  CK(cudaMemcpyAsync(d.smax, shadow_max, s->max_iter * sizeof(double), cudaMemcpyHostToDevice, s->st));
  CK(cudaStreamSynchronize(s->st));
  std::memcpy(s->state_h.data(), decision, s->p);
  s->t = t;
  s->finished = und == 0 || t >= s->max_iter;
  return 0;
}

int boruta_session_kernel_stats(boruta_session* s, double* hist_ms, int32_t* launches, double* hist_bytes,
                                double* split_ms, double* split_bytes) {
  if (!s) return fail(BORUTA_EINVAL, "session is NULL");
  if (hist_ms) *hist_ms = s->hist_ms;
  if (launches) *launches = s->split_launches;
  if (hist_bytes) *hist_bytes = s->hist_bytes;
  if (split_ms) *split_ms = s->split_ms;
  if (split_bytes) *split_bytes = s->split_bytes;
  return 0;
}

int boruta_session_tuning(boruta_session* s, int32_t capacity, int32_t* n_tried, uint32_t* group_work,
                          int64_t* band_bytes, int32_t* band_launch, double* ms, int32_t* chosen) {
  if (!s) return fail(BORUTA_EINVAL, "session is NULL");
  const int n = static_cast<int>(s->tune_ms.size());
  if (n_tried) *n_tried = n;
  if (chosen) *chosen = s->tune_chosen;
  for (int i = 0; i < n && i < capacity; ++i) {
    if (group_work) group_work[i] = s->tune_gw[i];
    if (band_bytes) band_bytes[i] = s->tune_bb[i];
    if (band_launch) band_launch[i] = s->tune_bl[i];
    if (ms) ms[i] = s->tune_ms[i];
  }
  return 0;
}

int boruta_session_kernel_launches(boruta_session* s, int64_t* kernels) {
  if (!s) return fail(BORUTA_EINVAL, "session is NULL");
  if (kernels) *kernels = s->iter_kernels;
  return 0;
}

int boruta_session_tuning_levels(boruta_session* s, int32_t capacity, int32_t* n_levels, int64_t* band_bytes,
                                 int32_t* band_launch, double* level_ms) {
  if (!s) return fail(BORUTA_EINVAL, "session is NULL");
  if (capacity < 0) return fail(BORUTA_EINVAL, "capacity < 0");
  const int D = s->d.D;
  if (n_levels) *n_levels = D;
  for (int l = 0; l < D && l < capacity; ++l) {
    const bool per = l < static_cast<int>(s->lvl_bb.size());
    const bool used = l < static_cast<int>(s->used_bl.size());
    if (band_bytes) band_bytes[l] = per ? s->lvl_bb[l] : s->band_bytes;
    if (band_launch) band_launch[l] = used ? s->used_bl[l] : -1;
  }
  if (level_ms)
    for (size_t i = 0; i < s->tune_lvl_ms.size(); ++i)
      for (int l = 0; l < D && l < capacity; ++l)
        level_ms[i * static_cast<size_t>(capacity) + l] =
            l < static_cast<int>(s->tune_lvl_ms[i].size()) ? s->tune_lvl_ms[i][l] : 0.0;
  return 0;
}

int boruta_session_importance_stats(boruta_session* s, double* ms, double* node_visits) {
  if (!s) return fail(BORUTA_EINVAL, "session is NULL");
  if (ms) *ms = s->imp_ms;
  if (node_visits) *node_visits = s->imp_visits;
  return 0;
}

static int copy_out(boruta_session* s, const void* src, int64_t bytes, void* host, int64_t cap,
                    int64_t* need) {
  if (need) *need = bytes;
  if (!host) return 0;
  if (cap < bytes) return fail(BORUTA_EINVAL, "capacity %lld < %lld bytes", (long long)cap, (long long)bytes);
  CK(cudaMemcpyAsync(host, src, bytes, cudaMemcpyDeviceToHost, s->st));
  CK(cudaStreamSynchronize(s->st));
  return 0;
}

int boruta_session_dump(boruta_session* s, int what, void* host, int64_t capacity, int64_t* bytes) {
  if (!s) return fail(BORUTA_EINVAL, "session is NULL");
  const Dev& d = s->d;
  if (s->t == 0) return fail(BORUTA_EINVAL, "no iteration has run yet");
  switch (what) {
    case BORUTA_DUMP_SHADOW: {
      const int64_t need = static_cast<int64_t>(d.n_sha) * d.N;
      if (bytes) *bytes = need;
      if (!host) return 0;
      if (capacity < need) return fail(BORUTA_EINVAL, "capacity too small");
      CK(cudaMemcpy2DAsync(host, d.N, d.Xaug + static_cast<int64_t>(d.p_live) * d.ldN, d.ldN, d.N, d.n_sha,
                           cudaMemcpyDeviceToHost, s->st));
      CK(cudaStreamSynchronize(s->st));
      return 0;
    }
    case BORUTA_DUMP_BOOT:
      return copy_out(s, d.bootcnt, static_cast<int64_t>(d.M) * d.N * 4, host, capacity, bytes);
    case BORUTA_DUMP_IMP:
      return copy_out(s, d.imp, static_cast<int64_t>(d.permut_form == 1 ? 1 : d.M) * d.p_aug * 8, host, capacity,
                      bytes);
    case BORUTA_DUMP_STAT:
      return copy_out(s, d.s, static_cast<int64_t>(d.p_aug) * 8, host, capacity, bytes);
    case BORUTA_DUMP_LIVE:
      return copy_out(s, s->live_d, static_cast<int64_t>(d.p_live) * 4, host, capacity, bytes);
    case BORUTA_DUMP_LEVELS: {
      const int64_t need = static_cast<int64_t>(d.D + 1) * 3 * 8;
      if (bytes) *bytes = need;
      if (!host) return 0;
      if (capacity < need) return fail(BORUTA_EINVAL, "capacity too small");
      std::vector<uint32_t> cnt(d.D + 2);
      CK(cudaMemcpy(cnt.data(), d.lvl_cnt, (d.D + 2) * 4, cudaMemcpyDeviceToHost));
      double* o = static_cast<double*>(host);
      for (int l = 0; l <= d.D; ++l) {
        const bool timed = l < static_cast<int>(s->level_ms.size());
        o[3 * l] = cnt[l];
        o[3 * l + 1] = timed ? s->level_ms[l] : 0.0;
        o[3 * l + 2] = timed ? s->level_hist_ms[l] : 0.0;
      }
      return 0;
    }
    case BORUTA_DUMP_NODES:
    case BORUTA_DUMP_TREE_PTR: {
      std::vector<uint32_t> off(d.D + 2), cnt(d.D + 2);
      CK(cudaMemcpy(off.data(), d.lvl_off, (d.D + 2) * 4, cudaMemcpyDeviceToHost));
      CK(cudaMemcpy(cnt.data(), d.lvl_cnt, (d.D + 2) * 4, cudaMemcpyDeviceToHost));
      const uint32_t total = off[d.D] + cnt[d.D];
      std::vector<uint32_t> tree(total), heap(total), len(total), n(total), split(total);
      std::vector<double> delta(total);
      std::vector<uint32_t> cnts(d.kind ? 0 : static_cast<size_t>(total) * d.C);
      std::vector<int64_t> S(d.kind ? total : 0);
      CK(cudaMemcpy(tree.data(), d.nd_tree, total * 4ull, cudaMemcpyDeviceToHost));
      CK(cudaMemcpy(heap.data(), d.nd_heap, total * 4ull, cudaMemcpyDeviceToHost));
      CK(cudaMemcpy(len.data(), d.nd_len, total * 4ull, cudaMemcpyDeviceToHost));
      CK(cudaMemcpy(n.data(), d.nd_n, total * 4ull, cudaMemcpyDeviceToHost));
      CK(cudaMemcpy(split.data(), d.nd_split, total * 4ull, cudaMemcpyDeviceToHost));
      CK(cudaMemcpy(delta.data(), d.nd_delta, total * 8ull, cudaMemcpyDeviceToHost));
      if (d.kind)
        CK(cudaMemcpy(S.data(), d.nd_S, total * 8ull, cudaMemcpyDeviceToHost));
      else
        CK(cudaMemcpy(cnts.data(), d.nd_cnt, cnts.size() * 4ull, cudaMemcpyDeviceToHost));
      std::vector<std::vector<boruta_node>> per(d.M);
      for (int l = 0; l <= d.D; ++l) {
        for (uint32_t k = off[l]; k < off[l] + cnt[l]; ++k) {
          boruta_node r;
          std::memset(&r, 0, sizeof r);
          r.heap = heap[k];
          r.depth = l;
          r.feature = split[k] == kLeaf ? -1 : static_cast<int32_t>(split[k] >> 8);
          r.bin = split[k] == kLeaf ? 0 : static_cast<int32_t>(split[k] & 255u);
          r.n_rows = len[k];
          r.n = n[k];
          if (d.kind)
            r.stat[0] = S[k];
          else
            for (int c = 0; c < d.C; ++c) r.stat[c] = cnts[static_cast<size_t>(k) * d.C + c];
          r.delta = split[k] == kLeaf ? 0.0 : delta[k];
          per[tree[k]].push_back(r);
        }
      }
      if (what == BORUTA_DUMP_TREE_PTR) {
        const int64_t need = static_cast<int64_t>(d.M + 1) * 8;
        if (bytes) *bytes = need;
        if (!host) return 0;
        if (capacity < need) return fail(BORUTA_EINVAL, "capacity too small");
        int64_t* o = static_cast<int64_t*>(host);
        o[0] = 0;
        for (int tau = 0; tau < d.M; ++tau) o[tau + 1] = o[tau] + static_cast<int64_t>(per[tau].size());
        return 0;
      }
      const int64_t need = static_cast<int64_t>(total) * sizeof(boruta_node);
      if (bytes) *bytes = need;
      if (!host) return 0;
      if (capacity < need) return fail(BORUTA_EINVAL, "capacity too small");
      boruta_node* o = static_cast<boruta_node*>(host);
      for (int tau = 0; tau < d.M; ++tau)
        for (const auto& r : per[tau]) *o++ = r;
      return 0;
    }
    default:
      return fail(BORUTA_EINVAL, "unknown dump %d", what);
  }
}

void boruta_session_destroy(boruta_session* s) { delete s; }

int boruta_fit(const uint8_t* X, int64_t ld, const void* y, int64_t N, int64_t p, int task, int n_trees,
               int max_depth, int mtry, int n_bins, int max_iter, double alpha, uint64_t seed,
               const boruta_opts* opts, boruta_result* out) {
  if (!out || !out->decision || !out->hits || !out->imp_history || !out->shadow_max)
    return fail(BORUTA_EINVAL, "out and its buffers must not be NULL");
  boruta_session* s = nullptr;
  int rc = boruta_session_create(X, ld, y, N, p, task, n_trees, max_depth, mtry, n_bins, max_iter,
                                 alpha, seed, opts, &s);
  if (rc) return rc;
  int32_t und = 1;
  while (!s->finished) {
    rc = boruta_session_step(s, &und);
    if (rc) break;
  }
  int32_t t = 0;
  if (!rc) rc = boruta_session_read(s, out->decision, out->hits, out->imp_history, out->shadow_max, &t);
  out->iterations = t;
  std::string msg = g_error;
  boruta_session_destroy(s);
  g_error = msg;
  return rc;
}

}  // extern "C"

struct boruta_batch {
  std::vector<boruta_session*> ss;
  std::vector<cudaEvent_t> done;  // per job, recorded after its iteration
  cudaStream_t user = nullptr;
  cudaEvent_t ready = nullptr;
  bool failed = false;
  ~boruta_batch() {
    for (auto* s : ss) boruta_session_destroy(s);
    for (cudaEvent_t e : done)
      if (e) cudaEventDestroy(e);
    if (ready) cudaEventDestroy(ready);
  }
};

extern "C" {

int boruta_batch_create(int n_jobs, const boruta_job* jobs, const boruta_opts* opts, boruta_batch** out) {
  if (!out || n_jobs < 0 || (n_jobs > 0 && !jobs)) return fail(BORUTA_EINVAL, "bad batch arguments");
  *out = nullptr;
  boruta_opts base;
  if (opts)
    base = *opts;
  else
    boruta_default_opts(&base);
  auto* b = new boruta_batch();
  b->user = static_cast<cudaStream_t>(base.stream);
  b->ss.assign(n_jobs, nullptr);
  b->done.assign(n_jobs, nullptr);
  auto bail = [&](int rc) {
    const std::string msg = g_error;
    delete b;
    g_error = msg;
    return rc;
  };
  if (cudaEventCreateWithFlags(&b->ready, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventRecord(b->ready, b->user) != cudaSuccess)
    return bail(fail(BORUTA_ECUDA, "batch: event creation failed"));
  for (int j = 0; j < n_jobs; ++j) {
    const boruta_job& J = jobs[j];
    boruta_opts o = base;
    o.job = base.job + static_cast<uint32_t>(j);
    o.n_classes = J.n_classes;
    cudaStream_t st = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamWaitEvent(st, b->ready, 0) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->done[j], cudaEventDisableTiming) != cudaSuccess) {
      if (st) cudaStreamDestroy(st);
      return bail(fail(BORUTA_ECUDA, "job %d: stream creation failed", j));
    }
    o.stream = st;
    const int rc = boruta_session_create(J.X, J.ld, J.y, J.N, J.p, J.task, J.n_trees, J.max_depth, J.mtry,
                                         J.n_bins, J.max_iter, J.alpha, J.seed, &o, &b->ss[j]);
    if (rc) {
      cudaStreamDestroy(st);
      return bail(fail(rc, "job %d: %s", j, std::string(g_error).c_str()));
    }
    b->ss[j]->own_stream = true;
  }
  *out = b;
  return 0;
}

// Lockstep: the unfinished jobs' iterations are enqueued one after another
// (each on its own stream, after the caller's stream), then collected.
int boruta_batch_step(boruta_batch* b, int32_t* running) {
  if (!b) return fail(BORUTA_EINVAL, "batch is NULL");
  if (b->failed) return fail(BORUTA_EINVAL, "batch: a previous step failed");
  std::vector<int> active;
  for (int j = 0; j < static_cast<int>(b->ss.size()); ++j)
    if (!b->ss[j]->finished) active.push_back(j);
  if (active.empty()) return fail(BORUTA_EINVAL, "batch: every job is finished");
  int rc = 0;
  if (cudaEventRecord(b->ready, b->user) != cudaSuccess) rc = fail(BORUTA_ECUDA, "batch: event record failed");
  for (int j : active) {
    if (rc) break;
    if (cudaStreamWaitEvent(b->ss[j]->st, b->ready, 0) != cudaSuccess) {
      rc = fail(BORUTA_ECUDA, "job %d: stream wait failed", j);
      break;
    }
    if ((rc = step_launch(b->ss[j]))) {
      fail(rc, "job %d: %s", j, std::string(g_error).c_str());
      break;
    }
    if (cudaEventRecord(b->done[j], b->ss[j]->st) != cudaSuccess ||
        cudaStreamWaitEvent(b->user, b->done[j], 0) != cudaSuccess)
      rc = fail(BORUTA_ECUDA, "job %d: event record failed", j);
  }
  for (int j : active) {
    if (!b->ss[j]->pending_t) continue;
    int32_t und = 0;
    const int r = step_finish(b->ss[j], &und);
    if (r && !rc) rc = fail(r, "job %d: %s", j, std::string(g_error).c_str());
  }
  if (rc) {
    b->failed = true;
    return rc;
  }
  int32_t left = 0;
  for (auto* s : b->ss) left += s->finished ? 0 : 1;
  if (running) *running = left;
  return 0;
}

int boruta_batch_run(boruta_batch* b, int iterations, int32_t* running) {
  if (!b) return fail(BORUTA_EINVAL, "batch is NULL");
  if (b->failed) return fail(BORUTA_EINVAL, "batch: a previous step failed");
  if (iterations < 0) return fail(BORUTA_EINVAL, "iterations = %d", iterations);
  const int n = static_cast<int>(b->ss.size());
  std::vector<int> left(n, 0);
  int rc = 0;
  if (cudaEventRecord(b->ready, b->user) != cudaSuccess) rc = fail(BORUTA_ECUDA, "batch: event record failed");
  auto launch = [&](int j) {
    if (cudaStreamWaitEvent(b->ss[j]->st, b->ready, 0) != cudaSuccess)
      return fail(BORUTA_ECUDA, "job %d: stream wait failed", j);
    int r = step_launch(b->ss[j]);
    if (r) return fail(r, "job %d: %s", j, std::string(g_error).c_str());
    if (cudaEventRecord(b->done[j], b->ss[j]->st) != cudaSuccess)
      return fail(BORUTA_ECUDA, "job %d: event record failed", j);
    return 0;
  };
  for (int j = 0; j < n && !rc; ++j) {
    left[j] = b->ss[j]->finished ? 0 : iterations;
    if (left[j] > 0) rc = launch(j);
  }
  // each job's next iteration is enqueued as soon as its last one completes
  for (bool busy = true; busy;) {
    busy = false;
    for (int j = 0; j < n; ++j) {
      if (!b->ss[j]->pending_t) continue;
      const cudaError_t q = cudaEventQuery(b->done[j]);
      if (q == cudaErrorNotReady && !rc) {
        busy = true;
        continue;
      }
      if (q != cudaSuccess && q != cudaErrorNotReady) cudaGetLastError();
      int32_t und = 0;
      const int r = step_finish(b->ss[j], &und);
      if (r && !rc) rc = fail(r, "job %d: %s", j, std::string(g_error).c_str());
      if (--left[j] > 0 && !b->ss[j]->finished && !rc) {
        rc = launch(j);
        busy = true;
      }
    }
    if (busy) std::this_thread::yield();
  }
  for (int j = 0; j < n; ++j)
    if (cudaStreamWaitEvent(b->user, b->done[j], 0) != cudaSuccess && !rc)
      rc = fail(BORUTA_ECUDA, "job %d: stream wait failed", j);
  if (rc) {
    b->failed = true;
    return rc;
  }
  int32_t still = 0;
  for (auto* s : b->ss) still += s->finished ? 0 : 1;
  if (running) *running = still;
  return 0;
}

int boruta_batch_kernel_launches(boruta_batch* b, int64_t* kernels) {
  if (!b) return fail(BORUTA_EINVAL, "batch is NULL");
  int64_t n = 0;
  for (const boruta_session* s : b->ss) n += s->total_kernels;
  if (kernels) *kernels = n;
  return 0;
}

int boruta_batch_read(boruta_batch* b, int job, int8_t* decision, int32_t* hits, double* imp_history,
                      double* shadow_max, int32_t* t) {
  if (!b || job < 0 || job >= static_cast<int>(b->ss.size())) return fail(BORUTA_EINVAL, "bad batch job index");
  const int rc = boruta_session_read(b->ss[job], decision, hits, imp_history, shadow_max, t);
  if (rc) return fail(rc, "job %d: %s", job, std::string(g_error).c_str());
  return 0;
}

void boruta_batch_destroy(boruta_batch* b) { delete b; }

int boruta_fit_batch(int n_jobs, const boruta_job* jobs, const boruta_opts* opts, boruta_result* outs) {
  if (n_jobs < 0 || (n_jobs > 0 && (!jobs || !outs))) return fail(BORUTA_EINVAL, "bad batch arguments");
  for (int j = 0; j < n_jobs; ++j)
    if (!outs[j].decision || !outs[j].hits || !outs[j].imp_history || !outs[j].shadow_max)
      return fail(BORUTA_EINVAL, "job %d: result buffers must not be NULL", j);
  boruta_batch* b = nullptr;
  int rc = boruta_batch_create(n_jobs, jobs, opts, &b);
  int32_t running = n_jobs;
  if (!rc && n_jobs > 0) rc = boruta_batch_run(b, kMaxIterations, &running);
  for (int j = 0; j < n_jobs && !rc; ++j) {
    int32_t t = 0;
    rc = boruta_batch_read(b, j, outs[j].decision, outs[j].hits, outs[j].imp_history, outs[j].shadow_max, &t);
    outs[j].iterations = t;
  }
  const std::string msg = g_error;
  boruta_batch_destroy(b);
  g_error = msg;
  return rc;
}

// ---------------------------------------------------------------- primitives
int boruta_philox(const uint32_t* ctr, const uint32_t* key, uint32_t* out, int64_t n, void* stream) {
  if (n < 0 || (n > 0 && (!ctr || !key || !out))) return fail(BORUTA_EINVAL, "bad arguments");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (n) launch_debug_philox(ctr, key, out, n, st);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(st));
  return 0;
}

int boruta_perm(uint64_t n_domain, uint64_t seed, uint32_t w1, uint32_t w2, uint32_t w3,
                const uint64_t* idx, uint64_t* out, int64_t count, void* stream) {
  if (n_domain < 1 || n_domain > 0xFFFFFFFFull || count < 0) return fail(BORUTA_EINVAL, "bad domain");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (count) launch_debug_perm(static_cast<uint32_t>(n_domain), seed, w1, w2, w3, idx, out, count, st);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(st));
  return 0;
}

int boruta_u256_to_double(const uint64_t* v, double* out, int64_t n, void* stream) {
  if (n < 0) return fail(BORUTA_EINVAL, "bad size");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (n) launch_debug_u256(v, out, n, st);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(st));
  return 0;
}

int boruta_binom_tails(const int32_t* t, const int32_t* h, double* p_acc, double* p_rej, int64_t n,
                       void* stream) {
  if (n < 0) return fail(BORUTA_EINVAL, "bad size");
  if (n == 0) return 0;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  std::vector<int32_t> th(n);
  CK(cudaMemcpyAsync(th.data(), t, n * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  for (int64_t i = 0; i < n; ++i)
    if (th[i] < 0 || th[i] > 126) return fail(BORUTA_EINVAL, "t[%lld] = %d outside [0, 126]", (long long)i, th[i]);
  std::vector<u128> tri(127 * 127, 0);
  tri[0] = 1;
  for (int r = 1; r <= 126; ++r) {
    tri[r * 127] = 1;
    for (int k = 1; k <= r; ++k) tri[r * 127 + k] = tri[(r - 1) * 127 + k - 1] + tri[(r - 1) * 127 + k];
  }
  void* dt = nullptr;
  CK(cudaMalloc(&dt, tri.size() * sizeof(u128)));
  cudaError_t e = cudaMemcpy(dt, tri.data(), tri.size() * sizeof(u128), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    launch_debug_binom(static_cast<const u128*>(dt), t, h, p_acc, p_rej, n, st);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  }
  cudaFree(dt);
  if (e != cudaSuccess) return fail(BORUTA_ECUDA, "binom tails: %s", cudaGetErrorString(e));
  return 0;
}

}  // extern "C"
