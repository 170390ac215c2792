// Internal interface between the host driver (api.cu) and the kernels (kernels.cu).
#pragma once
#include <cstdint>

#include <cuda_runtime.h>

#include "device.cuh"

namespace bgb {

// Everything a kernel needs, passed by value.  Sizes are fixed for a
// session except the per-iteration block (t, p_live, n_sha, p_aug, mtry).
struct Dev {
  // ---- problem
  const uint8_t* X;        // column-major bins, column j at X + j*ld
  int64_t ld;
  const uint8_t* ycls;     // labels (classification)
  const int64_t* yreg;     // fixed-point targets (regression)
  int32_t N, ldN, p, kind, C, B, D, M, max_iter;
  int32_t precision, tie_break, stat, permut;
  int32_t permut_form;           // Alg. 3 rows: 0 = each tree's OOB rows, 1 = all rows, forest prediction
  uint64_t seed;
  uint32_t job;
  double kl_eps, alpha;
  // ---- iteration
  int32_t t, p_live, n_sha, p_aug, mtry;
  const int32_t* live;           // [p_live]
  // ---- buffers
  uint8_t* Xaug;                 // [p_aug][ldN]: live original columns, then the shadows
  uint32_t* bootcnt;             // [M][N] bootstrap draw counts
  uint32_t* rows[2];             // [M][N] node-ordered row entries (row << 8 | weight)
  uint32_t* oob;                 // [M][N] out-of-bag rows, ascending
  uint32_t* oob_cnt;             // [M]
  uint32_t* piv;                 // [N] Alg. 3 flush_index of the iteration (Permut only)
  uint8_t* Xrow;                 // [N][ldP] row-major copy of Xaug, built each iteration: the
                                 //   small-node split and the Alg. 3 walks read one row's bins
                                 //   of many columns, which a row's record keeps together
  int32_t ldP;                   // round16(p_aug) of the iteration
  // ---- node pool (level-major; within a level, ordered by (tree, heap))
  uint32_t cap;
  uint32_t *nd_tree, *nd_heap, *nd_seg, *nd_len, *nd_n;
  uint32_t* nd_cnt;              // [cap][C] weighted class counts
  int64_t* nd_S;                 // [cap] weighted target sum
  uint32_t *nd_split, *nd_child; // split = feature << 8 | bin, kLeaf for leaves
  uint2* nd_sc;                  // (split, child) of every node, packed for the Alg. 3 walks (Permut only)
  double* nd_delta;
  uint32_t *nd_lrows, *nd_ln;    // left child: distinct rows, weighted rows
  uint32_t* nd_lcnt;             // [cap][C]
  int64_t* nd_lS;
  uint32_t *lvl_off, *lvl_cnt;   // [D + 2]
  uint32_t* work;                // [D + 2] per level: number of nodes in `big`
  uint32_t* chunk;               // [kScanBlocks] per-block split counts
  uint32_t* big;                 // [big_cap] this level's active nodes with > 32 rows
  uint32_t* small;               // [level_cap] this level's active nodes with <= 32 rows
  uint32_t* nsmall;              // [D + 2] per level: number of 17..32-row nodes at the start of `small`
  uint32_t* ntiny;               // [D + 2] per level: number of 9..16-row nodes at the end of `small`
  uint32_t* micro;               // [small_cap] this level's active nodes with <= 8 rows
  uint32_t* nmicro;              // [D + 2] per level: number of them
  uint32_t small_cap;            // entries of `small`
  void* ninfo;                   // [big_cap] node totals of `big`, by rank
  void* cand;                    // [big_cap * kItemsPerNode] best candidate per grouped item
  uint64_t* items_u;             // [item_cap] (node rank, slot, feature) per item; each node's
                                 //   mtry items together, ordered by feature band
  uint64_t* items_s;             // [item_cap] groups (node rank, first item, count), by band
  uint64_t* items_b;             // [item_cap] per group: its node's row-buffer offset << 24 | rows
  void* fbest;                   // [item_cap] packed best candidate per (node rank, slot)
  uint32_t* band_cnt;            // [kMaxBands + 1] groups per band, then cursors; last: total
  uint64_t item_cap;
  int32_t band_w, nbands;        // columns per band (0: grouped path only), bands
  uint32_t group_work;           // row x feature work per group of a larger node (tile shape)
  int32_t band_launch;           // 1: one histogram launch per feature band, 0: one per chunk
  uint32_t chunk0, chunk_cap;    // band path: first larger node of the chunk, nodes per chunk
  // ---- importance and Boruta state
  long long* acc;                // [M][p_aug][kCsaLimbs] exact per-tree accumulators (carry-save)
  double* imp;                   // [M][p_aug]
  double* s;                     // [p_aug]
  const u128* pascal;            // [127][127] binomial coefficients C(t, k)
  int8_t* state;                 // [p]
  int32_t* hits;                 // [p]
  double* hist;                  // [max_iter][p]
  double* smax;                  // [max_iter]
  uint32_t* status;              // [0] error flags, [1] undecided count, [2] n_classes seen
  // ---- Alg. 3 as printed (permut_form = 1)
  long long* fbase;              // [N][K][kCsaLimbs] exact sum over trees of each row's leaf value
  double* fbase_mean;            // [N][K] the forest's prediction (K = C, or 1 for regression)
  long long* facc;               // [frows][p_aug][K][kCsaLimbs] per (row of the block, column) delta
  uint32_t frows;                // rows per block
  unsigned long long* counters;  // [0] split-stage algorithmic bytes, [1] max |y|,
                                 // [2] histogram-kernel algorithmic bytes,
                                 // [3] node visits of the Alg. 3 tree walks
};

constexpr int kScanBlocks = 512;
constexpr int kSplitThreads = 256;
constexpr int kItemsPerNode = 16;  // work items (groups of draw slots) per larger node
constexpr int kMaxBands = 256;     // feature bands of the band-sorted path
constexpr int64_t kBandBytes = 48ll << 20;  // default column bytes per feature band
constexpr uint64_t kMaxItems = 128ull << 20;  // plan buffer capacity (items)
constexpr int kMaxIterations = 126;          // max_iter limit (exact binomial tails in 128 bits)
#ifndef BORUTA_STAGED_ROWS
#define BORUTA_STAGED_ROWS 64
#endif
constexpr uint32_t kRegRows = BORUTA_STAGED_ROWS;  // node rows a warp stages in shared memory
constexpr uint32_t kGroupWork = 8192;        // default row x feature work per group for larger nodes
// row state the method moves per row and tree level besides the bins: the
// row's entry read and rewritten by the partition (4 + 4 B), its weight and
// label (1 + 1 B), or weight and 8-byte fixed-point target (regression)
constexpr uint32_t kRowStateClass = 10, kRowStateReg = 17;

// launchers (kernels.cu); each returns the number of kernels it launched
void launch_validate(const Dev& d, cudaStream_t st);
int launch_shadow(const Dev& d, cudaStream_t st);
int launch_bootstrap(const Dev& d, int grid, cudaStream_t st);
// split.cu: one level's split search.  Nodes are classified on `st`; the
// small-node kernel then runs on `st2` while the larger-node kernels run on
// `st` (fork/join through the two events).
// hist_start/hist_end are recorded on `st` around the histogram kernel.
int launch_split(const Dev& d, int level, int grid_small, int grid_big, uint64_t big_bound, size_t smem, cudaStream_t st,
                  cudaStream_t st2, cudaEvent_t fork, cudaEvent_t join, cudaEvent_t hist_start,
                  cudaEvent_t hist_end);
size_t ninfo_bytes(int variant);
int split_variant(int kind, int C);
int variant_classes(int variant);  // largest class count of a kernel variant (1 for regression)
void split_kernel_ptrs(int variant, const void** ptrs, int* n);  // kernels taking dynamic shared memory
const void* small_kernel_ptr(int variant);  // for its occupancy
size_t cand_bytes(int variant);
size_t packed_bytes(int variant);
int launch_gather_live(const Dev& d, cudaStream_t st);
int launch_children(const Dev& d, int level, cudaStream_t st);
int launch_treeimp(const Dev& d, int grid, cudaStream_t st);
int launch_permut(const Dev& d, int grid, int walk_grid, cudaStream_t st);
// Xrow (the row-major copy of Xaug): built once per iteration, after the
// shadows, for the small-node split and the walks
int launch_transpose(const Dev& d, int grid, cudaStream_t st);
int launch_forest_permut(const Dev& d, int grid, cudaStream_t st);
const void* permut_kernel_ptr(int precision);  // for its occupancy
size_t permut_smem_bytes(int D);                // its dynamic shared memory per block (128 threads)
int launch_stats_decide(const Dev& d, cudaStream_t st);
// Warp-private histogram layout.  A lane scans 8 consecutive bins, so one
// padding slot follows every 8 bins: lane l's block then starts at a bank
// offset coprime with 32 and the scan reads are free of bank conflicts.
//   classification: count(b, k) at word b*C + k + b/8, or, packed (a node
//                   of total weight below 4096 and at most five classes),
//                   all classes of bin b in the u64 b + b/8
//   regression:     weight(b) at word b + b/8; sum(b) at u64 b + b/8 after the weights
__host__ __device__ inline int hist_words_n(int B) { return (B + (B >> 3) + 2) & ~1; }
__host__ __device__ inline size_t hist_smem_per_warp(int kind, int C, int B) {
  const size_t packed = static_cast<size_t>(B + (B >> 3) + 1) * 8;
  size_t b = kind == 0 ? (static_cast<size_t>(B) * C + (B >> 3) + 1) * 4
                       : static_cast<size_t>(hist_words_n(B)) * 4 + packed;
  if (b < packed) b = packed;
  return (b + 15) & ~static_cast<size_t>(15);
}
// per warp: the histogram, a node's row entries (up to kRegRows), then the
// histogram's occupancy bitmap (256 bits and one spare word, padded to 48 B)
__host__ __device__ inline size_t split_smem_per_warp(int kind, int C, int B) {
  return hist_smem_per_warp(kind, C, B) + kRegRows * 4 + 48;
}
__host__ __device__ inline size_t split_smem_bytes(int kind, int C, int B) {
  return (kSplitThreads / 32) * split_smem_per_warp(kind, C, B);
}

void launch_debug_philox(const uint32_t* ctr, const uint32_t* key, uint32_t* out, int64_t n,
                         cudaStream_t st);
void launch_debug_perm(uint32_t n, uint64_t seed, uint32_t w1, uint32_t w2, uint32_t w3,
                       const uint64_t* idx, uint64_t* out, int64_t count, cudaStream_t st);
void launch_debug_u256(const uint64_t* v, double* out, int64_t n, cudaStream_t st);
void launch_debug_binom(const u128* pascal, const int32_t* t, const int32_t* h, double* pa,
                        double* pr, int64_t n, cudaStream_t st);

}  // namespace bgb
