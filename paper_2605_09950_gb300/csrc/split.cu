// Split search of one tree level (all trees at once): per-node feature
// sample, histograms, exact best-split scan, impurity decrease into the
// TreeImp accumulators (Alg. 2) and the stable row partition.
//
// Kernels of a level:
//   k_classify      leaves, and the lists of small (<= 32 rows) and larger
//                   active nodes.
//   k_split_small   (second stream) one warp per node of at most 32 rows:
//                   one row per lane, left class counts from ballots over the
//                   bin bits against weight and class bit planes (regression:
//                   shuffles, or warp reductions for columns of <= 4 bins).
//   larger nodes, feature-band path (default), in chunks of nodes whose
//   items fit the plan buffers:
//     k_plan_gen / k_plan_scan / k_plan_scatter  the nodes' (node, draw slot)
//                   items ordered by the band of columns their feature lies
//                   in, cut into (node, band) groups sorted by band, so that
//                   the columns being gathered at any moment fit in L2;
//     k_items_band  one warp per group: per feature a warp-private
//                   shared-memory histogram (entries of nodes of <= 64 rows
//                   staged once per group; class weights packed 12 bits
//                   each into one 64-bit word per bin when they fit), a
//                   float pre-screen over the non-empty bins, and the
//                   feature's exact best candidate, kept as the integers
//                   that define it;
//     k_finalize_band  one warp per node: float screen of its features'
//                   candidates, exact argmax, split record and partition.
//   larger nodes, grouped path (split_path = 1, or mtry >= 2^14): k_items
//   (one warp per group of draw slots, exact) and k_finalize.
// Candidate (f, b): rows with bin <= b go left.  Score num/den =
// (A_L n_R + A_R n_L) / (n_L n_R) with A = sum_k c_k^2 (Gini) or S^2
// (variance); scores are compared exactly (256-bit cross products) after a
// float pre-screen; equal scores go to the lower key = (feature index, or
// the draw slot with tie_break = 1) << 8 | bin.
#include <cstdint>
#include <type_traits>

#include "engine.cuh"

// resident CTAs per SM the kernels are compiled for (register budget)
#ifndef BORUTA_SMALL_MINB
#define BORUTA_SMALL_MINB 4
#endif
#ifndef BORUTA_SMALL_AHEAD
#define BORUTA_SMALL_AHEAD 8  // features whose bins a small-node warp loads at once
#endif
#ifndef BORUTA_STREAM_BATCH
#define BORUTA_STREAM_BATCH 8  // rows per lane per pass of a streamed histogram
#endif
#ifndef BORUTA_ITEMS_MINB
#define BORUTA_ITEMS_MINB 3
#endif

namespace bgb {

namespace {

constexpr int kSmallAhead = BORUTA_SMALL_AHEAD;

constexpr unsigned kFull = 0xFFFFFFFFu;

// Class count of a variant: the kernels are instantiated with CM = 3, 4 and 5
// for exactly that many classes (their class loops then unroll to the real
// count), CM = 2 for one or two classes and CM = 8 for six to eight.
template <int CM>
__device__ __forceinline__ int ncls(const Dev& d) {
  return (CM == 3 || CM == 4 || CM == 5) ? CM : d.C;
}

__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

__device__ __forceinline__ const uint8_t* column(const Dev& d, uint32_t f) {
  return d.Xaug + static_cast<int64_t>(f) * d.ldN;
}

// The bin of one row and column for a node's row-by-row reads, from the
// row-major copy: a row's sampled columns then share its few kilobytes
// instead of lying a column apart.
__device__ __forceinline__ uint32_t row_bin(const Dev& d, uint32_t row, uint32_t f) {
  return d.Xrow[static_cast<int64_t>(row) * d.ldP + f];
}

// L2 residency in the histogram kernels.  The bins are gathered band by band
// (the groups are sorted by feature band), and a band's columns must stay in
// L2 while its groups run; the nodes' row entries, streamed once per feature
// group, would otherwise push them out.  So the gathers carry an evict-last
// policy and the entry reads are streaming (evict-first) loads.
__device__ __forceinline__ uint64_t keep_policy() {
  uint64_t p;
  asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}

__device__ __forceinline__ uint32_t ld_keep(const uint8_t* a, uint64_t pol) {
  uint32_t v;
  asm("ld.global.L2::cache_hint.u8 %0, [%1], %2;" : "=r"(v) : "l"(a), "l"(pol));
  return v;
}

__device__ __forceinline__ uint32_t ld_stream(const uint32_t* a) { return __ldcs(a); }

__device__ __forceinline__ void prefetch_l2(const void* a) { asm volatile("prefetch.global.L2 [%0];" ::"l"(a)); }

// Row entries: row << 8 | low byte.  Classification: low byte = y << 5 | w
// (label < 8, bootstrap count < 32); regression: low byte = w (< 256).
template <int KIND>
__device__ __forceinline__ uint32_t ent_w(uint32_t e) {
  return KIND == 0 ? (e & 31u) : (e & 255u);
}
__device__ __forceinline__ uint32_t ent_y(uint32_t e) { return (e >> 5) & 7u; }

template <int CM>
struct Cand {
  U192 num;
  uint64_t den;
  uint32_t key;
  uint32_t nL;
  uint32_t cL[CM];
  long long SL;
  int32_t feat;
  int32_t bin;
  bool valid;
};

template <int CM>
__device__ __forceinline__ bool better(const Cand<CM>& a, const Cand<CM>& b) {
  if (!a.valid) return false;
  if (!b.valid) return true;
  const int c = frac_cmp(a.num, a.den, b.num, b.den);
  if (c != 0) return c > 0;
  return a.key < b.key;
}

__device__ __forceinline__ U192 u192_mul(u128 a, uint64_t b) {
  const u128 lo = static_cast<u128>(static_cast<uint64_t>(a)) * b;
  const u128 hi = static_cast<u128>(static_cast<uint64_t>(a >> 64)) * b + (lo >> 64);
  U192 r;
  r.w[0] = static_cast<uint64_t>(lo);
  r.w[1] = static_cast<uint64_t>(hi);
  r.w[2] = static_cast<uint64_t>(hi >> 64);
  return r;
}

__device__ __forceinline__ U192 u192_add(const U192& a, const U192& b) {
  U192 r;
  u128 s = static_cast<u128>(a.w[0]) + b.w[0];
  r.w[0] = static_cast<uint64_t>(s);
  s = static_cast<u128>(a.w[1]) + b.w[1] + (s >> 64);
  r.w[1] = static_cast<uint64_t>(s);
  r.w[2] = a.w[2] + b.w[2] + static_cast<uint64_t>(s >> 64);
  return r;
}

__device__ __forceinline__ u128 sq_i64(long long v) {
  const uint64_t m = v < 0 ? 0ull - static_cast<uint64_t>(v) : static_cast<uint64_t>(v);
  return static_cast<u128>(m) * m;
}

template <int CM>
struct NodeInfo {
  int64_t base;  // tree row-buffer offset + segment offset
  uint32_t len, n;
  uint32_t cp[CM];
  long long SP;
};

// ---- scores
// Exact u32 -> float for v < 2^24 on the integer and FP32 pipes: the bits
// 0x4B000000 | m are the float 2^23 + m for m < 2^23.
__device__ __forceinline__ float u24_to_float(uint32_t v) {
  const float b = __uint_as_float(0x4B000000u | (v & 0x7FFFFFu));
  return (v & 0x800000u) ? b : b - 8388608.0f;
}

// |v| as float for a 64-bit v, from three exact 22-bit pieces (all terms
// non-negative: relative error below 2^-22)
__device__ __forceinline__ float abs_i64_to_float(long long v) {
  const uint64_t a = v < 0 ? 0ull - static_cast<uint64_t>(v) : static_cast<uint64_t>(v);
  return (u24_to_float(static_cast<uint32_t>(a >> 44)) * 17592186044416.0f +
          u24_to_float(static_cast<uint32_t>(a >> 22) & 0x3FFFFFu) * 4194304.0f) +
         u24_to_float(static_cast<uint32_t>(a) & 0x3FFFFFu);
}

// Float scores of the pre-screen (counts and n below 2^24, so the integer
// inputs convert exactly).  Relative error below 2^-20.
template <int CM>
__device__ __forceinline__ float score_class_f(const uint32_t* cl, const uint32_t* cp, int C, uint32_t nL,
                                               uint32_t n) {
  float AL = 0.0f, AR = 0.0f;
#pragma unroll
  for (int k = 0; k < CM; ++k)
    if (k < C) {
      const float l = u24_to_float(cl[k]), r = u24_to_float(cp[k] - cl[k]);
      AL += l * l;
      AR += r * r;
    }
  return __fdividef(AL, u24_to_float(nL)) + __fdividef(AR, u24_to_float(n - nL));
}

__device__ __forceinline__ float score_reg_f(long long SL, long long SP, uint32_t nL, uint32_t n) {
  const float l = abs_i64_to_float(SL), r = abs_i64_to_float(SP - SL);
  return __fdividef(l * l, u24_to_float(nL)) + __fdividef(r * r, u24_to_float(n - nL));
}

template <int CM>
__device__ __forceinline__ void make_class(Cand<CM>& c, const uint32_t* cl, const uint32_t* cp, int C,
                                           uint32_t nL, uint32_t n) {
  uint64_t AL = 0, AR = 0;
#pragma unroll
  for (int k = 0; k < CM; ++k) {
    c.cL[k] = k < C ? cl[k] : 0u;
    if (k < C) {
      const uint64_t l = cl[k], r = cp[k] - cl[k];
      AL += l * l;
      AR += r * r;
    }
  }
  const uint32_t nR = n - nL;
  c.num = u192_from(static_cast<u128>(AL) * nR + static_cast<u128>(AR) * nL);
  c.den = static_cast<uint64_t>(nL) * nR;
  c.nL = nL;
  c.SL = 0;
  c.valid = true;
}

template <int CM>
__device__ __forceinline__ void make_reg(Cand<CM>& c, long long SL, long long SP, uint32_t nL, uint32_t n) {
  const uint32_t nR = n - nL;
  c.num = u192_add(u192_mul(sq_i64(SL), nR), u192_mul(sq_i64(SP - SL), nL));
  c.den = static_cast<uint64_t>(nL) * nR;
  c.nL = nL;
  c.SL = SL;
#pragma unroll
  for (int k = 0; k < CM; ++k) c.cL[k] = 0u;
  c.valid = true;
}

// Relative window of the float pre-screen.  A float score is within 2^-20 of
// the exact score, so every candidate whose exact score is the maximum has a
// float score above (1 - 2^-16) * (best float score); only those are compared
// exactly.
__device__ __forceinline__ float screen(float m) { return m - m * 0.0000152587890625f; }

// all lanes: out = best of the lane candidates flagged valid
template <int KIND, int CM>
__device__ void warp_select(const Cand<CM>& mine, Cand<CM>& out) {
  unsigned m = __ballot_sync(kFull, mine.valid);
  out.valid = false;
  while (m) {
    const int l = __ffs(m) - 1;
    m &= m - 1;
    Cand<CM> c;
    c.num.w[0] = __shfl_sync(kFull, mine.num.w[0], l);
    c.num.w[1] = __shfl_sync(kFull, mine.num.w[1], l);
    c.num.w[2] = __shfl_sync(kFull, mine.num.w[2], l);
    c.den = __shfl_sync(kFull, mine.den, l);
    c.key = __shfl_sync(kFull, mine.key, l);
    c.nL = __shfl_sync(kFull, mine.nL, l);
    c.feat = __shfl_sync(kFull, mine.feat, l);
    c.bin = __shfl_sync(kFull, mine.bin, l);
    if (KIND == 1) {
      c.SL = __shfl_sync(kFull, mine.SL, l);
#pragma unroll
      for (int k = 0; k < CM; ++k) c.cL[k] = 0u;
    } else {
      c.SL = 0;
#pragma unroll
      for (int k = 0; k < CM; ++k) c.cL[k] = __shfl_sync(kFull, mine.cL[k], l);
    }
    c.valid = true;
    if (better(c, out)) out = c;
  }
}

// Exact impurity decrease of the chosen split:
//   delta = num/den - A_P/n_P = (num*n_P - A_P*den) / (den*n_P), rounded as
//   RN(numerator) / RN(denominator) in the working precision.
template <int KIND, int CM>
__device__ bool split_delta(const Cand<CM>& c, const NodeInfo<CM>& nd, int C, int precision, double* delta) {
  u128 AP = 0;
  if (KIND == 1) {
    AP = sq_i64(nd.SP);
  } else {
#pragma unroll
    for (int k = 0; k < CM; ++k)
      if (k < C) AP += static_cast<u128>(static_cast<uint64_t>(nd.cp[k]) * nd.cp[k]);
  }
  uint64_t lhs[4], rhs[4];
  mul192x64(c.num, nd.n, lhs);
  mul192x64(u192_from(AP), c.den, rhs);
  if (cmp_limbs4(lhs, rhs) <= 0) return false;
  uint64_t dn[4];
  uint64_t borrow = 0;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const uint64_t a = lhs[i], b = rhs[i];
    const uint64_t t = a - b;
    const uint64_t b1 = a < b;
    dn[i] = t - borrow;
    const uint64_t b2 = t < borrow;
    borrow = b1 | b2;
  }
  const u128 dd = static_cast<u128>(c.den) * nd.n;
  const uint64_t dl[2] = {static_cast<uint64_t>(dd), static_cast<uint64_t>(dd >> 64)};
  if (precision == 0)
    *delta = limbs_to_double(dn, 4, 0) / limbs_to_double(dl, 2, 0);
  else
    *delta = static_cast<double>(__fdiv_rn(limbs_to_float(dn, 4, 0), limbs_to_float(dl, 2, 0)));
  return true;
}

// Records the split of node k (or marks it a leaf); one thread.
template <int KIND, int CM>
__device__ uint32_t commit_split(const Dev& d, uint32_t k, const Cand<CM>& b, const NodeInfo<CM>& nd) {
  double delta = 0.0;
  uint32_t sp = kLeaf;
  if (b.valid && split_delta<KIND, CM>(b, nd, ncls<CM>(d), d.precision, &delta)) {
    sp = (static_cast<uint32_t>(b.feat) << 8) | static_cast<uint32_t>(b.bin);
    d.nd_delta[k] = delta;
    d.nd_ln[k] = b.nL;
    if (KIND == 1) {
      d.nd_lS[k] = b.SL;
    } else {
#pragma unroll
      for (int c = 0; c < CM; ++c)
        if (c < ncls<CM>(d)) d.nd_lcnt[static_cast<int64_t>(k) * d.C + c] = b.cL[c];
    }
    if (!d.permut) {  // Alg. 2: this node's gain x samples, summed exactly per (tree, feature)
      if (!csa_add(d.acc + (static_cast<int64_t>(d.nd_tree[k]) * d.p_aug + b.feat) * kCsaLimbs, delta))
        atomicOr(&d.status[0], kErrAcc);
    }
  }
  d.nd_split[k] = sp;
  return sp;
}

template <int KIND, int CM>
__device__ bool load_node(const Dev& d, uint32_t k, int level, NodeInfo<CM>& nd) {
  const uint32_t tau = d.nd_tree[k];
  nd.base = static_cast<int64_t>(tau) * d.N + d.nd_seg[k];
  nd.len = d.nd_len[k];
  nd.n = d.nd_n[k];
  nd.SP = 0;
  bool pure = false;
#pragma unroll
  for (int c = 0; c < CM; ++c) {
    nd.cp[c] = 0u;
    if (KIND == 0 && c < d.C) {
      nd.cp[c] = d.nd_cnt[static_cast<int64_t>(k) * d.C + c];
      pure |= nd.cp[c] == nd.n;
    }
  }
  if (KIND == 1) nd.SP = d.nd_S[k];
  return level < d.D && nd.len >= 2u && !pure;
}

__device__ __forceinline__ void node_perm(const Dev& d, uint32_t k, Perm& P) {
  perm_init(P, static_cast<uint32_t>(d.p_aug), d.seed, d.nd_heap[k], unit_word(d.t, d.nd_tree[k]),
            purpose_word(kPurposeMtry, d.job));
}

// Stable partition of a node's rows by warp: left rows in order from the
// front, right rows in order from the back (reversed); 8 gathers per lane
// in flight.  Returns the number of left rows.
__device__ uint32_t warp_partition(const Dev& d, int64_t base, uint32_t len, uint32_t sp, const uint32_t* rows_in,
                                   uint32_t* rows_out) {
  const int lane = threadIdx.x & 31;
  const uint8_t* col = column(d, sp >> 8);
  const uint32_t thr = sp & 255u;
  uint32_t lbase = 0, rbase = 0;
  const uint32_t lt = lanemask_lt();
  for (uint32_t r0 = 0; r0 < len; r0 += 256) {
    uint32_t e[8], b[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const uint32_t r = r0 + q * 32 + lane;
      e[q] = r < len ? rows_in[base + r] : 0u;
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const uint32_t r = r0 + q * 32 + lane;
      b[q] = r < len ? col[e[q] >> 8] : 0u;
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const bool v = r0 + q * 32 + lane < len;
      const bool gl = v && b[q] <= thr, gr = v && !gl;
      const unsigned bl = __ballot_sync(kFull, gl), br = __ballot_sync(kFull, gr);
      if (gl) rows_out[base + lbase + __popc(bl & lt)] = e[q];
      if (gr) rows_out[base + len - 1u - (rbase + __popc(br & lt))] = e[q];
      lbase += __popc(bl);
      rbase += __popc(br);
    }
  }
  return lbase;
}

// ============================================================ small nodes
// Bit planes of a small node's rows (one row per lane): the valid lanes, the
// five bits of each row's weight and, per class, the lanes of that class.
template <int CM>
struct SmallPlanes {
  unsigned valid;
  unsigned w[5];
  unsigned y[CM];
};

// A small node's rows sit one per lane in a segment of SEG lanes: the whole
// warp (SEG = 32, nodes of 17..32 rows), a half warp (SEG = 16: two nodes of
// 9..16 rows per warp) or a quarter warp (SEG = 8: four nodes of <= 8 rows).
// Segment helpers: the lanes' mask, and reductions that stay inside the
// segment.
template <int SEG>
__device__ __forceinline__ unsigned seg_mask() {
  return SEG == 32 ? kFull : (((1u << SEG) - 1u) << ((threadIdx.x & 31) & (32 - SEG)));
}

template <int SEG>
__device__ __forceinline__ float seg_max_f(float v) {
#pragma unroll
  for (int off = SEG / 2; off > 0; off >>= 1) v = fmaxf(v, __shfl_xor_sync(kFull, v, off));
  return v;
}

template <int SEG>
__device__ __forceinline__ uint32_t seg_sum_u32(uint32_t v) {
  if constexpr (SEG == 32) {
    return __reduce_add_sync(kFull, v);
  } else {
#pragma unroll
    for (int off = SEG / 2; off > 0; off >>= 1) v += __shfl_xor_sync(kFull, v, off);
    return v;
  }
}

template <int SEG>
__device__ __forceinline__ long long seg_sum_i64(long long v) {
#pragma unroll
  for (int off = SEG / 2; off > 0; off >>= 1) v += __shfl_xor_sync(kFull, v, off);
  return v;
}

// best of the segment's lane candidates flagged valid (all lanes take part;
// each segment walks its own candidates, as many rounds as the busier one)
template <int KIND, int CM, int SEG>
__device__ void seg_select(const Cand<CM>& mine, Cand<CM>& out) {
  if (SEG == 32) {
    warp_select<KIND, CM>(mine, out);
    return;
  }
  unsigned m = __ballot_sync(kFull, mine.valid) & seg_mask<SEG>();
  const int rounds = __reduce_max_sync(kFull, static_cast<unsigned>(__popc(m)));
  out.valid = false;
  for (int r = 0; r < rounds; ++r) {
    const bool have = m != 0u;
    const int l = have ? __ffs(m) - 1 : static_cast<int>(threadIdx.x & 31);
    if (have) m &= m - 1;
    Cand<CM> c;
    c.num.w[0] = __shfl_sync(kFull, mine.num.w[0], l);
    c.num.w[1] = __shfl_sync(kFull, mine.num.w[1], l);
    c.num.w[2] = __shfl_sync(kFull, mine.num.w[2], l);
    c.den = __shfl_sync(kFull, mine.den, l);
    c.key = __shfl_sync(kFull, mine.key, l);
    c.nL = __shfl_sync(kFull, mine.nL, l);
    c.feat = __shfl_sync(kFull, mine.feat, l);
    c.bin = __shfl_sync(kFull, mine.bin, l);
    if (KIND == 1) {
      c.SL = __shfl_sync(kFull, mine.SL, l);
#pragma unroll
      for (int k = 0; k < CM; ++k) c.cL[k] = 0u;
    } else {
      c.SL = 0;
#pragma unroll
      for (int k = 0; k < CM; ++k) c.cL[k] = __shfl_sync(kFull, mine.cL[k], l);
    }
    c.valid = have;
    if (better(c, out)) out = c;
  }
}

// Best split of one feature for a node of <= SEG rows, one row per lane of
// its segment.  Classification: the lanes whose bin is <= this lane's bin
// come from eight ballots over the bin bits (most significant first), and
// the left class counts from population counts against the weight and class
// bit planes.  Regression: the left sums are accumulated over the rows by
// shuffles (rows up to lenmax, the longest node of the warp; lanes past a
// node's rows carry weight 0).  Updates the node's exact best (best) and
// best float score so far (bestf).  Every lane runs every warp-wide step:
// a segment with nothing to contribute goes on with no candidate.
template <int KIND, int CM, int SEG>
__device__ void small_feature(const NodeInfo<CM>& nd, int C, int B, bool v, uint32_t b, uint32_t w, uint32_t y,
                              long long yv, const SmallPlanes<CM>& pl, int feat, uint32_t tkey, float& bestf,
                              Cand<CM>& best, uint32_t lenmax) {
  const unsigned sm = seg_mask<SEG>();
  if (KIND == 1 && B <= 4) {
    // Regression on a column of at most 4 bins: the left sums of each of
    // the <= 3 thresholds come from segment reductions, the same on every
    // lane of the segment.  A threshold whose bin holds no row repeats the
    // partition of a lower one and loses the tie to it.
    float sf[3];
    uint32_t nLt[3];
    long long SLt[3];
    float mx = -1.0f;
#pragma unroll
    for (int t = 0; t < 3; ++t) {
      sf[t] = -1.0f;
      nLt[t] = 0u;
      SLt[t] = 0;
      if (t >= B - 1) break;  // uniform
      const bool in = v && b <= static_cast<uint32_t>(t);
      const uint32_t nl = seg_sum_u32<SEG>(in ? w : 0u);
      const long long sl = seg_sum_i64<SEG>(in ? static_cast<long long>(w) * yv : 0ll);
      nLt[t] = nl;
      SLt[t] = sl;
      if (nl > 0u && nl < nd.n) {
        sf[t] = score_reg_f(sl, nd.SP, nl, nd.n);
        mx = fmaxf(mx, sf[t]);
      }
    }
    if (mx < 0.0f || mx < screen(bestf)) return;  // no warp-wide step follows
    const float thr = screen(fmaxf(mx, bestf));
    bestf = fmaxf(mx, bestf);
#pragma unroll
    for (int t = 0; t < 3; ++t) {
      if (sf[t] < 0.0f || sf[t] < thr) continue;
      Cand<CM> c;
      make_reg<CM>(c, SLt[t], nd.SP, nLt[t], nd.n);
      c.feat = feat;
      c.bin = t;
      c.key = (tkey << 8) | static_cast<uint32_t>(t);
      if (better(c, best)) best = c;
    }
    return;
  }
  uint32_t cl[CM];
#pragma unroll
  for (int k = 0; k < CM; ++k) cl[k] = 0u;
  uint32_t nL = 0;
  long long SL = 0;
  unsigned same;
  if (KIND == 0) {
    unsigned lt = 0u, eq = pl.valid & sm;
#pragma unroll
    for (int t = 7; t >= 0; --t) {
      const unsigned bt = __ballot_sync(kFull, (b >> t) & 1u);
      const bool one = (b >> t) & 1u;
      lt |= one ? (eq & ~bt) : 0u;
      eq &= one ? bt : ~bt;
    }
    const unsigned le = lt | eq;
#pragma unroll
    for (int k = 0; k < CM; ++k)
      if (k < C) {
        const unsigned m = le & pl.y[k];
        uint32_t c = 0;
#pragma unroll
        for (int t = 0; t < 5; ++t) c += static_cast<uint32_t>(__popc(m & pl.w[t])) << t;
        cl[k] = c;
        nL += c;
      }
    same = v ? eq : 0u;
  } else {
    const int base = static_cast<int>(threadIdx.x & 31) & ~(SEG - 1);
    for (int j = 0; j < static_cast<int>(lenmax); ++j) {
      const uint32_t bj = __shfl_sync(kFull, b, base + j), wj = __shfl_sync(kFull, w, base + j);
      const long long yj = __shfl_sync(kFull, yv, base + j);
      if (bj <= b) {  // rows past the node's own carry weight 0
        nL += wj;
        SL += static_cast<long long>(wj) * yj;
      }
    }
    same = __match_any_sync(kFull, v ? b : 0xFFFFFFFFu) & sm;
  }
  // lanes holding the same bin propose the same partition: the lowest one speaks
  const bool ok = v && nL < nd.n && (__ffs(same) - 1) == static_cast<int>(threadIdx.x & 31);
  float sf = -1.0f;
  if (ok) sf = KIND == 1 ? score_reg_f(SL, nd.SP, nL, nd.n) : score_class_f<CM>(cl, nd.cp, C, nL, nd.n);
  const float mx = seg_max_f<SEG>(sf);
  // a feature whose best float score is below the window of the node's best
  // so far cannot hold the node's exact best
  const bool take = !(mx < 0.0f || mx < screen(bestf));
  float thr = 0.0f;
  if (take) {
    thr = screen(fmaxf(mx, bestf));
    bestf = fmaxf(mx, bestf);
  }
  Cand<CM> mine;
  mine.valid = false;
  if (take && ok && sf >= thr) {
    if (KIND == 1)
      make_reg<CM>(mine, SL, nd.SP, nL, nd.n);
    else
      make_class<CM>(mine, cl, nd.cp, C, nL, nd.n);
    mine.feat = feat;
    mine.bin = static_cast<int32_t>(b);
    mine.key = (tkey << 8) | b;
  }
  Cand<CM> c;
  seg_select<KIND, CM, SEG>(mine, c);
  if (take && better(c, best)) best = c;
}

// One thread per node of the level: leaves are marked, active nodes are
// listed as micro (<= 8 rows, in `micro`), tiny (9..16 rows, from the end of
// `small`), small (17..32 rows, from its start) or larger (warp-aggregated
// appends).
template <int KIND, int CM>
__global__ void __launch_bounds__(256) k_classify(Dev d, int level) {
  const int lane = threadIdx.x & 31;
  const uint32_t lcount = d.lvl_cnt[level], loff = d.lvl_off[level];
  for (uint32_t base = (blockIdx.x * blockDim.x + threadIdx.x) & ~31u; base < lcount;
       base += gridDim.x * blockDim.x) {
    const uint32_t idx = base + lane;
    int cls = 0;  // 0 none, 1 small, 2 larger, 3 tiny, 4 micro
    uint32_t k = 0;
    if (idx < lcount) {
      k = loff + idx;
      NodeInfo<CM> nd;
      if (load_node<KIND, CM>(d, k, level, nd))
        cls = nd.len > 32u ? 2 : (nd.len > 16u ? 1 : (nd.len > 8u ? 3 : 4));
      else
        d.nd_split[k] = kLeaf;
    }
    const unsigned ms = __ballot_sync(kFull, cls == 1), mb = __ballot_sync(kFull, cls == 2),
                   mt = __ballot_sync(kFull, cls == 3), mm = __ballot_sync(kFull, cls == 4);
    uint32_t s0 = 0, b0 = 0, t0 = 0, m0 = 0;
    if (lane == 0) {
      if (ms) s0 = atomicAdd(&d.nsmall[level], static_cast<uint32_t>(__popc(ms)));
      if (mb) b0 = atomicAdd(&d.work[level], static_cast<uint32_t>(__popc(mb)));
      if (mt) t0 = atomicAdd(&d.ntiny[level], static_cast<uint32_t>(__popc(mt)));
      if (mm) m0 = atomicAdd(&d.nmicro[level], static_cast<uint32_t>(__popc(mm)));
    }
    s0 = __shfl_sync(kFull, s0, 0);
    b0 = __shfl_sync(kFull, b0, 0);
    t0 = __shfl_sync(kFull, t0, 0);
    m0 = __shfl_sync(kFull, m0, 0);
    if (cls == 1) d.small[s0 + __popc(ms & lanemask_lt())] = k;
    if (cls == 2) d.big[b0 + __popc(mb & lanemask_lt())] = k;
    if (cls == 3) d.small[d.small_cap - 1u - (t0 + __popc(mt & lanemask_lt()))] = k;
    if (cls == 4) d.micro[m0 + __popc(mm & lanemask_lt())] = k;
  }
}

constexpr uint32_t kNoNode = 0xFFFFFFFFu;

// The split of the small node k of this lane's segment (kNoNode: none; its
// lanes still take part in every warp-wide step), its record and partition.
template <int KIND, int CM, int SEG>
__device__ void small_node(const Dev& d, int level, uint32_t k, uint8_t* sbin, unsigned long long& bytes) {
  const int lane = threadIdx.x & 31;
  const int hl = lane & (SEG - 1);
  const uint32_t* rows_in = d.rows[level & 1];
  uint32_t* rows_out = d.rows[(level & 1) ^ 1];
  const int C = ncls<CM>(d);
  const bool has = k != kNoNode;
  NodeInfo<CM> nd;
  nd.base = 0;
  nd.len = 0u;
  nd.n = 0u;
  nd.SP = 0;
#pragma unroll
  for (int c = 0; c < CM; ++c) nd.cp[c] = 0u;
  Perm P;
  if (has) {
    load_node<KIND, CM>(d, k, level, nd);
    node_perm(d, k, P);
  }
  const bool v = hl < static_cast<int>(nd.len);
  const uint32_t e = v ? rows_in[nd.base + hl] : 0u;
  const uint32_t row = e >> 8, w = v ? ent_w<KIND>(e) : 0u;
  const uint32_t y = KIND == 0 ? ent_y(e) : 0u;
  const long long yv = (KIND == 1 && v) ? d.yreg[row] : 0ll;
  SmallPlanes<CM> pl;
  pl.valid = __ballot_sync(kFull, v);
#pragma unroll
  for (int t = 0; t < 5; ++t) pl.w[t] = __ballot_sync(kFull, (w >> t) & 1u);
#pragma unroll
  for (int c = 0; c < CM; ++c) pl.y[c] = __ballot_sync(kFull, v && y == static_cast<uint32_t>(c));
  const uint32_t lenmax = SEG == 32 ? nd.len : __reduce_max_sync(kFull, nd.len);
  Cand<CM> best;
  best.valid = false;
  float bestf = -1.0f;
  for (int r0 = 0; r0 < d.mtry; r0 += SEG) {
    const int ns = min(SEG, d.mtry - r0);
    const uint32_t myf = (has && hl < ns) ? perm_apply(P, static_cast<uint32_t>(r0 + hl)) : 0u;
    for (int j0 = 0; j0 < ns; j0 += kSmallAhead) {
      // the row's bins of the next kSmallAhead features, all loads in
      // flight at once (the shuffles run on all lanes, outside the per-lane
      // conditions), parked in the warp's shared memory
      uint32_t bv[kSmallAhead];
#pragma unroll
      for (int u = 0; u < kSmallAhead; ++u) {
        const uint32_t fu = __shfl_sync(kFull, myf, min(j0 + u, ns - 1), SEG);
        bv[u] = (v && j0 + u < ns) ? row_bin(d, row, fu) : 0u;
      }
      __syncwarp();
#pragma unroll
      for (int u = 0; u < kSmallAhead; ++u) sbin[u * 32 + lane] = static_cast<uint8_t>(bv[u]);
      __syncwarp();
      const int nu = min(kSmallAhead, ns - j0);
      for (int u = 0; u < nu; ++u) {
        const uint32_t f = __shfl_sync(kFull, myf, j0 + u, SEG);
        const uint32_t tkey = d.tie_break == 1 ? static_cast<uint32_t>(r0 + j0 + u) : f;
        small_feature<KIND, CM, SEG>(nd, C, d.B, v, sbin[u * 32 + lane], w, y, yv, pl, static_cast<int>(f), tkey,
                                     bestf, best, lenmax);
      }
    }
  }
  uint32_t sp = kLeaf;
  if (has && hl == 0) sp = commit_split<KIND, CM>(d, k, best, nd);
  sp = __shfl_sync(kFull, sp, 0, SEG);
  if (has && hl == 0) bytes += static_cast<unsigned long long>(nd.len) * (d.mtry + 4ull + (KIND ? 8ull : 0ull));
  // stable partition: left rows in order, then right rows in order
  const bool split = has && sp != kLeaf;
  const uint32_t bs = (v && split) ? row_bin(d, row, sp >> 8) : 0u;
  const bool gl = v && split && bs <= (sp & 255u), gr = v && split && !gl;
  const unsigned sm = seg_mask<SEG>();
  const unsigned bl = __ballot_sync(kFull, gl) & sm, br = __ballot_sync(kFull, gr) & sm;
  const uint32_t nl = __popc(bl);
  if (gl) rows_out[nd.base + __popc(bl & lanemask_lt())] = e;
  if (gr) rows_out[nd.base + nl + __popc(br & lanemask_lt())] = e;
  if (split && hl == 0) {
    d.nd_lrows[k] = nl;
    bytes += static_cast<unsigned long long>(nd.len) * 5ull;
  }
}

// SEG = 8: one warp per four micro nodes (a quarter warp each); SEG = 16:
// one warp per pair of tiny nodes (a half warp each); SEG = 32: one warp per
// small node.
template <int KIND, int CM, int SEG>
__global__ void __launch_bounds__(256, BORUTA_SMALL_MINB) k_split_small(Dev d, int level) {
  __shared__ uint8_t sbins[8][kSmallAhead * 32];
  const int lane = threadIdx.x & 31;
  uint8_t* sbin = sbins[threadIdx.x >> 5];
  const uint32_t gwarp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
  unsigned long long bytes = 0;
  if (SEG == 8) {
    const uint32_t nm = d.nmicro[level], nquads = (nm + 3u) / 4u;
    for (uint32_t idx = gwarp; idx < nquads; idx += nwarps) {
      const uint32_t t = 4u * idx + static_cast<uint32_t>(lane >> 3);
      const uint32_t k = t < nm ? d.micro[t] : kNoNode;
      small_node<KIND, CM, SEG>(d, level, k, sbin, bytes);
    }
  } else if (SEG == 16) {
    const uint32_t nt = d.ntiny[level], npairs = (nt + 1u) / 2u;
    for (uint32_t idx = gwarp; idx < npairs; idx += nwarps) {
      const uint32_t t = 2u * idx + static_cast<uint32_t>(lane >> 4);
      const uint32_t k = t < nt ? d.small[d.small_cap - 1u - t] : kNoNode;
      small_node<KIND, CM, SEG>(d, level, k, sbin, bytes);
    }
  } else {
    const uint32_t ns_nodes = d.nsmall[level];
    for (uint32_t idx = gwarp; idx < ns_nodes; idx += nwarps) small_node<KIND, CM, SEG>(d, level, d.small[idx], sbin, bytes);
  }
  if (bytes) atomicAdd(&d.counters[0], bytes);
}

// ============================================================ larger nodes
template <int KIND>
__device__ __forceinline__ void hist_clear(const Dev& d, uint32_t* hw) {
  const int lane = threadIdx.x & 31;
  const int C = d.C, B = d.B;
  if (KIND == 0) {
    const int vecs = static_cast<int>(hist_smem_per_warp(0, C, B) / 16);  // either layout, whole
    for (int i = lane; i < vecs; i += 32) reinterpret_cast<uint4*>(hw)[i] = make_uint4(0u, 0u, 0u, 0u);
  } else {
    uint32_t* hn = hw;
    unsigned long long* hs = reinterpret_cast<unsigned long long*>(hw + hist_words_n(B));
    for (int i = lane; i < B + (B >> 3) + 1; i += 32) {
      hn[i] = 0u;
      hs[i] = 0ull;
    }
  }
}

// Adds up to 32 * kBatch rows, entries already in registers (entry q of
// lane l is row r0 + q * 32 + l of the node), to the warp's histogram.
// Columns with at most 4 bins (e.g. genotypes): each lane keeps its rows'
// weights (per class for two classes) and weighted targets per bin in
// registers, and the warp totals are written to the histogram at the end --
// no shared-memory atomics, which would serialise on the few addresses.
__device__ __forceinline__ bool regs4(const Dev& d, int kind) { return d.B <= 4 && (kind == 1 || d.C <= 2); }

template <int KIND>
__device__ __forceinline__ void regs4_add(uint32_t b, uint32_t e, bool valid, long long yv, uint32_t (&c0)[4],
                                          uint32_t (&c1)[4], long long (&sy)[4]) {
  const uint32_t w = valid ? ent_w<KIND>(e) : 0u;
  const bool one = KIND == 0 && ent_y(e) != 0u;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const uint32_t add = b == static_cast<uint32_t>(k) ? w : 0u;
    if (KIND == 0) {
      c0[k] += one ? 0u : add;
      c1[k] += one ? add : 0u;
    } else {
      c0[k] += add;
      sy[k] += static_cast<long long>(add) * yv;
    }
  }
}

template <int KIND>
__device__ __forceinline__ void regs4_store(const Dev& d, uint32_t* hw, const uint32_t (&c0)[4],
                                            const uint32_t (&c1)[4], const long long (&sy)[4]) {
  const int lane = threadIdx.x & 31;
  __syncwarp();
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    if (k >= d.B) break;  // uniform
    const uint32_t t0 = __reduce_add_sync(kFull, c0[k]);
    if (KIND == 0) {
      const uint32_t t1 = __reduce_add_sync(kFull, c1[k]);
      if (lane == 0) {
        hw[k * d.C] = t0;  // bin k < 8: no padding word before it
        if (d.C == 2) hw[k * d.C + 1] = t1;
      }
    } else {
      long long v = sy[k];
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(kFull, v, off);
      if (lane == 0) {
        hw[k] = t0;
        reinterpret_cast<long long*>(hw + hist_words_n(d.B))[k] = v;
      }
    }
  }
  __syncwarp();
}

template <int KIND, int kBatch>
__device__ __forceinline__ void hist_add(const Dev& d, uint32_t r0, uint32_t len, const uint32_t (&e)[kBatch],
                                         const uint8_t* col, uint32_t* hw) {
  const int lane = threadIdx.x & 31;
  const int C = d.C, B = d.B;
  uint32_t b[kBatch];
  const uint64_t pol = keep_policy();
#pragma unroll
  for (int q = 0; q < kBatch; ++q) {
    const uint32_t r = r0 + q * 32 + lane;
    b[q] = r < len ? ld_keep(col + (e[q] >> 8), pol) : 0u;
  }
  if (KIND == 0) {
#pragma unroll
    for (int q = 0; q < kBatch; ++q)
      if (r0 + q * 32 + lane < len) atomicAdd(&hw[b[q] * C + ent_y(e[q]) + (b[q] >> 3)], ent_w<0>(e[q]));
  } else {
    uint32_t* hn = hw;
    unsigned long long* hs = reinterpret_cast<unsigned long long*>(hw + hist_words_n(B));
    long long yq[kBatch];
#pragma unroll
    for (int q = 0; q < kBatch; ++q) {
      const uint32_t r = r0 + q * 32 + lane;
      yq[q] = r < len ? d.yreg[e[q] >> 8] : 0ll;
    }
#pragma unroll
    for (int q = 0; q < kBatch; ++q)
      if (r0 + q * 32 + lane < len) {
        const uint32_t w = ent_w<1>(e[q]);
        atomicAdd(&hn[b[q] + (b[q] >> 3)], w);
        atomicAdd(&hs[b[q] + (b[q] >> 3)], static_cast<unsigned long long>(static_cast<long long>(w) * yq[q]));
      }
  }
}

// Warp-private histogram of one feature over a node's rows.  Rows are
// gathered BORUTA_STREAM_BATCH per lane per pass so that as many independent
// loads per lane are in flight.
// kClear: clear the histogram first (false: it is known to be zero).
template <int KIND, bool kClear = true>
__device__ void build_hist(const Dev& d, int64_t base, uint32_t len, const uint32_t* rows, const uint8_t* col,
                           uint32_t* hw) {
  const int lane = threadIdx.x & 31;
  constexpr int kBatch = BORUTA_STREAM_BATCH;
  if (regs4(d, KIND)) {
    uint32_t c0[4] = {0u, 0u, 0u, 0u}, c1[4] = {0u, 0u, 0u, 0u};
    long long sy[4] = {0, 0, 0, 0};
    const uint64_t pol = keep_policy();
    for (uint32_t r0 = 0; r0 < len; r0 += 32 * kBatch) {
      uint32_t e[kBatch], b[kBatch];
#pragma unroll
      for (int q = 0; q < kBatch; ++q) {
        const uint32_t r = r0 + q * 32 + lane;
        e[q] = r < len ? ld_stream(rows + base + r) : 0u;
      }
#pragma unroll
      for (int q = 0; q < kBatch; ++q) b[q] = r0 + q * 32 + lane < len ? ld_keep(col + (e[q] >> 8), pol) : 0u;
#pragma unroll
      for (int q = 0; q < kBatch; ++q) {
        const bool v = r0 + q * 32 + lane < len;
        regs4_add<KIND>(b[q], e[q], v, (KIND == 1 && v) ? d.yreg[e[q] >> 8] : 0ll, c0, c1, sy);
      }
    }
    regs4_store<KIND>(d, hw, c0, c1, sy);
    return;
  }
  if (kClear) hist_clear<KIND>(d, hw);
  uint32_t e[kBatch];
#pragma unroll
  for (int q = 0; q < kBatch; ++q) {
    const uint32_t r = q * 32 + lane;
    e[q] = r < len ? ld_stream(rows + base + r) : 0u;
  }
  __syncwarp();
  for (uint32_t r0 = 0; r0 < len; r0 += 32 * kBatch) {
    if (r0 > 0) {
#pragma unroll
      for (int q = 0; q < kBatch; ++q) {
        const uint32_t r = r0 + q * 32 + lane;
        e[q] = r < len ? ld_stream(rows + base + r) : 0u;
      }
    }
    hist_add<KIND, kBatch>(d, r0, len, e, col, hw);
  }
  __syncwarp();
}

// Float pre-screen of a built histogram.  Lane l owns bins [l*bpl,
// (l+1)*bpl).  An empty bin repeats the partition of the nearest non-empty
// bin below it, which has the lower bin and wins the tie, so empty bins are
// skipped: a lane visits only its non-empty bins (a bit mask), and keeps its
// best float score with that bin's left totals, and its second-best score.
template <int CM>
struct Screen {
  uint32_t pre[CM];  // left totals before the lane's bins (regression: count)
  long long ps;      // regression: target sum before the lane's bins
  uint32_t mask;     // non-empty bins of the lane that can be thresholds
  float lmax, s2;    // best and second-best float score (-1: none)
  int bbest;         // bin of lmax
  uint32_t nLb;      // left count at bbest
  uint32_t cb[CM];   // class: left class counts at bbest
  long long SLb;     // regression: left target sum at bbest
};

template <int CM>
__device__ __forceinline__ void screen_keep(Screen<CM>& S, float sc, int bb, uint32_t nL, const uint32_t* cum,
                                            long long SL) {
  if (sc > S.lmax) {
    S.s2 = S.lmax;
    S.lmax = sc;
    S.bbest = bb;
    S.nLb = nL;
#pragma unroll
    for (int k = 0; k < CM; ++k) S.cb[k] = cum[k];
    S.SLb = SL;
  } else if (sc > S.s2) {
    S.s2 = sc;
  }
}

// occ: the lane's bins that may be non-empty (bit q: bin b0 + q); the others
// are known to be empty and are not read.
template <int KIND, int CM>
__device__ __forceinline__ void scan_screen(const Dev& d, const NodeInfo<CM>& nd, const uint32_t* hw, Screen<CM>& S,
                                            uint32_t occ = 0xFFu) {
  const int lane = threadIdx.x & 31;
  const int C = ncls<CM>(d), B = d.B;
  const int bpl = (B + 31) >> 5;  // bins per lane (<= 8)
  const int b0 = lane * bpl;
  S.mask = 0u;
  S.lmax = -1.0f;
  S.s2 = -1.0f;
  S.bbest = 0;
  S.nLb = 0u;
  S.SLb = 0;
  S.ps = 0;
  if (KIND == 0) {
    uint32_t cum[CM];
#pragma unroll
    for (int k = 0; k < CM; ++k) {
      S.pre[k] = 0u;
      S.cb[k] = 0u;
    }
    for (uint32_t m = occ & ((1u << bpl) - 1u); m; m &= m - 1) {
      const int q = __ffs(m) - 1;
      const int bb = b0 + q;
      if (bb < B) {
        uint32_t wb = 0;
#pragma unroll
        for (int k = 0; k < CM; ++k)
          if (k < C) {
            const uint32_t h = hw[bb * C + k + (bb >> 3)];
            S.pre[k] += h;
            wb += h;
          }
        if (wb > 0u && bb < B - 1) S.mask |= 1u << q;
      }
    }
#pragma unroll
    for (int k = 0; k < CM; ++k) {
      S.pre[k] = warp_excl_scan_u32(S.pre[k], lane);
      cum[k] = S.pre[k];
    }
    for (uint32_t m = S.mask; m; m &= m - 1) {
      const int bb = b0 + __ffs(m) - 1;
      uint32_t nL = 0;
#pragma unroll
      for (int k = 0; k < CM; ++k)
        if (k < C) {
          cum[k] += hw[bb * C + k + (bb >> 3)];
          nL += cum[k];
        }
      if (nL < nd.n) screen_keep<CM>(S, score_class_f<CM>(cum, nd.cp, C, nL, nd.n), bb, nL, cum, 0);
    }
  } else {
    const uint32_t* hn = hw;
    const unsigned long long* hs = reinterpret_cast<const unsigned long long*>(hw + hist_words_n(B));
    uint32_t tn = 0;
    long long ts = 0;
#pragma unroll
    for (int k = 0; k < CM; ++k) S.cb[k] = 0u;
    for (uint32_t m = occ & ((1u << bpl) - 1u); m; m &= m - 1) {
      const int q = __ffs(m) - 1;
      const int bb = b0 + q;
      if (bb < B) {
        const uint32_t h = hn[bb + (bb >> 3)];
        tn += h;
        ts += static_cast<long long>(hs[bb + (bb >> 3)]);
        if (h > 0u && bb < B - 1) S.mask |= 1u << q;
      }
    }
    S.pre[0] = warp_excl_scan_u32(tn, lane);
    S.ps = warp_excl_scan_i64(ts, lane);
    uint32_t cn = S.pre[0];
    long long cs = S.ps;
    for (uint32_t m = S.mask; m; m &= m - 1) {
      const int bb = b0 + __ffs(m) - 1;
      cn += hn[bb + (bb >> 3)];
      cs += static_cast<long long>(hs[bb + (bb >> 3)]);
      if (cn < nd.n) screen_keep<CM>(S, score_reg_f(cs, nd.SP, cn, nd.n), bb, cn, S.cb, cs);
    }
  }
}

// Exact best among the candidates whose float score is at least thr (all
// lanes; only a lane whose own best is inside the window revisits its bins).
template <int KIND, int CM>
__device__ void scan_exact(int C, int B, const NodeInfo<CM>& nd, const uint32_t* hw, const Screen<CM>& S, float thr,
                           int feat, uint32_t tkey, Cand<CM>& out) {
  const int lane = threadIdx.x & 31;
  const int b0 = lane * ((B + 31) >> 5);
  Cand<CM> mine;
  mine.valid = false;
  if (S.lmax >= thr) {
    if (KIND == 0) {
      uint32_t cum[CM];
#pragma unroll
      for (int k = 0; k < CM; ++k) cum[k] = S.pre[k];
      for (uint32_t m = S.mask; m; m &= m - 1) {
        const int bb = b0 + __ffs(m) - 1;
        uint32_t nL = 0;
#pragma unroll
        for (int k = 0; k < CM; ++k)
          if (k < C) {
            cum[k] += hw[bb * C + k + (bb >> 3)];
            nL += cum[k];
          }
        if (nL < nd.n && score_class_f<CM>(cum, nd.cp, C, nL, nd.n) >= thr) {
          Cand<CM> c;
          make_class<CM>(c, cum, nd.cp, C, nL, nd.n);
          c.feat = feat;
          c.bin = bb;
          c.key = (tkey << 8) | static_cast<uint32_t>(bb);
          if (better(c, mine)) mine = c;
        }
      }
    } else {
      const uint32_t* hn = hw;
      const unsigned long long* hs = reinterpret_cast<const unsigned long long*>(hw + hist_words_n(B));
      uint32_t cn = S.pre[0];
      long long cs = S.ps;
      for (uint32_t m = S.mask; m; m &= m - 1) {
        const int bb = b0 + __ffs(m) - 1;
        cn += hn[bb + (bb >> 3)];
        cs += static_cast<long long>(hs[bb + (bb >> 3)]);
        if (cn < nd.n && score_reg_f(cs, nd.SP, cn, nd.n) >= thr) {
          Cand<CM> c;
          make_reg<CM>(c, cs, nd.SP, cn, nd.n);
          c.feat = feat;
          c.bin = bb;
          c.key = (tkey << 8) | static_cast<uint32_t>(bb);
          if (better(c, mine)) mine = c;
        }
      }
    }
  }
  warp_select<KIND, CM>(mine, out);
}

// Scan of a built histogram: returns the warp's best float score (-1 if no
// valid candidate) and in `out` the feature's exact best candidate (all
// lanes).  The float screen keeps every candidate whose exact score is the
// maximum, and only those are compared exactly.
template <int KIND, int CM>
__device__ float scan_hist(const Dev& d, const NodeInfo<CM>& nd, const uint32_t* hw, bool exact, int feat,
                           uint32_t tkey, Cand<CM>& out) {
  Screen<CM> S;
  scan_screen<KIND, CM>(d, nd, hw, S);
  const float mx = warp_max_f(S.lmax);
  out.valid = false;
  if (!exact || mx < 0.0f) return mx;
  scan_exact<KIND, CM>(ncls<CM>(d), d.B, nd, hw, S, screen(mx), feat, tkey, out);
  return mx;
}

template <int KIND, int CM>
__device__ void dense_feature(const Dev& d, const NodeInfo<CM>& nd, const uint32_t* rows, int feat, uint32_t tkey,
                              uint32_t* hw, Cand<CM>& out) {
  build_hist<KIND>(d, nd.base, nd.len, rows, column(d, static_cast<uint32_t>(feat)), hw);
  scan_hist<KIND, CM>(d, nd, hw, true, feat, tkey, out);
}

__device__ __forceinline__ bool band_path(const Dev& d, uint32_t) { return d.band_w > 0; }

// The band path runs the level's larger nodes in chunks of chunk_cap nodes
// (their items fill the plan buffers at most); this launch's chunk starts at
// chunk0.  Returns the number of nodes of the chunk (0: nothing to do).
__device__ __forceinline__ uint32_t chunk_nodes(const Dev& d, int level) {
  const uint32_t nbig = d.work[level];
  if (d.band_w == 0 || d.chunk0 >= nbig) return 0u;
  return min(nbig - d.chunk0, d.chunk_cap);
}

// A feature's exact best candidate, kept as the integers that define it:
// the node's totals turn them back into the exact score.
template <int CM>
struct PackedCand {
  uint32_t fb;  // feature << 8 | bin, or kLeaf when the feature has no valid split
  uint32_t nL;
  uint32_t cL[CM > 1 ? CM : 2];  // class counts, or the target sum's two halves
};

template <int KIND, int CM>
__device__ __forceinline__ PackedCand<CM> pack_cand(const Cand<CM>& c) {
  PackedCand<CM> p;
  p.fb = c.valid ? ((static_cast<uint32_t>(c.feat) << 8) | static_cast<uint32_t>(c.bin)) : kLeaf;
  p.nL = c.nL;
  if (KIND == 1) {
    p.cL[0] = static_cast<uint32_t>(static_cast<unsigned long long>(c.SL));
    p.cL[1] = static_cast<uint32_t>(static_cast<unsigned long long>(c.SL) >> 32);
  } else {
#pragma unroll
    for (int k = 0; k < CM; ++k) p.cL[k] = c.cL[k];
  }
  return p;
}

template <int KIND, int CM>
__device__ __forceinline__ void unpack_cand(const PackedCand<CM>& p, const NodeInfo<CM>& nd, int C, uint32_t tkey,
                                            Cand<CM>& c) {
  c.valid = false;
  if (p.fb == kLeaf) return;
  if (KIND == 1) {
    const long long SL = static_cast<long long>(static_cast<unsigned long long>(p.cL[0]) |
                                                (static_cast<unsigned long long>(p.cL[1]) << 32));
    make_reg<CM>(c, SL, nd.SP, p.nL, nd.n);
  } else {
    make_class<CM>(c, p.cL, nd.cp, C, p.nL, nd.n);
  }
  c.feat = static_cast<int32_t>(p.fb >> 8);
  c.bin = static_cast<int32_t>(p.fb & 255u);
  c.key = (tkey << 8) | (p.fb & 255u);
}

// The exact comparison of scan_pack when several candidates lie inside the
// screen window: rare, so kept out of line (arguments by value).
template <int KIND, int CM>
__device__ __noinline__ void scan_exact_pack(int C, int B, const NodeInfo<CM> nd, const uint32_t* hw,
                                             const Screen<CM> S, float thr, uint32_t f, PackedCand<CM>* dst) {
  Cand<CM> c;
  scan_exact<KIND, CM>(C, B, nd, hw, S, thr, static_cast<int>(f), 0u, c);
  if ((threadIdx.x & 31) == 0) *dst = pack_cand<KIND, CM>(c);
}

// A feature's exact best candidate, packed, from its built histogram.  When
// a single candidate lies inside the float screen window it is the exact
// best and is packed as is; otherwise the candidates inside the window are
// compared exactly.
template <int KIND, int CM>
__device__ void scan_pack(const Dev& d, const NodeInfo<CM>& nd, const uint32_t* hw, uint32_t f, PackedCand<CM>* dst,
                          uint32_t occ = 0xFFu) {
  const int lane = threadIdx.x & 31;
  Screen<CM> S;
  scan_screen<KIND, CM>(d, nd, hw, S, occ);
  const float mx = warp_max_f(S.lmax);
  if (mx < 0.0f) {
    if (lane == 0) {
      PackedCand<CM> p;
      p.fb = kLeaf;
      p.nL = 0u;
#pragma unroll
      for (int k = 0; k < (CM > 1 ? CM : 2); ++k) p.cL[k] = 0u;
      *dst = p;
    }
    return;
  }
  const float thr = screen(mx);
  const uint32_t mine = (S.lmax >= thr ? 1u : 0u) + (S.s2 >= thr ? 1u : 0u);
  if (__reduce_add_sync(kFull, mine) == 1u) {
    if (mine) {
      PackedCand<CM> p;
      p.fb = (f << 8) | static_cast<uint32_t>(S.bbest);
      p.nL = S.nLb;
      if (KIND == 1) {
        p.cL[0] = static_cast<uint32_t>(static_cast<unsigned long long>(S.SLb));
        p.cL[1] = static_cast<uint32_t>(static_cast<unsigned long long>(S.SLb) >> 32);
      } else {
#pragma unroll
        for (int k = 0; k < CM; ++k) p.cL[k] = S.cb[k];
      }
      *dst = p;
    }
  } else {
    scan_exact_pack<KIND, CM>(ncls<CM>(d), d.B, nd, hw, S, thr, f, dst);
  }
}

// ---- packed class histograms
// A classification node of at most five classes whose total weight is below
// 4096 keeps all class weights of a bin in one 64-bit word, 12 bits per
// class (class k in bits 12k .. 12k+11).  Every partial sum of a bin or of a
// prefix of bins is at most the node's total weight, so no field carries into
// the next: one shared-memory add, load, scan step or store moves all the
// classes of a bin.  Staged nodes (at most kRegRows rows of bootstrap count
// below 32) always qualify.
constexpr int kPkBits = 12;
constexpr uint32_t kPkLimit = 1u << kPkBits;

template <int KIND, int CM>
__device__ __forceinline__ bool packed_ok(const Dev& d, const NodeInfo<CM>& nd) {
  return KIND == 0 && CM <= 5 && !regs4(d, 0) && nd.n < kPkLimit;
}

// class weights of a packed word; returns their sum
template <int CM>
__device__ __forceinline__ uint32_t pk_unpack(unsigned long long v, uint32_t (&c)[CM], int C) {
  uint32_t n = 0u;
#pragma unroll
  for (int k = 0; k < CM; ++k) {
    c[k] = k < C ? static_cast<uint32_t>(v >> (kPkBits * k)) & (kPkLimit - 1u) : 0u;
    n += c[k];
  }
  return n;
}

__device__ __forceinline__ unsigned long long pk_entry(uint32_t e) {
  return static_cast<unsigned long long>(ent_w<0>(e)) << (kPkBits * ent_y(e));
}

// Adds up to 32 * kBatch rows (entries in registers) to a packed histogram.
template <int kBatch>
__device__ __forceinline__ void hist_add_pk(uint32_t r0, uint32_t len, const uint32_t (&e)[kBatch],
                                            const uint8_t* col, unsigned long long* hp) {
  const int lane = threadIdx.x & 31;
  uint32_t b[kBatch];
  const uint64_t pol = keep_policy();
#pragma unroll
  for (int q = 0; q < kBatch; ++q) {
    const uint32_t r = r0 + q * 32 + lane;
    b[q] = r < len ? ld_keep(col + (e[q] >> 8), pol) : 0u;
  }
#pragma unroll
  for (int q = 0; q < kBatch; ++q)
    if (r0 + q * 32 + lane < len) atomicAdd(&hp[b[q] + (b[q] >> 3)], pk_entry(e[q]));
}

// Packed histogram of one feature over a node's rows, streamed from the row
// buffer (the histogram is zero on entry).
__device__ void build_hist_pk(int64_t base, uint32_t len, const uint32_t* rows, const uint8_t* col,
                              unsigned long long* hp) {
  const int lane = threadIdx.x & 31;
  constexpr int kBatch = BORUTA_STREAM_BATCH;
  for (uint32_t r0 = 0; r0 < len; r0 += 32 * kBatch) {
    uint32_t e[kBatch];
#pragma unroll
    for (int q = 0; q < kBatch; ++q) {
      const uint32_t r = r0 + q * 32 + lane;
      e[q] = r < len ? ld_stream(rows + base + r) : 0u;
    }
    hist_add_pk<kBatch>(r0, len, e, col, hp);
  }
  __syncwarp();
}

// Packed histogram of one feature over a staged node (entries in ebuf, the
// feature's bins gathered into b; the histogram is zero on entry).
__device__ __forceinline__ void hist_staged_pk(uint32_t len, const uint32_t* ebuf, const uint32_t (&b)[kRegRows / 32],
                                               unsigned long long* hp) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int q = 0; q < static_cast<int>(kRegRows / 32); ++q) {
    const uint32_t r = q * 32 + lane;
    if (r < len) atomicAdd(&hp[b[q] + (b[q] >> 3)], pk_entry(ebuf[r]));
  }
  __syncwarp();
}

// Exact best among a packed histogram's candidates whose float score is at
// least thr (several lie inside the screen window: rare, so kept out of line).
// cand: the lane's candidate bins to revisit; pre: the warp prefix before them.
// (Arguments by value: nothing of the caller's state has to live in memory.)
template <int CM>
__device__ __noinline__ void pk_exact(int C, int B, const NodeInfo<CM> nd, const unsigned long long* hp,
                                      unsigned long long pre, uint32_t cand, float thr, uint32_t f,
                                      PackedCand<CM>* dst) {
  const int lane = threadIdx.x & 31;
  const int b0 = lane * ((B + 31) >> 5);
  Cand<CM> best;
  best.valid = false;
  unsigned long long cum = pre;
  for (uint32_t m = cand; m; m &= m - 1) {
    const int bb = b0 + __ffs(m) - 1;
    cum += hp[bb + (bb >> 3)];
    uint32_t cl[CM];
    const uint32_t nL = pk_unpack<CM>(cum, cl, C);
    if (nL < nd.n && score_class_f<CM>(cl, nd.cp, C, nL, nd.n) >= thr) {
      Cand<CM> c;
      make_class<CM>(c, cl, nd.cp, C, nL, nd.n);
      c.feat = static_cast<int32_t>(f);
      c.bin = bb;
      c.key = static_cast<uint32_t>(bb);
      if (better(c, best)) best = c;
    }
  }
  Cand<CM> c;
  warp_select<0, CM>(best, c);
  if (lane == 0) *dst = pack_cand<0, CM>(c);
}

// scan_pack over a packed histogram, which it leaves zero.  Lane l owns bins
// [l*bpl, (l+1)*bpl) as in scan_screen: it reads them all at once, scans
// the warp's totals once for all classes, and scores only its non-empty
// bins below the last (an empty bin repeats the partition of the nearest
// non-empty bin below it, which wins the tie).
template <int CM>
__device__ void scan_pack_pk(const Dev& d, const NodeInfo<CM>& nd, unsigned long long* hp, uint32_t f,
                             PackedCand<CM>* dst) {
  const int lane = threadIdx.x & 31;
  const int C = ncls<CM>(d), B = d.B;
  const int bpl = (B + 31) >> 5;  // <= 8
  const int b0 = lane * bpl;
  uint32_t nz = 0u, cand = 0u;
  unsigned long long tot = 0ull;
  {
    unsigned long long v[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int bb = b0 + q;
      v[q] = (q < bpl && bb < B) ? hp[bb + (bb >> 3)] : 0ull;
    }
#pragma unroll
    for (int q = 0; q < 8; ++q)
      if (v[q] != 0ull) {
        nz |= 1u << q;
        tot += v[q];
        if (b0 + q < B - 1) cand |= 1u << q;
      }
  }
  const unsigned long long pre = static_cast<unsigned long long>(warp_excl_scan_i64(static_cast<long long>(tot), lane));
  float lmax = -1.0f, s2 = -1.0f;
  int bbest = 0;
  unsigned long long cbest = 0ull, cum = pre;
  for (uint32_t m = cand; m; m &= m - 1) {
    const int bb = b0 + __ffs(m) - 1;
    cum += hp[bb + (bb >> 3)];
    uint32_t cl[CM];
    const uint32_t nL = pk_unpack<CM>(cum, cl, C);
    if (nL < nd.n) {
      const float sc = score_class_f<CM>(cl, nd.cp, C, nL, nd.n);
      if (sc > lmax) {
        s2 = lmax;
        lmax = sc;
        bbest = bb;
        cbest = cum;
      } else if (sc > s2) {
        s2 = sc;
      }
    }
  }
  const float mx = warp_max_f(lmax);
  if (mx < 0.0f) {
    if (lane == 0) {
      PackedCand<CM> p;
      p.fb = kLeaf;
      p.nL = 0u;
#pragma unroll
      for (int k = 0; k < CM; ++k) p.cL[k] = 0u;
      *dst = p;
    }
  } else {
    const float thr = screen(mx);
    const uint32_t mine = (lmax >= thr ? 1u : 0u) + (s2 >= thr ? 1u : 0u);
    if (__reduce_add_sync(kFull, mine) == 1u) {
      if (mine) {  // the only candidate inside the window is the exact best
        PackedCand<CM> p;
        uint32_t cl[CM];
        p.fb = (f << 8) | static_cast<uint32_t>(bbest);
        p.nL = pk_unpack<CM>(cbest, cl, C);
#pragma unroll
        for (int k = 0; k < CM; ++k) p.cL[k] = cl[k];
        *dst = p;
      }
    } else {
      pk_exact<CM>(C, B, nd, hp, pre, lmax >= thr ? cand : 0u, thr, f, dst);
    }
  }
  for (uint32_t m = nz; m; m &= m - 1) {  // each lane clears its own bins, after its own reads
    const int bb = b0 + __ffs(m) - 1;
    hp[bb + (bb >> 3)] = 0ull;
  }
  __syncwarp();
}

// Histogram of one feature over a node of at most kRegRows rows whose entries
// are staged in the warp's shared memory (ebuf), the feature's bins already
// gathered into b (lane l holds rows q * 32 + l).
// The histogram is all zero on entry (the staged path leaves it so, see
// hist_unstage); the bins that receive rows are marked in occ.
template <int KIND>
__device__ __forceinline__ void hist_staged(const Dev& d, uint32_t len, const uint32_t* ebuf,
                                            const uint32_t (&b)[kRegRows / 32], uint32_t* hw, uint32_t* occ,
                                            bool mark) {
  const int lane = threadIdx.x & 31;
  if (regs4(d, KIND)) {
    if (lane == 0 && mark) occ[0] = (1u << d.B) - 1u;  // regs4_store writes bins 0..B-1
    uint32_t c0[4] = {0u, 0u, 0u, 0u}, c1[4] = {0u, 0u, 0u, 0u};
    long long sy[4] = {0, 0, 0, 0};
#pragma unroll
    for (int q = 0; q < static_cast<int>(kRegRows / 32); ++q) {
      const uint32_t r = q * 32 + lane;
      const bool v = r < len;
      const uint32_t e = v ? ebuf[r] : 0u;
      regs4_add<KIND>(b[q], e, v, (KIND == 1 && v) ? d.yreg[e >> 8] : 0ll, c0, c1, sy);
    }
    regs4_store<KIND>(d, hw, c0, c1, sy);
    return;
  }
  if (KIND == 0) {
#pragma unroll
    for (int q = 0; q < static_cast<int>(kRegRows / 32); ++q) {
      const uint32_t r = q * 32 + lane;
      if (r < len) {
        const uint32_t e = ebuf[r];
        atomicAdd(&hw[b[q] * d.C + ent_y(e) + (b[q] >> 3)], ent_w<0>(e));
        if (mark) atomicOr(&occ[b[q] >> 5], 1u << (b[q] & 31u));
      }
    }
  } else {
    uint32_t* hn = hw;
    unsigned long long* hs = reinterpret_cast<unsigned long long*>(hw + hist_words_n(d.B));
#pragma unroll
    for (int q = 0; q < static_cast<int>(kRegRows / 32); ++q) {
      const uint32_t r = q * 32 + lane;
      if (r < len) {
        const uint32_t e = ebuf[r];
        const uint32_t w = ent_w<1>(e);
        const long long yq = d.yreg[e >> 8];
        atomicAdd(&hn[b[q] + (b[q] >> 3)], w);
        atomicAdd(&hs[b[q] + (b[q] >> 3)], static_cast<unsigned long long>(static_cast<long long>(w) * yq));
        if (mark) atomicOr(&occ[b[q] >> 5], 1u << (b[q] & 31u));
      }
    }
  }
  __syncwarp();
}

// The lane's bits of the occupancy bitmap: its bins b0 .. b0 + bpl - 1.
__device__ __forceinline__ uint32_t lane_occ(const Dev& d, const uint32_t* occ) {
  const int bpl = (d.B + 31) >> 5;
  const int b0 = (threadIdx.x & 31) * bpl;
  const uint64_t w = static_cast<uint64_t>(occ[b0 >> 5]) | (static_cast<uint64_t>(occ[(b0 >> 5) + 1]) << 32);
  return static_cast<uint32_t>(w >> (b0 & 31)) & ((1u << bpl) - 1u);
}

// Zeroes the occupied bins of a staged histogram (each lane its own, after
// its own reads) and the bitmap, so that the next feature starts from zero.
template <int KIND>
__device__ __forceinline__ void hist_unstage(const Dev& d, uint32_t* hw, uint32_t* occ, uint32_t mine) {
  const int lane = threadIdx.x & 31;
  const int bpl = (d.B + 31) >> 5;
  const int b0 = lane * bpl;
  for (uint32_t m = mine; m; m &= m - 1) {
    const int bb = b0 + __ffs(m) - 1;
    if (KIND == 0) {
      for (int k = 0; k < d.C; ++k) hw[bb * d.C + k + (bb >> 3)] = 0u;
    } else {
      hw[bb + (bb >> 3)] = 0u;
      reinterpret_cast<unsigned long long*>(hw + hist_words_n(d.B))[bb + (bb >> 3)] = 0ull;
    }
  }
  __syncwarp();
  if (lane < 9) occ[lane] = 0u;
  __syncwarp();
}

__device__ __forceinline__ void gather_staged(const uint8_t* col, uint32_t len, const uint32_t* ebuf,
                                              uint32_t (&b)[kRegRows / 32]) {
  const int lane = threadIdx.x & 31;
  const uint64_t pol = keep_policy();
#pragma unroll
  for (int q = 0; q < static_cast<int>(kRegRows / 32); ++q) {
    const uint32_t r = q * 32 + lane;
    b[q] = r < len ? ld_keep(col + (ebuf[r] >> 8), pol) : 0u;
  }
}

// float score of a packed candidate (-1 for a feature without a valid split)
template <int KIND, int CM>
__device__ __forceinline__ float packed_score_f(const PackedCand<CM>& p, const NodeInfo<CM>& nd, int C) {
  if (p.fb == kLeaf) return -1.0f;
  if (KIND == 1) {
    const long long SL = static_cast<long long>(static_cast<unsigned long long>(p.cL[0]) |
                                                (static_cast<unsigned long long>(p.cL[1]) << 32));
    return score_reg_f(SL, nd.SP, p.nL, nd.n);
  }
  return score_class_f<CM>(p.cL, nd.cp, C, p.nL, nd.n);
}

// ---------------------------------------------------------------- feature-band path
// The level's (larger node, draw slot) items are cut into groups: the items
// of one node whose features fall in one band of columns.  Groups are sorted
// by band, so the warps sweep the augmented matrix band by band and a band's
// columns stay in L2 while its groups run; a group of a node of at most
// kRegRows rows reads the node's row entries once for all of its features,
// into the warp's shared memory.
//   item  = rank << 36 | slot << 22 | feature      (items_u, per node by band)
//   group = rank << 28 | first item << 14 | count-1 (items_s, by band)
__device__ __forceinline__ uint64_t pack_item(uint32_t rank, uint32_t slot, uint32_t f) {
  return (static_cast<uint64_t>(rank) << 36) | (static_cast<uint64_t>(slot) << 22) | f;
}

__device__ __forceinline__ uint64_t pack_group(uint32_t rank, uint32_t first, uint32_t count) {
  return (static_cast<uint64_t>(rank) << 28) | (static_cast<uint64_t>(first) << 14) | (count - 1u);
}

// most items in a group of a node with len rows
__device__ __forceinline__ uint32_t group_cap(const Dev& d, uint32_t len) {
  return len <= kRegRows ? (1u << 14) : max(1u, d.group_work / len);
}

// Exclusive scan of a warp's per-band counters in place; returns the total.
__device__ __forceinline__ uint32_t warp_scan_bands(uint32_t* cnt, int nbands, int lane) {
  const int bpl = (nbands + 31) >> 5;
  uint32_t sum = 0;
  for (int q = 0; q < bpl; ++q) {
    const int b = lane * bpl + q;
    if (b < nbands) sum += cnt[b];
  }
  uint32_t run = warp_excl_scan_u32(sum, lane);
  const uint32_t total = __shfl_sync(kFull, run + sum, 31);
  for (int q = 0; q < bpl; ++q) {
    const int b = lane * bpl + q;
    if (b < nbands) {
      const uint32_t c = cnt[b];
      cnt[b] = run;
      run += c;
    }
  }
  __syncwarp();
  return total;
}

// Per larger node (one warp): cache its totals, draw its mtry features,
// write its items ordered by band and count its groups per band.
template <int KIND, int CM>
__global__ void __launch_bounds__(256) k_plan_gen(Dev d, int level) {
  __shared__ uint32_t sband[kMaxBands];
  __shared__ uint32_t wcnt[8][kMaxBands];
  const uint32_t nbig = chunk_nodes(d, level);
  if (nbig == 0u) return;
  for (int b = threadIdx.x; b < d.nbands; b += blockDim.x) sband[b] = 0u;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t* cnt = wcnt[warp];
  const uint32_t bw = static_cast<uint32_t>(d.band_w);
  const uint32_t gwarp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
  for (uint32_t rank = gwarp; rank < nbig; rank += nwarps) {
    const uint32_t k = d.big[d.chunk0 + rank];
    uint32_t len = 0;
    if (lane == 0) {  // the node's totals, read once here instead of by each of its groups
      NodeInfo<CM> nd;
      load_node<KIND, CM>(d, k, level, nd);
      reinterpret_cast<NodeInfo<CM>*>(d.ninfo)[rank] = nd;
      len = nd.len;
    }
    len = __shfl_sync(kFull, len, 0);
    for (int b = lane; b < d.nbands; b += 32) cnt[b] = 0u;
    __syncwarp();
    Perm P;
    node_perm(d, k, P);
    for (int s = lane; s < d.mtry; s += 32) atomicAdd(&cnt[perm_apply(P, static_cast<uint32_t>(s)) / bw], 1u);
    __syncwarp();
    const uint32_t gc = group_cap(d, len);
    for (int b = lane; b < d.nbands; b += 32)
      if (cnt[b]) atomicAdd(&sband[b], (cnt[b] + gc - 1) / gc);
    __syncwarp();
    warp_scan_bands(cnt, d.nbands, lane);
    uint64_t* out = d.items_u + static_cast<uint64_t>(rank) * d.mtry;
    for (int s = lane; s < d.mtry; s += 32) {
      const uint32_t f = perm_apply(P, static_cast<uint32_t>(s));
      out[atomicAdd(&cnt[f / bw], 1u)] = pack_item(rank, static_cast<uint32_t>(s), f);
    }
    __syncwarp();
  }
  __syncthreads();
  for (int b = threadIdx.x; b < d.nbands; b += blockDim.x)
    if (sband[b]) atomicAdd(&d.band_cnt[b], sband[b]);
}

// exclusive scan of the per-band group counts into band cursors, and the
// total (one warp)
__global__ void k_plan_scan(Dev d, int level) {
  if (chunk_nodes(d, level) == 0u) return;
  const uint32_t total = warp_scan_bands(d.band_cnt, d.nbands, threadIdx.x & 31);
  if (threadIdx.x == 0) d.band_cnt[kMaxBands] = total;
}

// Per larger node (one warp): its groups, placed in their bands.
template <int KIND, int CM>
__global__ void __launch_bounds__(256) k_plan_scatter(Dev d, int level) {
  __shared__ uint32_t wcnt[8][kMaxBands];
  const uint32_t nbig = chunk_nodes(d, level);
  if (nbig == 0u) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t* cnt = wcnt[warp];
  const uint32_t bw = static_cast<uint32_t>(d.band_w);
  const uint32_t gwarp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
  const int bpl = (d.nbands + 31) >> 5;
  for (uint32_t rank = gwarp; rank < nbig; rank += nwarps) {
    const NodeInfo<CM>* nd = reinterpret_cast<const NodeInfo<CM>*>(d.ninfo) + rank;
    const uint32_t len = nd->len;
    const uint64_t where = (static_cast<uint64_t>(nd->base) << 24) | len;  // N < 2^24
    const uint64_t* items = d.items_u + static_cast<uint64_t>(rank) * d.mtry;
    for (int b = lane; b < d.nbands; b += 32) cnt[b] = 0u;
    __syncwarp();
    for (int s = lane; s < d.mtry; s += 32)
      atomicAdd(&cnt[static_cast<uint32_t>(items[s] & 0x3FFFFFu) / bw], 1u);
    __syncwarp();
    // lane-owned bands: count, then node-local start (the items are in band order)
    uint32_t c[8];  // bpl <= 8 (at most 256 bands)
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int b = lane * bpl + q;
      c[q] = (q < bpl && b < d.nbands) ? cnt[b] : 0u;
    }
    __syncwarp();
    warp_scan_bands(cnt, d.nbands, lane);
    const uint32_t gc = group_cap(d, len);
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int b = lane * bpl + q;
      if (q >= bpl || b >= d.nbands || c[q] == 0u) continue;
      const uint32_t first = cnt[b], n = c[q], ng = (n + gc - 1) / gc;
      const uint32_t pos = atomicAdd(&d.band_cnt[b], ng);
      for (uint32_t g = 0; g < ng; ++g) {
        d.items_s[pos + g] = pack_group(rank, first + g * gc, min(gc, n - g * gc));
        d.items_b[pos + g] = where;
      }
    }
    __syncwarp();
  }
}

// one warp per group: each feature's exact best candidate, packed
// band < 0: every group of the chunk; else only the groups of that band
// (one launch per band keeps the warps, and the L2, on one band at a time).
template <int KIND, int CM>
__global__ void __launch_bounds__(kSplitThreads, BORUTA_ITEMS_MINB) k_items_band(Dev d, int level, int band) {
  extern __shared__ __align__(16) uint32_t smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t* hw = smem + warp * (split_smem_per_warp(d.kind, d.C, d.B) / 4);
  uint32_t* ebuf = hw + hist_smem_per_warp(d.kind, d.C, d.B) / 4;
  uint32_t* occ = ebuf + kRegRows;
  unsigned long long* hp = reinterpret_cast<unsigned long long*>(hw);  // the packed layout
  if (chunk_nodes(d, level) == 0u) return;
  hist_clear<KIND>(d, hw);  // from here on a feature leaves the histogram zeroed
  if (lane < 9) occ[lane] = 0u;
  __syncwarp();
  const uint32_t gwarp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
  const uint32_t* rows_in = d.rows[level & 1];
  // after k_plan_scatter band_cnt[b] is the end of band b's groups
  const uint32_t g0 = band <= 0 ? 0u : d.band_cnt[band - 1];
  const uint32_t g1 = band < 0 ? d.band_cnt[kMaxBands] : d.band_cnt[band];
  // staged nodes: the scan reads only the occupied bins when the histogram
  // is large (it is then mostly empty); small histograms are read whole
  const bool sparse = d.B * (KIND ? 3 : ncls<CM>(d)) >= 512;
  unsigned long long bytes = 0;
  // Software pipeline over the warp's groups: a group's record (node rank,
  // items, and the node's row offset and size) is loaded one group ahead,
  // so a group starts with the loads of its row entries, node totals and
  // items all in flight at once, and the next staged node's entries are
  // prefetched into L2 while this group's features run.
  uint32_t g = g0 + gwarp;
  uint64_t gr = 0ull, gb = 0ull;
  if (g < g1) {
    gr = d.items_s[g];
    gb = d.items_b[g];
  }
  for (; g < g1; g += nwarps) {
    const uint32_t gn = g + nwarps;
    uint64_t gr_n = 0ull, gb_n = 0ull;
    if (gn < g1) {
      gr_n = d.items_s[gn];
      gb_n = d.items_b[gn];
    }
    const uint32_t rank = static_cast<uint32_t>(gr >> 28);
    const uint32_t first = static_cast<uint32_t>(gr >> 14) & 0x3FFFu;
    const uint32_t count = static_cast<uint32_t>(gr & 0x3FFFu) + 1u;
    const uint32_t len = static_cast<uint32_t>(gb & 0xFFFFFFu);
    // A node of at most kRegRows rows: its entries are read once, into the
    // warp's shared-memory buffer, for all the group's features, and the
    // next feature's bins are gathered while this one's are counted and
    // scanned.  Larger nodes stream their entries per feature.
    const bool staged = len <= kRegRows;
    uint32_t ev[kRegRows / 32];
    if (staged) {
      const uint32_t* src = rows_in + static_cast<int64_t>(gb >> 24);
#pragma unroll
      for (int q = 0; q < static_cast<int>(kRegRows / 32); ++q) {
        const uint32_t r = q * 32 + lane;
        ev[q] = r < len ? ld_stream(src + r) : 0u;
      }
    }
    const NodeInfo<CM> nd = reinterpret_cast<const NodeInfo<CM>*>(d.ninfo)[rank];
    const uint64_t* items = d.items_u + static_cast<uint64_t>(rank) * d.mtry + first;
    PackedCand<CM>* out = reinterpret_cast<PackedCand<CM>*>(d.fbest) + static_cast<uint64_t>(rank) * d.mtry;
    uint64_t chunk = items[lane < count ? lane : 0u];  // items j..j+31 of the group, one per lane
    if (staged) {
#pragma unroll
      for (int q = 0; q < static_cast<int>(kRegRows / 32); ++q)
        if (q * 32 + lane < len) ebuf[q * 32 + lane] = ev[q];
      __syncwarp();
    }
    const bool pk = packed_ok<KIND, CM>(d, nd);
    uint32_t bn[kRegRows / 32];
    if (staged) gather_staged(column(d, static_cast<uint32_t>(__shfl_sync(kFull, chunk, 0) & 0x3FFFFFu)), len,
                              ebuf, bn);
    if (gn < g1) {  // the next staged node's entries, into L2 (one 128-byte line per lane)
      const uint32_t len_n = static_cast<uint32_t>(gb_n & 0xFFFFFFu);
      if (len_n <= kRegRows && lane * 32u < len_n)
        prefetch_l2(rows_in + static_cast<int64_t>(gb_n >> 24) + lane * 32u);
    }
    for (uint32_t j = 0; j < count; ++j) {
      const uint64_t it = __shfl_sync(kFull, chunk, j & 31);
      const uint32_t f = static_cast<uint32_t>(it & 0x3FFFFFu);
      if (j + 1 < count && ((j + 1) & 31) == 0) chunk = items[j + 1 + lane < count ? j + 1 + lane : j + 1];
      PackedCand<CM>* dst = out + (static_cast<uint32_t>(it >> 22) & 0x3FFFu);
      if (staged) {
        uint32_t b[kRegRows / 32];
#pragma unroll
        for (int q = 0; q < static_cast<int>(kRegRows / 32); ++q) b[q] = bn[q];
        if (j + 1 < count)
          gather_staged(column(d, static_cast<uint32_t>(__shfl_sync(kFull, chunk, (j + 1) & 31) & 0x3FFFFFu)),
                        nd.len, ebuf, bn);
        if constexpr (KIND == 0 && CM <= 5) {
          if (pk) {
            hist_staged_pk(nd.len, ebuf, b, hp);
            scan_pack_pk<CM>(d, nd, hp, f, dst);
            continue;
          }
        }
        hist_staged<KIND>(d, nd.len, ebuf, b, hw, occ, sparse);
        if (sparse) {
          const uint32_t mine = lane_occ(d, occ);
          scan_pack<KIND, CM>(d, nd, hw, f, out + (static_cast<uint32_t>(it >> 22) & 0x3FFFu), mine);
          hist_unstage<KIND>(d, hw, occ, mine);
        } else {
          scan_pack<KIND, CM>(d, nd, hw, f, out + (static_cast<uint32_t>(it >> 22) & 0x3FFFu));
          __syncwarp();
          hist_clear<KIND>(d, hw);
          __syncwarp();
        }
      } else {
        if constexpr (KIND == 0 && CM <= 5) {
          if (pk) {
            build_hist_pk(nd.base, nd.len, rows_in, column(d, f), hp);
            scan_pack_pk<CM>(d, nd, hp, f, dst);
            continue;
          }
        }
        build_hist<KIND, false>(d, nd.base, nd.len, rows_in, column(d, f), hw);
        scan_pack<KIND, CM>(d, nd, hw, f, out + (static_cast<uint32_t>(it >> 22) & 0x3FFFu));
        __syncwarp();
        hist_clear<KIND>(d, hw);
        __syncwarp();
      }
    }
    __syncwarp();  // the entry buffer is reused by the next group
    // algorithmic bytes (the method's per-level figure): one bin per row and
    // feature, and the node's row state once (entry read and rewritten, weight
    // and label, or the 8-byte target for regression)
    bytes += static_cast<unsigned long long>(nd.len) * (count + (first == 0u ? (KIND ? kRowStateReg : kRowStateClass) : 0u));
    gr = gr_n;
    gb = gb_n;
  }
  if (lane == 0 && bytes) atomicAdd(&d.counters[2], bytes);
}

// one warp per larger node: exact argmax over the node's per-feature
// candidates (lanes over draw slots), split record, partition
template <int KIND, int CM>
__global__ void __launch_bounds__(256, BORUTA_SMALL_MINB) k_finalize_band(Dev d, int level) {
  const int lane = threadIdx.x & 31;
  const uint32_t nbig = chunk_nodes(d, level);
  if (nbig == 0u) return;
  const uint32_t gwarp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
  const uint32_t* rows_in = d.rows[level & 1];
  uint32_t* rows_out = d.rows[(level & 1) ^ 1];
  unsigned long long bytes = 0;
  for (uint32_t rank = gwarp; rank < nbig; rank += nwarps) {
    const uint32_t k = d.big[d.chunk0 + rank];
    NodeInfo<CM> nd;
    load_node<KIND, CM>(d, k, level, nd);
    const PackedCand<CM>* pc = reinterpret_cast<const PackedCand<CM>*>(d.fbest) + static_cast<uint64_t>(rank) * d.mtry;
    // float screen over the per-feature bests, then the exact argmax among
    // those inside the window
    float lmax = -1.0f;
    for (int s = lane; s < d.mtry; s += 32) lmax = fmaxf(lmax, packed_score_f<KIND, CM>(pc[s], nd, ncls<CM>(d)));
    const float mx = warp_max_f(lmax);
    const float thr = screen(mx);
    Cand<CM> best;
    best.valid = false;
    for (int s0 = 0; mx >= 0.0f && s0 < d.mtry; s0 += 32) {
      const int s = s0 + lane;
      Cand<CM> mine;
      mine.valid = false;
      if (s < d.mtry) {
        const PackedCand<CM> p = pc[s];
        if (packed_score_f<KIND, CM>(p, nd, ncls<CM>(d)) >= thr) {
          const uint32_t tkey = d.tie_break == 1 ? static_cast<uint32_t>(s) : (p.fb >> 8);
          unpack_cand<KIND, CM>(p, nd, ncls<CM>(d), tkey, mine);
        }
      }
      if (__ballot_sync(kFull, mine.valid) == 0u) continue;
      Cand<CM> c;
      warp_select<KIND, CM>(mine, c);
      if (better(c, best)) best = c;
    }
    uint32_t sp = 0;
    if (lane == 0) sp = commit_split<KIND, CM>(d, k, best, nd);
    sp = __shfl_sync(kFull, sp, 0);
    bytes += static_cast<unsigned long long>(nd.len) * (d.mtry + 4ull + (KIND ? 8ull : 0ull));
    if (sp == kLeaf) continue;
    const uint32_t nl = warp_partition(d, nd.base, nd.len, sp, rows_in, rows_out);
    if (lane == 0) d.nd_lrows[k] = nl;
    bytes += static_cast<unsigned long long>(nd.len) * 5ull;
  }
  if (lane == 0 && bytes) atomicAdd(&d.counters[0], bytes);
}

// ---------------------------------------------------------------- grouped path
// Work items of a level's larger nodes: (node, group of G consecutive draw
// slots), one warp each, spread round-robin over all warps; each item writes
// its exact best candidate and k_finalize reduces them per node.
template <int KIND, int CM>
__global__ void __launch_bounds__(kSplitThreads, BORUTA_ITEMS_MINB) k_items(Dev d, int level) {
  extern __shared__ __align__(16) uint32_t smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t* hw = smem + warp * (split_smem_per_warp(d.kind, d.C, d.B) / 4);
  const uint32_t nbig = d.work[level];
  if (band_path(d, nbig)) return;
  const uint32_t gwarp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
  const uint32_t* rows_in = d.rows[level & 1];
  const int G = (d.mtry + kItemsPerNode - 1) / kItemsPerNode;
  const int ipn = (d.mtry + G - 1) / G;
  Cand<CM>* out = reinterpret_cast<Cand<CM>*>(d.cand);
  const uint64_t total = static_cast<uint64_t>(nbig) * ipn;
  unsigned long long bytes = 0;
  for (uint64_t it = gwarp; it < total; it += nwarps) {
    const uint32_t rank = static_cast<uint32_t>(it / ipn);
    const int part = static_cast<int>(it - static_cast<uint64_t>(rank) * ipn);
    const uint32_t k = d.big[rank];
    NodeInfo<CM> nd;
    load_node<KIND, CM>(d, k, level, nd);
    Perm P;
    node_perm(d, k, P);
    Cand<CM> best;
    best.valid = false;
    const int s1 = min(d.mtry, (part + 1) * G);
    for (int slot = part * G; slot < s1; ++slot) {
      const uint32_t f = perm_apply(P, static_cast<uint32_t>(slot));
      const uint32_t tkey = d.tie_break == 1 ? static_cast<uint32_t>(slot) : f;
      Cand<CM> c;
      dense_feature<KIND, CM>(d, nd, rows_in, static_cast<int>(f), tkey, hw, c);
      if (better(c, best)) best = c;
    }
    if (lane == 0) out[it] = best;
    bytes += static_cast<unsigned long long>(s1 - part * G) * nd.len * (KIND ? 13ull : 5ull) + sizeof(Cand<CM>);
  }
  if (lane == 0 && bytes) atomicAdd(&d.counters[2], bytes);
}

// One warp per larger node: exact argmax over the node's item candidates,
// split record, partition.
template <int KIND, int CM>
__global__ void __launch_bounds__(256, BORUTA_SMALL_MINB) k_finalize(Dev d, int level) {
  const int lane = threadIdx.x & 31;
  const uint32_t nbig = d.work[level];
  if (band_path(d, nbig)) return;
  const uint32_t gwarp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
  const uint32_t* rows_in = d.rows[level & 1];
  uint32_t* rows_out = d.rows[(level & 1) ^ 1];
  const int G = (d.mtry + kItemsPerNode - 1) / kItemsPerNode;
  const int ipn = (d.mtry + G - 1) / G;
  const Cand<CM>* cand = reinterpret_cast<const Cand<CM>*>(d.cand);
  unsigned long long bytes = 0;
  for (uint32_t rank = gwarp; rank < nbig; rank += nwarps) {
    const uint32_t k = d.big[rank];
    NodeInfo<CM> nd;
    load_node<KIND, CM>(d, k, level, nd);
    Cand<CM> mine;
    mine.valid = false;
    if (lane < ipn) mine = cand[static_cast<uint64_t>(rank) * ipn + lane];
    Cand<CM> best;
    warp_select<KIND, CM>(mine, best);
    uint32_t sp = 0;
    if (lane == 0) sp = commit_split<KIND, CM>(d, k, best, nd);
    sp = __shfl_sync(kFull, sp, 0);
    bytes += static_cast<unsigned long long>(nd.len) * (d.mtry + 4ull + (KIND ? 8ull : 0ull));
    if (sp == kLeaf) continue;
    const uint32_t nl = warp_partition(d, nd.base, nd.len, sp, rows_in, rows_out);
    if (lane == 0) d.nd_lrows[k] = nl;
    bytes += static_cast<unsigned long long>(nd.len) * 5ull;
  }
  if (lane == 0 && bytes) atomicAdd(&d.counters[0], bytes);
}

template <int KIND, int CM>
int launch_level(const Dev& d, int level, int grid_small, int grid_items, uint64_t big_bound, size_t smem,
                 cudaStream_t st, cudaStream_t st2, cudaEvent_t fork, cudaEvent_t join, cudaEvent_t hist_start,
                 cudaEvent_t hist_end) {
  int n = 4;  // k_classify and the three small-node kernels
  k_classify<KIND, CM><<<grid_small, 256, 0, st>>>(d, level);
  // small nodes on st2, concurrently with the larger-node kernels on st
  cudaEventRecord(fork, st);
  cudaStreamWaitEvent(st2, fork, 0);
  k_split_small<KIND, CM, 8><<<grid_small, 256, 0, st2>>>(d, level);
  k_split_small<KIND, CM, 16><<<grid_small, 256, 0, st2>>>(d, level);
  k_split_small<KIND, CM, 32><<<grid_small, 256, 0, st2>>>(d, level);
  cudaEventRecord(join, st2);
  // band path: the larger nodes in chunks of chunk_cap (at most big_bound
  // nodes exist; chunks past the level's count return at once)
  const uint64_t nchunks =
      d.band_w > 0 ? (big_bound + d.chunk_cap - 1) / d.chunk_cap + (big_bound == 0 ? 1 : 0) : 0;
  for (uint64_t c = 0; c < nchunks; ++c) {
    Dev dc = d;
    dc.chunk0 = static_cast<uint32_t>(c * d.chunk_cap);
    cudaMemsetAsync(d.band_cnt, 0, (kMaxBands + 1) * sizeof(uint32_t), st);
    k_plan_gen<KIND, CM><<<grid_small, 256, 0, st>>>(dc, level);
    k_plan_scan<<<1, 32, 0, st>>>(dc, level);
    k_plan_scatter<KIND, CM><<<grid_small, 256, 0, st>>>(dc, level);
    // the histogram kernel of the level (with several chunks the window also
    // holds the later chunks' plan and finalize kernels)
    if (c == 0 && hist_start) cudaEventRecord(hist_start, st);
    if (d.band_launch)
      for (int b = 0; b < d.nbands; ++b) k_items_band<KIND, CM><<<grid_items, kSplitThreads, smem, st>>>(dc, level, b);
    else
      k_items_band<KIND, CM><<<grid_items, kSplitThreads, smem, st>>>(dc, level, -1);
    if (c + 1 == nchunks && hist_end) cudaEventRecord(hist_end, st);
    k_finalize_band<KIND, CM><<<grid_small, 256, 0, st>>>(dc, level);
    n += 4 + (d.band_launch ? d.nbands : 1);
  }
  if (nchunks == 0) {  // grouped path
    if (hist_start) cudaEventRecord(hist_start, st);
    k_items<KIND, CM><<<grid_items, kSplitThreads, smem, st>>>(d, level);
    if (hist_end) cudaEventRecord(hist_end, st);
    k_finalize<KIND, CM><<<grid_small, 256, 0, st>>>(d, level);
    n += 2;
  }
  cudaStreamWaitEvent(st, join, 0);
  return n;
}

// Kernel variants: 0..4 classification with CM = 2, 3, 4, 5, 8 classes at
// most (3, 4 and 5 exactly), 5 regression.
template <typename F>
auto with_variant(int variant, F&& f) {
  switch (variant) {
    case 0: return f(std::integral_constant<int, 0>{}, std::integral_constant<int, 2>{});
    case 1: return f(std::integral_constant<int, 0>{}, std::integral_constant<int, 3>{});
    case 2: return f(std::integral_constant<int, 0>{}, std::integral_constant<int, 4>{});
    case 3: return f(std::integral_constant<int, 0>{}, std::integral_constant<int, 5>{});
    case 4: return f(std::integral_constant<int, 0>{}, std::integral_constant<int, 8>{});
    default: return f(std::integral_constant<int, 1>{}, std::integral_constant<int, 1>{});
  }
}

}  // namespace

int split_variant(int kind, int C) {
  if (kind != 0) return 5;
  return C <= 2 ? 0 : (C <= 5 ? C - 2 : 4);
}

int variant_classes(int variant) { return with_variant(variant, [](auto, auto cm) { return decltype(cm)::value; }); }

size_t packed_bytes(int variant) {
  return with_variant(variant, [](auto, auto cm) { return sizeof(PackedCand<decltype(cm)::value>); });
}

size_t cand_bytes(int variant) {
  return with_variant(variant, [](auto, auto cm) { return sizeof(Cand<decltype(cm)::value>); });
}

size_t ninfo_bytes(int variant) {
  return with_variant(variant, [](auto, auto cm) { return sizeof(NodeInfo<decltype(cm)::value>); });
}

void split_kernel_ptrs(int variant, const void** ptrs, int* n) {
  with_variant(variant, [&](auto kind, auto cm) {
    constexpr int K = decltype(kind)::value, CM = decltype(cm)::value;
    ptrs[0] = reinterpret_cast<const void*>(&k_items<K, CM>);
    ptrs[1] = reinterpret_cast<const void*>(&k_items_band<K, CM>);
    return 0;
  });
  *n = 2;
}

const void* small_kernel_ptr(int variant) {
  return with_variant(variant, [](auto kind, auto cm) {
    return reinterpret_cast<const void*>(&k_split_small<decltype(kind)::value, decltype(cm)::value, 32>);
  });
}

int launch_split(const Dev& d, int level, int grid_small, int grid_big, uint64_t big_bound, size_t smem,
                 cudaStream_t st, cudaStream_t st2, cudaEvent_t fork, cudaEvent_t join, cudaEvent_t hs,
                 cudaEvent_t he) {
  return with_variant(split_variant(d.kind, d.C), [&](auto kind, auto cm) {
    return launch_level<decltype(kind)::value, decltype(cm)::value>(d, level, grid_small, grid_big, big_bound, smem,
                                                                     st, st2, fork, join, hs, he);
  });
}

}  // namespace bgb
