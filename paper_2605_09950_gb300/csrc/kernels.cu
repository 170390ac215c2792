// GPU Boruta kernels for sm_103a.
//
// One Boruta iteration (Alg. 1 loop body) runs as:
//   k_shadow           X_sha = per-column shuffled copies of X_cur       (Alg. 1)
//   k_boot_count       bootstrap draw counts for every tree               (forest fit)
//   k_boot_compact     in-bag row lists, out-of-bag lists, root nodes
//   per level:  k_split     per-node feature sample, histograms, exact split scan,
//                           impurity decrease into the TreeImp accumulators (Alg. 2),
//                           stable row partition
//               k_count / k_children   next level's nodes
//   k_treeimp_norm  or  k_permut + k_permut_final                       (Alg. 2 / Alg. 3)
//   k_stats, k_decide  Z score / mean over trees, hits, binomial test   (Alg. 1)
// Every tree of the iteration is processed by the same launches (level
// synchronous); node work is claimed dynamically by persistent CTAs.
#include <cstdint>

#include "engine.cuh"

namespace bgb {

namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;

__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// exclusive block scan of one u32 per thread; returns the block total in *total
__device__ uint32_t block_excl_scan(uint32_t v, uint32_t* total, uint32_t* smem_warp) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  uint32_t x = v;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const uint32_t y = __shfl_up_sync(kFull, x, d);
    if (lane >= d) x += y;
  }
  if (lane == 31) smem_warp[warp] = x;
  __syncthreads();
  if (warp == 0) {
    uint32_t w = lane < nw ? smem_warp[lane] : 0u;
    uint32_t z = w;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const uint32_t y = __shfl_up_sync(kFull, z, d);
      if (lane >= d) z += y;
    }
    if (lane < nw) smem_warp[lane] = z - w;
    if (lane == 31) smem_warp[32] = z;
  }
  __syncthreads();
  const uint32_t r = smem_warp[warp] + x - v;
  *total = smem_warp[32];
  __syncthreads();
  return r;
}

template <typename T>
__device__ T block_sum(T v, T* smem) {
  // smem: blockDim.x entries
  smem[threadIdx.x] = v;
  __syncthreads();
  for (int s = blockDim.x >> 1; s > 0; s >>= 1) {
    if (threadIdx.x < s) smem[threadIdx.x] += smem[threadIdx.x + s];
    __syncthreads();
  }
  const T r = smem[0];
  __syncthreads();
  return r;
}

}  // namespace

// ============================================================ input validation
__global__ void k_validate(Dev d) {
  bool bad = false;
  uint32_t maxlab = 0;
  for (int j = blockIdx.y; j < d.p; j += gridDim.y) {
    const uint8_t* col = d.X + static_cast<int64_t>(j) * d.ld;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < d.N; i += gridDim.x * blockDim.x)
      bad |= col[i] >= d.B;
  }
  if (blockIdx.y == 0 && d.kind == 0) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < d.N; i += gridDim.x * blockDim.x) {
      const uint32_t y = d.ycls[i];
      maxlab = max(maxlab, y);
      bad |= static_cast<int>(y) >= kMaxClasses;
    }
    if (maxlab) atomicMax(&d.status[2], maxlab);
  }
  if (blockIdx.y == 0 && d.kind != 0) {
    unsigned long long mx = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < d.N; i += gridDim.x * blockDim.x) {
      const long long v = d.yreg[i];
      const unsigned long long a = v < 0 ? 0ull - static_cast<unsigned long long>(v) : static_cast<unsigned long long>(v);
      mx = a > mx ? a : mx;
    }
    if (mx) atomicMax(&d.counters[1], mx);
  }
  if (bad) atomicOr(&d.status[0], kErrInput);
}

void launch_validate(const Dev& d, cudaStream_t st) {
  dim3 grid((d.N + 255) / 256 > 64 ? 64 : (d.N + 255) / 256, d.p < 1024 ? d.p : 1024);
  k_validate<<<grid, 256, 0, st>>>(d);
}

// ============================================================ Alg. 1: shadow features
// Xsha[c][i] = X[sigma_c(i)][live[c mod p_live]]; 16 rows per thread, one
// 16-byte store.  The source column is read through L2 (random gather).
__global__ void k_shadow(Dev d) {
  const int c = blockIdx.y;
  __shared__ Perm sp;
  if (threadIdx.x == 0)
    perm_init(sp, static_cast<uint32_t>(d.N), d.seed, 0u, unit_word(d.t, c),
              purpose_word(kPurposeShadow, d.job));
  __syncthreads();
  const Perm P = sp;
  const uint8_t* src = d.X + static_cast<int64_t>(d.live[c % d.p_live]) * d.ld;
  uint8_t* dst = d.Xsha + static_cast<int64_t>(c) * d.ldN;
  for (int base = (blockIdx.x * blockDim.x + threadIdx.x) * 16; base < d.N;
       base += gridDim.x * blockDim.x * 16) {
    uint32_t v[4] = {0u, 0u, 0u, 0u};
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      const int i = base + k;
      if (i < d.N) v[k >> 2] |= static_cast<uint32_t>(src[perm_apply(P, i)]) << (8 * (k & 3));
    }
    *reinterpret_cast<uint4*>(dst + base) = make_uint4(v[0], v[1], v[2], v[3]);
  }
}

void launch_shadow(const Dev& d, cudaStream_t st) {
  int bx = (d.N + 16 * 256 - 1) / (16 * 256);
  if (bx > 32) bx = 32;
  k_shadow<<<dim3(bx, d.n_sha), 256, 0, st>>>(d);
}

// ============================================================ bootstrap
// Draw d of tree tau picks row floor(r * N / 2^64), r = Philox(t, BOOT, tau, d).
__global__ void k_boot_count(Dev d) {
  for (int tau = blockIdx.y; tau < d.M; tau += gridDim.y) {
    uint32_t* cnt = d.bootcnt + static_cast<int64_t>(tau) * d.N;
    const uint32_t w2 = unit_word(d.t, tau), w3 = purpose_word(kPurposeBoot, d.job);
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < d.N; k += gridDim.x * blockDim.x) {
      const uint64_t r = draw64(d.seed, static_cast<uint32_t>(k), 0u, w2, w3);
      atomicAdd(cnt + __umul64hi(r, static_cast<uint64_t>(d.N)), 1u);
    }
  }
}

// One CTA per tree: in-bag entries (row << 8 | count) ascending, OOB rows
// ascending, and the root node with its weighted class counts / target sum.
__global__ void k_boot_compact(Dev d) {
  __shared__ uint32_t sw[33];
  __shared__ unsigned long long sred[256];
  for (int tau = blockIdx.x; tau < d.M; tau += gridDim.x) {
    const uint32_t* cnt = d.bootcnt + static_cast<int64_t>(tau) * d.N;
    uint32_t* rows = d.rows[0] + static_cast<int64_t>(tau) * d.N;
    uint32_t* oob = d.oob + static_cast<int64_t>(tau) * d.N;
    uint32_t nin = 0, noob = 0;
    uint32_t ccnt[kMaxClasses];
#pragma unroll
    for (int k = 0; k < kMaxClasses; ++k) ccnt[k] = 0;
    long long S = 0;
    bool wbad = false;
    for (int base = 0; base < d.N; base += blockDim.x) {
      const int i = base + threadIdx.x;
      const uint32_t c = i < d.N ? cnt[i] : 0u;
      const bool in = c > 0u, out = (i < d.N) && c == 0u;
      wbad |= c > 255u;
      uint32_t tin, tout;
      const uint32_t rin = block_excl_scan(in ? 1u : 0u, &tin, sw);
      const uint32_t rout = block_excl_scan(out ? 1u : 0u, &tout, sw);
      if (in) {
        rows[nin + rin] = (static_cast<uint32_t>(i) << 8) | min(c, 255u);
        if (d.kind == 0) {
          const uint32_t y = d.ycls[i];
#pragma unroll
          for (int k = 0; k < kMaxClasses; ++k) ccnt[k] += (y == static_cast<uint32_t>(k)) ? c : 0u;
        } else {
          S += static_cast<long long>(c) * d.yreg[i];
        }
      }
      if (out) oob[noob + rout] = static_cast<uint32_t>(i);
      nin += tin;
      noob += tout;
    }
    if (wbad) atomicOr(&d.status[0], kErrWeight);
    const uint32_t root = static_cast<uint32_t>(tau);  // level 0 holds the M roots in tree order
    uint32_t nsum = 0;
    if (d.kind == 0) {
      for (int k = 0; k < d.C; ++k) {
        const unsigned long long tot = block_sum<unsigned long long>(ccnt[k], sred);
        if (threadIdx.x == 0) d.nd_cnt[static_cast<int64_t>(root) * d.C + k] = static_cast<uint32_t>(tot);
        nsum += static_cast<uint32_t>(tot);
      }
    } else {
      const unsigned long long tot =
          block_sum<unsigned long long>(static_cast<unsigned long long>(S), sred);
      if (threadIdx.x == 0) d.nd_S[root] = static_cast<long long>(tot);
      nsum = static_cast<uint32_t>(d.N);
    }
    if (threadIdx.x == 0) {
      d.nd_tree[root] = static_cast<uint32_t>(tau);
      d.nd_heap[root] = 0u;
      d.nd_seg[root] = 0u;
      d.nd_len[root] = nin;
      d.nd_n[root] = nsum;
      d.nd_split[root] = kLeaf;
      d.nd_child[root] = 0u;
      d.nd_delta[root] = 0.0;
      d.oob_cnt[tau] = noob;
    }
    __syncthreads();
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    d.lvl_off[0] = 0u;
    d.lvl_cnt[0] = static_cast<uint32_t>(d.M);
  }
}

void launch_bootstrap(const Dev& d, int grid, cudaStream_t st) {
  int bx = (d.N + 255) / 256;
  if (bx > 64) bx = 64;
  int by = d.M < 4096 ? d.M : 4096;
  k_boot_count<<<dim3(bx, by), 256, 0, st>>>(d);
  k_boot_compact<<<grid, 256, 0, st>>>(d);
}

// ============================================================ split search
// Candidate split of a node: left = rows with bin <= `bin` of feature `feat`.
// Score num/den = (A_L n_R + A_R n_L) / (n_L n_R), A = sum_k c_k^2 (Gini) or
// S^2 (variance), compared exactly; equal scores go to the lower key =
// (feature draw slot, or feature index) << 8 | bin.
struct Cand {
  U192 num;
  uint64_t den;
  uint32_t key;
  uint32_t nL;
  uint32_t cL[kMaxClasses];
  long long SL;
  int32_t feat;
  int32_t bin;
  bool valid;
};

__device__ __forceinline__ bool cand_better(const Cand& a, const Cand& b) {
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

// exact classification candidate from left counts
__device__ __forceinline__ void cand_class(Cand& c, const uint32_t* cl, const uint32_t* cp, int C,
                                           uint32_t nL, uint32_t n) {
  uint64_t AL = 0, AR = 0;
#pragma unroll
  for (int k = 0; k < kMaxClasses; ++k) {
    if (k < C) {
      const uint64_t l = cl[k], r = cp[k] - cl[k];
      AL += l * l;
      AR += r * r;
      c.cL[k] = cl[k];
    }
  }
  const uint32_t nR = n - nL;
  c.num = u192_from(static_cast<u128>(AL) * nR + static_cast<u128>(AR) * nL);
  c.den = static_cast<uint64_t>(nL) * nR;
  c.nL = nL;
  c.valid = true;
}

__device__ __forceinline__ void cand_reg(Cand& c, long long SL, long long SP, uint32_t nL, uint32_t n) {
  const uint32_t nR = n - nL;
  c.num = u192_add(u192_mul(sq_i64(SL), nR), u192_mul(sq_i64(SP - SL), nL));
  c.den = static_cast<uint64_t>(nL) * nR;
  c.nL = nL;
  c.SL = SL;
  c.valid = true;
}

__device__ __forceinline__ float score_class_f(const uint32_t* cl, const uint32_t* cp, int C,
                                               uint32_t nL, uint32_t n) {
  uint64_t AL = 0, AR = 0;
#pragma unroll
  for (int k = 0; k < kMaxClasses; ++k) {
    if (k < C) {
      const uint64_t l = cl[k], r = cp[k] - cl[k];
      AL += l * l;
      AR += r * r;
    }
  }
  return __fdividef(static_cast<float>(AL), static_cast<float>(nL)) +
         __fdividef(static_cast<float>(AR), static_cast<float>(n - nL));
}

__device__ __forceinline__ float score_reg_f(long long SL, long long SP, uint32_t nL, uint32_t n) {
  const float l = static_cast<float>(SL), r = static_cast<float>(SP - SL);
  return __fdividef(l * l, static_cast<float>(nL)) + __fdividef(r * r, static_cast<float>(n - nL));
}

// all lanes: out = best of the valid lane candidates (lanes scanned in order)
__device__ void warp_select(const Cand& mine, Cand& out, int C, bool reg) {
  unsigned m = __ballot_sync(kFull, mine.valid);
  out.valid = false;
  while (m) {
    const int l = __ffs(m) - 1;
    m &= m - 1;
    Cand c;
    c.num.w[0] = __shfl_sync(kFull, mine.num.w[0], l);
    c.num.w[1] = __shfl_sync(kFull, mine.num.w[1], l);
    c.num.w[2] = __shfl_sync(kFull, mine.num.w[2], l);
    c.den = __shfl_sync(kFull, mine.den, l);
    c.key = __shfl_sync(kFull, mine.key, l);
    c.nL = __shfl_sync(kFull, mine.nL, l);
    c.feat = __shfl_sync(kFull, mine.feat, l);
    c.bin = __shfl_sync(kFull, mine.bin, l);
    if (reg) {
      c.SL = __shfl_sync(kFull, mine.SL, l);
    } else {
#pragma unroll
      for (int k = 0; k < kMaxClasses; ++k)
        if (k < C) c.cL[k] = __shfl_sync(kFull, mine.cL[k], l);
    }
    c.valid = true;
    if (cand_better(c, out)) out = c;
  }
}

// Relative window of the float pre-screen.  The float score of a candidate
// is within ~2^-21 of its exact value, so every candidate whose exact score
// is the maximum has a float score above (1 - 2^-12) * (best float score);
// only those are compared exactly.
#define SCREEN(m) ((m) - (m) * 0.000244140625f)

struct NodeInfo {
  int64_t base;  // tree row-buffer offset + segment offset
  uint32_t len, n;
  uint32_t cp[kMaxClasses];
  long long SP;
};

// Best split of feature `feat` (draw slot `slot`) at the node, warp-wide.
// Nodes with at most 32 distinct rows: one row per lane, candidates at the
// bins present.  Larger nodes: warp-private shared-memory histogram, a warp
// prefix scan over the bins, float screen, exact comparison.
__device__ void feature_best(const Dev& d, const NodeInfo& nd, const uint32_t* rows, int feat,
                             uint32_t tkey, uint32_t* hw, Cand& out) {
  const int lane = threadIdx.x & 31;
  const bool reg = d.kind != 0;
  const int C = d.C;
  const uint8_t* col = d.colptr[feat];
  Cand mine;
  mine.valid = false;
  mine.feat = feat;
  if (nd.len <= 32u) {
    const bool v = lane < static_cast<int>(nd.len);
    const uint32_t e = v ? rows[nd.base + lane] : 0u;
    const uint32_t row = e >> 8, w = e & 255u;
    const uint32_t b = v ? col[row] : 0u;
    const uint32_t y = (v && !reg) ? d.ycls[row] : 0u;
    const long long yv = (v && reg) ? d.yreg[row] : 0ll;
    uint32_t cl[kMaxClasses];
#pragma unroll
    for (int k = 0; k < kMaxClasses; ++k) cl[k] = 0u;
    uint32_t nL = 0;
    long long SL = 0;
    for (int j = 0; j < static_cast<int>(nd.len); ++j) {
      const uint32_t bj = __shfl_sync(kFull, b, j), wj = __shfl_sync(kFull, w, j);
      if (reg) {
        const long long yj = __shfl_sync(kFull, yv, j);
        if (bj <= b) {
          nL += wj;
          SL += static_cast<long long>(wj) * yj;
        }
      } else {
        const uint32_t yj = __shfl_sync(kFull, y, j);
        if (bj <= b) {
          nL += wj;
#pragma unroll
          for (int k = 0; k < kMaxClasses; ++k) cl[k] += (yj == static_cast<uint32_t>(k)) ? wj : 0u;
        }
      }
    }
    const bool ok = v && nL < nd.n;
    float sf = -1.0f;
    if (ok) sf = reg ? score_reg_f(SL, nd.SP, nL, nd.n) : score_class_f(cl, nd.cp, C, nL, nd.n);
    const float mx = warp_max_f(sf);
    if (mx < 0.0f) {
      out.valid = false;
      return;
    }
    if (ok && sf >= SCREEN(mx)) {
      if (reg)
        cand_reg(mine, SL, nd.SP, nL, nd.n);
      else
        cand_class(mine, cl, nd.cp, C, nL, nd.n);
      mine.bin = static_cast<int32_t>(b);
      mine.key = (tkey << 8) | b;
    }
    warp_select(mine, out, C, reg);
    return;
  }

  // ---- dense histogram
  const int B = d.B;
  const int bpl = (B + 31) >> 5;  // bins per lane
  const int b0 = lane * bpl;
  if (!reg) {
    for (int i = lane; i < B * C; i += 32) hw[i] = 0u;
    __syncwarp();
    for (uint32_t r = lane; r < nd.len; r += 32) {
      const uint32_t e = rows[nd.base + r];
      const uint32_t row = e >> 8;
      atomicAdd(&hw[col[row] * C + d.ycls[row]], e & 255u);
    }
    __syncwarp();
    uint32_t tot[kMaxClasses], pre[kMaxClasses];
#pragma unroll
    for (int k = 0; k < kMaxClasses; ++k) tot[k] = 0u;
    for (int q = 0; q < bpl; ++q) {
      const int b = b0 + q;
      if (b < B) {
#pragma unroll
        for (int k = 0; k < kMaxClasses; ++k)
          if (k < C) tot[k] += hw[b * C + k];
      }
    }
#pragma unroll
    for (int k = 0; k < kMaxClasses; ++k) pre[k] = (k < C) ? warp_excl_scan_u32(tot[k], lane) : 0u;
    // pass 1: float scores
    float sf[8];
    float lmax = -1.0f;
    uint32_t cum[kMaxClasses];
#pragma unroll
    for (int k = 0; k < kMaxClasses; ++k) cum[k] = pre[k];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      sf[q] = -1.0f;
      const int b = b0 + q;
      if (q < bpl && b < B - 1) {
        uint32_t nL = 0;
#pragma unroll
        for (int k = 0; k < kMaxClasses; ++k)
          if (k < C) {
            cum[k] += hw[b * C + k];
            nL += cum[k];
          }
        if (nL > 0u && nL < nd.n) {
          sf[q] = score_class_f(cum, nd.cp, C, nL, nd.n);
          lmax = fmaxf(lmax, sf[q]);
        }
      }
    }
    const float mx = warp_max_f(lmax);
    if (mx < 0.0f) {
      out.valid = false;
      return;
    }
    const float thr = SCREEN(mx);
    // pass 2: exact among the contenders (bins ascending: first of equals kept)
#pragma unroll
    for (int k = 0; k < kMaxClasses; ++k) cum[k] = pre[k];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int b = b0 + q;
      if (q < bpl && b < B - 1) {
        uint32_t nL = 0;
#pragma unroll
        for (int k = 0; k < kMaxClasses; ++k)
          if (k < C) {
            cum[k] += hw[b * C + k];
            nL += cum[k];
          }
        if (sf[q] >= 0.0f && sf[q] >= thr) {
          Cand c;
          cand_class(c, cum, nd.cp, C, nL, nd.n);
          c.feat = feat;
          c.bin = b;
          c.key = (tkey << 8) | static_cast<uint32_t>(b);
          if (cand_better(c, mine)) mine = c;
        }
      }
    }
  } else {
    uint32_t* hn = hw;
    unsigned long long* hs = reinterpret_cast<unsigned long long*>(hw + ((B + 1) & ~1));
    for (int i = lane; i < B; i += 32) {
      hn[i] = 0u;
      hs[i] = 0ull;
    }
    __syncwarp();
    for (uint32_t r = lane; r < nd.len; r += 32) {
      const uint32_t e = rows[nd.base + r];
      const uint32_t row = e >> 8, w = e & 255u;
      const uint32_t b = col[row];
      atomicAdd(&hn[b], w);
      atomicAdd(&hs[b], static_cast<unsigned long long>(static_cast<long long>(w) * d.yreg[row]));
    }
    __syncwarp();
    uint32_t tn = 0;
    long long ts = 0;
    for (int q = 0; q < bpl; ++q) {
      const int b = b0 + q;
      if (b < B) {
        tn += hn[b];
        ts += static_cast<long long>(hs[b]);
      }
    }
    const uint32_t pn = warp_excl_scan_u32(tn, lane);
    const long long ps = warp_excl_scan_i64(ts, lane);
    float sf[8];
    float lmax = -1.0f;
    uint32_t cn = pn;
    long long cs = ps;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      sf[q] = -1.0f;
      const int b = b0 + q;
      if (q < bpl && b < B - 1) {
        cn += hn[b];
        cs += static_cast<long long>(hs[b]);
        if (cn > 0u && cn < nd.n) {
          sf[q] = score_reg_f(cs, nd.SP, cn, nd.n);
          lmax = fmaxf(lmax, sf[q]);
        }
      }
    }
    const float mx = warp_max_f(lmax);
    if (mx < 0.0f) {
      out.valid = false;
      return;
    }
    const float thr = SCREEN(mx);
    cn = pn;
    cs = ps;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int b = b0 + q;
      if (q < bpl && b < B - 1) {
        cn += hn[b];
        cs += static_cast<long long>(hs[b]);
        if (sf[q] >= 0.0f && sf[q] >= thr) {
          Cand c;
          cand_reg(c, cs, nd.SP, cn, nd.n);
          c.feat = feat;
          c.bin = b;
          c.key = (tkey << 8) | static_cast<uint32_t>(b);
          if (cand_better(c, mine)) mine = c;
        }
      }
    }
  }
  warp_select(mine, out, C, reg);
}

// Exact impurity decrease of the chosen split:
//   delta = num/den - A_P/n_P = (num*n_P - A_P*den) / (den*n_P), rounded as
//   RN(numerator) / RN(denominator).  Returns false if delta <= 0.
__device__ bool split_delta(const Cand& c, const NodeInfo& nd, int C, bool reg, int precision,
                            double* delta) {
  u128 AP;
  if (reg) {
    AP = sq_i64(nd.SP);
  } else {
    AP = 0;
    for (int k = 0; k < C; ++k) AP += static_cast<u128>(static_cast<uint64_t>(nd.cp[k]) * nd.cp[k]);
  }
  uint64_t lhs[4], rhs[4];
  mul192x64(c.num, nd.n, lhs);
  const U192 ap = u192_from(AP);
  mul192x64(ap, c.den, rhs);
  if (cmp_limbs4(lhs, rhs) <= 0) return false;
  uint64_t dn[4];
  uint64_t borrow = 0;
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
  if (precision == 0) {
    *delta = limbs_to_double(dn, 4, 0) / limbs_to_double(dl, 2, 0);
  } else {
    *delta = static_cast<double>(__fdiv_rn(limbs_to_float(dn, 4, 0), limbs_to_float(dl, 2, 0)));
  }
  return true;
}

// One CTA per node (claimed dynamically).  Warps take the node's feature
// draw slots in turn; the CTA keeps the best candidate, records the split,
// adds its impurity decrease to the tree's TreeImp accumulator and
// partitions the node's rows (left rows first, right rows last, both in
// order) into the next level's buffer.
__global__ void __launch_bounds__(kSplitThreads) k_split(Dev d, int level) {
  extern __shared__ __align__(16) uint32_t smem[];
  __shared__ Perm sperm;
  __shared__ NodeInfo snd;
  __shared__ Cand swarp[kSplitThreads / 32];
  __shared__ uint32_t snode, ssplit, swl[kSplitThreads / 32], swr[kSplitThreads / 32];
  __shared__ int sact;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const bool reg = d.kind != 0;
  const int C = d.C;
  uint32_t* hw = smem + warp * (split_smem_per_warp(d.kind, C, d.B) / 4);
  const uint32_t* rows_in = d.rows[level & 1];
  uint32_t* rows_out = d.rows[(level & 1) ^ 1];
  const uint32_t lcount = d.lvl_cnt[level], loff = d.lvl_off[level];

  for (;;) {
    if (threadIdx.x == 0) snode = atomicAdd(&d.work[level], 1u);
    __syncthreads();
    const uint32_t idx = snode;
    if (idx >= lcount) break;
    const uint32_t k = loff + idx;
    if (threadIdx.x == 0) {
      NodeInfo nd;
      const uint32_t tau = d.nd_tree[k];
      nd.base = static_cast<int64_t>(tau) * d.N + d.nd_seg[k];
      nd.len = d.nd_len[k];
      nd.n = d.nd_n[k];
      nd.SP = 0;
      bool pure = false;
      if (!reg) {
        for (int c = 0; c < kMaxClasses; ++c) {
          nd.cp[c] = c < C ? d.nd_cnt[static_cast<int64_t>(k) * C + c] : 0u;
          pure |= (c < C) && nd.cp[c] == nd.n;
        }
      } else {
        nd.SP = d.nd_S[k];
      }
      snd = nd;
      const bool act = level < d.D && nd.len >= 2u && !pure;
      sact = act;
      if (act)
        perm_init(sperm, static_cast<uint32_t>(d.p_aug), d.seed, d.nd_heap[k], unit_word(d.t, tau),
                  purpose_word(kPurposeMtry, d.job));
      else
        d.nd_split[k] = kLeaf;
    }
    __syncthreads();
    if (!sact) continue;
    const NodeInfo nd = snd;
    const Perm P = sperm;

    Cand best;
    best.valid = false;
    for (int slot = warp; slot < d.mtry; slot += nw) {
      const int f = static_cast<int>(perm_apply(P, static_cast<uint32_t>(slot)));
      const uint32_t tkey = d.tie_break == 0 ? static_cast<uint32_t>(slot) : static_cast<uint32_t>(f);
      Cand c;
      feature_best(d, nd, rows_in, f, tkey, hw, c);
      if (cand_better(c, best)) best = c;
    }
    if (lane == 0) swarp[warp] = best;
    __syncthreads();
    if (threadIdx.x == 0) {
      Cand b = swarp[0];
      for (int w = 1; w < nw; ++w)
        if (cand_better(swarp[w], b)) b = swarp[w];
      double delta = 0.0;
      uint32_t sp = kLeaf;
      if (b.valid && split_delta(b, nd, C, reg, d.precision, &delta)) {
        sp = (static_cast<uint32_t>(b.feat) << 8) | static_cast<uint32_t>(b.bin);
        d.nd_delta[k] = delta;
        d.nd_ln[k] = b.nL;
        if (reg)
          d.nd_lS[k] = b.SL;
        else
          for (int c = 0; c < C; ++c) d.nd_lcnt[static_cast<int64_t>(k) * C + c] = b.cL[c];
        uint64_t v[kFixLimbs];
        if (!fix_from_double(delta, v)) atomicOr(&d.status[0], kErrAcc);
        if (!d.permut)
          fix_atomic_add(d.acc + (static_cast<int64_t>(d.nd_tree[k]) * d.p_aug + b.feat) * kFixLimbs, v);
      }
      d.nd_split[k] = sp;
      ssplit = sp;
      const unsigned long long ybytes = reg ? 8ull : 1ull;
      atomicAdd(&d.counters[0], static_cast<unsigned long long>(nd.len) * d.mtry +
                                    static_cast<unsigned long long>(nd.len) * (4ull + ybytes) +
                                    (sp != kLeaf ? static_cast<unsigned long long>(nd.len) * 5ull : 0ull));
    }
    __syncthreads();
    const uint32_t sp = ssplit;
    if (sp == kLeaf) continue;

    // ---- stable partition into rows_out[base .. base+len)
    const uint8_t* col = d.colptr[sp >> 8];
    const uint32_t thr = sp & 255u;
    uint32_t lbase = 0, rbase = 0;
    for (uint32_t off = 0; off < nd.len; off += blockDim.x) {
      const uint32_t r = off + threadIdx.x;
      const bool v = r < nd.len;
      const uint32_t e = v ? rows_in[nd.base + r] : 0u;
      const bool gl = v && col[e >> 8] <= thr;
      const bool gr = v && !gl;
      const unsigned bl = __ballot_sync(kFull, gl), br = __ballot_sync(kFull, gr);
      if (lane == 0) {
        swl[warp] = __popc(bl);
        swr[warp] = __popc(br);
      }
      __syncthreads();
      uint32_t pl = 0, pr = 0, tl = 0, tr = 0;
      for (int w = 0; w < nw; ++w) {
        if (w < warp) {
          pl += swl[w];
          pr += swr[w];
        }
        tl += swl[w];
        tr += swr[w];
      }
      if (gl) rows_out[nd.base + lbase + pl + __popc(bl & lanemask_lt())] = e;
      if (gr) rows_out[nd.base + nd.len - 1u - (rbase + pr + __popc(br & lanemask_lt()))] = e;
      lbase += tl;
      rbase += tr;
      __syncthreads();
    }
    if (threadIdx.x == 0) d.nd_lrows[k] = lbase;
  }
}

const void* split_kernel_ptr() { return reinterpret_cast<const void*>(&k_split); }

void launch_split(const Dev& d, int level, int grid, size_t smem, cudaStream_t st) {
  k_split<<<grid, kSplitThreads, smem, st>>>(d, level);
}

// ============================================================ next level
// Children of split node k sit at next_off + 2*rank and +1, rank = number
// of split nodes before k in the level; (tree, heap) order is preserved.
__global__ void k_count(Dev d, int level) {
  __shared__ uint32_t sred[256];
  const uint32_t n = d.lvl_cnt[level], off = d.lvl_off[level];
  const uint32_t chunk = (n + gridDim.x - 1) / gridDim.x;
  const uint32_t lo = blockIdx.x * chunk, hi = min(n, lo + chunk);
  uint32_t c = 0;
  for (uint32_t i = lo + threadIdx.x; i < hi; i += blockDim.x) c += d.nd_split[off + i] != kLeaf;
  const uint32_t tot = block_sum<uint32_t>(c, sred);
  if (threadIdx.x == 0) d.chunk[blockIdx.x] = tot;
}

__global__ void k_children(Dev d, int level) {
  __shared__ uint32_t sw[33];
  __shared__ uint32_t sred[256];
  const uint32_t n = d.lvl_cnt[level], off = d.lvl_off[level];
  const uint32_t chunk = (n + gridDim.x - 1) / gridDim.x;
  uint32_t before = 0, total = 0;
  for (uint32_t b = threadIdx.x; b < gridDim.x; b += blockDim.x) {
    const uint32_t v = d.chunk[b];
    total += v;
    before += b < blockIdx.x ? v : 0u;
  }
  before = block_sum<uint32_t>(before, sred);
  total = block_sum<uint32_t>(total, sred);
  const uint32_t next_off = off + n;
  const uint64_t need = static_cast<uint64_t>(next_off) + 2ull * total;
  if (need > d.cap) {
    // no room for the children: the level's nodes become leaves so that every
    // tree stays well formed (the host reports BORUTA_EOVERFLOW)
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
      d.nd_split[off + i] = kLeaf;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      atomicOr(&d.status[0], kErrPool);
      d.lvl_off[level + 1] = next_off;
      d.lvl_cnt[level + 1] = 0u;
    }
    return;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    d.lvl_off[level + 1] = next_off;
    d.lvl_cnt[level + 1] = 2u * total;
  }
  const uint32_t lo = blockIdx.x * chunk, hi = min(n, lo + chunk);
  uint32_t run = before;
  const bool reg = d.kind != 0;
  const int C = d.C;
  for (uint32_t base = lo; base < hi; base += blockDim.x) {
    const uint32_t i = base + threadIdx.x;
    const uint32_t k = off + i;
    const bool sp = i < hi && d.nd_split[k] != kLeaf;
    uint32_t tot;
    const uint32_t r = block_excl_scan(sp ? 1u : 0u, &tot, sw);
    if (sp) {
      const uint32_t L = next_off + 2u * (run + r), R = L + 1u;
      d.nd_child[k] = L;
      const uint32_t tau = d.nd_tree[k], heap = d.nd_heap[k], seg = d.nd_seg[k];
      const uint32_t len = d.nd_len[k], lrows = d.nd_lrows[k], n_ = d.nd_n[k], ln = d.nd_ln[k];
      d.nd_tree[L] = tau;
      d.nd_tree[R] = tau;
      d.nd_heap[L] = 2u * heap + 1u;
      d.nd_heap[R] = 2u * heap + 2u;
      d.nd_seg[L] = seg;
      d.nd_seg[R] = seg + lrows;
      d.nd_len[L] = lrows;
      d.nd_len[R] = len - lrows;
      d.nd_n[L] = ln;
      d.nd_n[R] = n_ - ln;
      if (reg) {
        const long long sl = d.nd_lS[k];
        d.nd_S[L] = sl;
        d.nd_S[R] = d.nd_S[k] - sl;
      } else {
        for (int c = 0; c < C; ++c) {
          const uint32_t lc = d.nd_lcnt[static_cast<int64_t>(k) * C + c];
          d.nd_cnt[static_cast<int64_t>(L) * C + c] = lc;
          d.nd_cnt[static_cast<int64_t>(R) * C + c] = d.nd_cnt[static_cast<int64_t>(k) * C + c] - lc;
        }
      }
      d.nd_split[L] = kLeaf;
      d.nd_split[R] = kLeaf;
      d.nd_child[L] = 0u;
      d.nd_child[R] = 0u;
      d.nd_delta[L] = 0.0;
      d.nd_delta[R] = 0.0;
    }
    run += tot;
  }
}

void launch_children(const Dev& d, int level, cudaStream_t st) {
  k_count<<<kScanBlocks, 256, 0, st>>>(d, level);
  k_children<<<kScanBlocks, 256, 0, st>>>(d, level);
}

// ============================================================ Alg. 2 normalisation
// imp[tau][j] = g_j / sum_j g_j with g_j = RN(exact sum of the tree's
// impurity decreases on feature j) and the total summed exactly.
__global__ void k_treeimp_norm(Dev d) {
  __shared__ unsigned long long sacc[256 * kFixLimbs];
  for (int tau = blockIdx.x; tau < d.M; tau += gridDim.x) {
    uint64_t a[kFixLimbs];
#pragma unroll
    for (int i = 0; i < kFixLimbs; ++i) a[i] = 0;
    bool bad = false;
    for (int j = threadIdx.x; j < d.p_aug; j += blockDim.x) {
      const unsigned long long* src = d.acc + (static_cast<int64_t>(tau) * d.p_aug + j) * kFixLimbs;
      uint64_t g[kFixLimbs];
#pragma unroll
      for (int i = 0; i < kFixLimbs; ++i) g[i] = src[i];
      const double gj = d.precision == 0 ? fix_to_double(g) : static_cast<double>(fix_to_float(g));
      d.imp[static_cast<int64_t>(tau) * d.p_aug + j] = gj;
      uint64_t v[kFixLimbs];
      bad |= !fix_from_double(gj, v);
      fix_add(a, v);
    }
    if (bad) atomicOr(&d.status[0], kErrAcc);
#pragma unroll
    for (int i = 0; i < kFixLimbs; ++i) sacc[threadIdx.x * kFixLimbs + i] = a[i];
    __syncthreads();
    for (int s = blockDim.x >> 1; s > 0; s >>= 1) {
      if (threadIdx.x < s) {
        uint64_t x[kFixLimbs], y[kFixLimbs];
#pragma unroll
        for (int i = 0; i < kFixLimbs; ++i) {
          x[i] = sacc[threadIdx.x * kFixLimbs + i];
          y[i] = sacc[(threadIdx.x + s) * kFixLimbs + i];
        }
        fix_add(x, y);
#pragma unroll
        for (int i = 0; i < kFixLimbs; ++i) sacc[threadIdx.x * kFixLimbs + i] = x[i];
      }
      __syncthreads();
    }
    uint64_t tot[kFixLimbs];
#pragma unroll
    for (int i = 0; i < kFixLimbs; ++i) tot[i] = sacc[i];
    __syncthreads();
    if (d.precision == 0) {
      const double T = fix_to_double(tot);
      for (int j = threadIdx.x; j < d.p_aug; j += blockDim.x) {
        double* x = d.imp + static_cast<int64_t>(tau) * d.p_aug + j;
        *x = T > 0.0 ? *x / T : 0.0;
      }
    } else {
      const float T = fix_to_float(tot);
      for (int j = threadIdx.x; j < d.p_aug; j += blockDim.x) {
        double* x = d.imp + static_cast<int64_t>(tau) * d.p_aug + j;
        *x = T > 0.0f ? static_cast<double>(__fdiv_rn(static_cast<float>(*x), T)) : 0.0;
      }
    }
  }
}

void launch_treeimp(const Dev& d, int grid, cudaStream_t st) {
  k_treeimp_norm<<<grid, 256, 0, st>>>(d);
}

// ============================================================ Alg. 3 on OOB rows
__device__ __forceinline__ uint32_t leaf_of(const Dev& d, uint32_t k, uint32_t row, int f,
                                            uint8_t xf) {
  for (int guard = 0; guard <= kMaxDepth; ++guard) {  // trees are at most kMaxDepth deep
    const uint32_t sp = d.nd_split[k];
    if (sp == kLeaf) return k;
    const int g = static_cast<int>(sp >> 8);
    const uint8_t x = (g == f) ? xf : d.colptr[g][row];
    k = d.nd_child[k] + (x > (sp & 255u) ? 1u : 0u);
  }
  return k;
}

// loss between the unpermuted leaf q and the permuted leaf q2
__device__ double loss64(const Dev& d, uint32_t q, uint32_t q2) {
  const double na = static_cast<double>(d.nd_n[q]), nb = static_cast<double>(d.nd_n[q2]);
  if (d.kind != 0) {
    const double ma = static_cast<double>(d.nd_S[q]) / na, mb = static_cast<double>(d.nd_S[q2]) / nb;
    const double df = (ma - mb) * 0x1p-20;
    return df * df;
  }
  const double eps = d.kl_eps;
  const double norm = 1.0 + static_cast<double>(d.C) * eps;
  double kl = 0.0;
  for (int c = 0; c < d.C; ++c) {
    const double pa = (static_cast<double>(d.nd_cnt[static_cast<int64_t>(q) * d.C + c]) / na + eps) / norm;
    const double pb = (static_cast<double>(d.nd_cnt[static_cast<int64_t>(q2) * d.C + c]) / nb + eps) / norm;
    kl += pa * log(pa / pb);
  }
  return kl;
}

// phi(r) = r log r - r + 1 >= 0, accurate near r = 1 (series in r - 1)
__device__ __forceinline__ float kl_phi(float r) {
  const float dl = r - 1.0f;
  if (fabsf(dl) < 0.25f) {
    // sum_{n>=2} (-1)^n dl^n / (n (n-1))
    float s = 0.0f, pw = dl * dl;
#pragma unroll
    for (int n = 2; n <= 14; ++n) {
      const float term = pw / static_cast<float>(n * (n - 1));
      s += (n & 1) ? -term : term;
      pw *= dl;
    }
    return s;
  }
  return r * logf(r) - dl;
}

__device__ float loss32(const Dev& d, uint32_t q, uint32_t q2) {
  const uint32_t na = d.nd_n[q], nb = d.nd_n[q2];
  if (d.kind != 0) {
    // mean difference from exact integers: (S_a n_b - S_b n_a) / (n_a n_b)
    const __int128 num = static_cast<__int128>(d.nd_S[q]) * nb - static_cast<__int128>(d.nd_S[q2]) * na;
    const u128 mag = num < 0 ? static_cast<u128>(-num) : static_cast<u128>(num);
    const uint64_t ml[2] = {static_cast<uint64_t>(mag), static_cast<uint64_t>(mag >> 64)};
    const uint64_t den = static_cast<uint64_t>(na) * nb;
    const float df = __fdiv_rn(limbs_to_float(ml, 2, -20), limbs_to_float(&den, 1, 0));
    return df * df;
  }
  const float eps = static_cast<float>(d.kl_eps);
  const float norm = 1.0f + static_cast<float>(d.C) * eps;
  float kl = 0.0f;
  for (int c = 0; c < d.C; ++c) {
    const float pa = __fdiv_rn(__fdiv_rn(static_cast<float>(d.nd_cnt[static_cast<int64_t>(q) * d.C + c]),
                                         static_cast<float>(na)) + eps, norm);
    const float pb = __fdiv_rn(__fdiv_rn(static_cast<float>(d.nd_cnt[static_cast<int64_t>(q2) * d.C + c]),
                                         static_cast<float>(nb)) + eps, norm);
    kl += pb * kl_phi(__fdiv_rn(pa, pb));
  }
  return kl;
}

// One thread per (tree, OOB row): walk the row's path; for each distinct
// feature f on it, re-walk from f's first node with x_f replaced by
// X[pi(i)][f] (all later f nodes use the swapped value too).  Features off
// the path leave the leaf unchanged and add exactly 0.
__global__ void k_permut(Dev d) {
  __shared__ Perm sp;
  if (threadIdx.x == 0)
    perm_init(sp, static_cast<uint32_t>(d.N), d.seed, 0u, unit_word(d.t, 0u),
              purpose_word(kPurposePermut, d.job));
  __syncthreads();
  const Perm P = sp;
  for (int tau = blockIdx.y; tau < d.M; tau += gridDim.y) {
    const uint32_t noob = d.oob_cnt[tau];
    const uint32_t* oob = d.oob + static_cast<int64_t>(tau) * d.N;
    for (uint32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < noob; r += gridDim.x * blockDim.x) {
      const uint32_t i = oob[r];
      const uint32_t pi = perm_apply(P, i);
      uint32_t path[kMaxDepth];
      int depth = 0;
      uint32_t k = static_cast<uint32_t>(tau);
      while (depth < kMaxDepth) {
        const uint32_t s = d.nd_split[k];
        if (s == kLeaf) break;
        path[depth++] = k;
        const uint8_t x = d.colptr[s >> 8][i];
        k = d.nd_child[k] + (x > (s & 255u) ? 1u : 0u);
      }
      const uint32_t q = k;
      for (int a = 0; a < depth; ++a) {
        const int f = static_cast<int>(d.nd_split[path[a]] >> 8);
        bool seen = false;
        for (int b = 0; b < a; ++b) seen |= static_cast<int>(d.nd_split[path[b]] >> 8) == f;
        if (seen) continue;
        const uint8_t xp = d.colptr[f][pi];
        const uint32_t q2 = leaf_of(d, path[a], i, f, xp);
        if (q2 == q) continue;
        const double L = d.precision == 0 ? loss64(d, q, q2) : static_cast<double>(loss32(d, q, q2));
        uint64_t v[kFixLimbs];
        if (!fix_from_double(L, v)) {
          atomicOr(&d.status[0], kErrAcc);
          continue;
        }
        fix_atomic_add(d.acc + (static_cast<int64_t>(tau) * d.p_aug + f) * kFixLimbs, v);
      }
    }
  }
}

__global__ void k_permut_final(Dev d) {
  const int64_t total = static_cast<int64_t>(d.M) * d.p_aug;
  for (int64_t g = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; g < total;
       g += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int tau = static_cast<int>(g / d.p_aug);
    const uint32_t n = d.oob_cnt[tau];
    uint64_t a[kFixLimbs];
#pragma unroll
    for (int i = 0; i < kFixLimbs; ++i) a[i] = d.acc[g * kFixLimbs + i];
    double v = 0.0;
    if (n > 0) {
      if (d.precision == 0)
        v = fix_to_double(a) / static_cast<double>(n);
      else
        v = static_cast<double>(__fdiv_rn(fix_to_float(a), static_cast<float>(n)));
    }
    d.imp[g] = v;
  }
}

void launch_permut(const Dev& d, int grid, cudaStream_t st) {
  int by = d.M < 4096 ? d.M : 4096;
  int bx = grid / by;
  if (bx < 1) bx = 1;
  k_permut<<<dim3(bx, by), 128, 0, st>>>(d);
  k_permut_final<<<grid, 256, 0, st>>>(d);
}

// ============================================================ Alg. 1: statistic, hits, test
// s_j over trees, exact sums rounded once:
//   mean = RN(sum imp)/M,  sd = sqrt(RN(sum (imp - mean)^2)/(M-1)),  Z = mean/(sd/sqrt(M))
__global__ void k_stats(Dev d) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < d.p_aug; j += gridDim.x * blockDim.x) {
    uint64_t a[kFixLimbs], v[kFixLimbs];
#pragma unroll
    for (int i = 0; i < kFixLimbs; ++i) a[i] = 0;
    bool bad = false;
    for (int tau = 0; tau < d.M; ++tau) {
      bad |= !fix_from_double(d.imp[static_cast<int64_t>(tau) * d.p_aug + j], v);
      fix_add(a, v);
    }
    const double mean = fix_to_double(a) / static_cast<double>(d.M);
    double sd = 0.0;
    if (d.M > 1) {
#pragma unroll
      for (int i = 0; i < kFixLimbs; ++i) a[i] = 0;
      for (int tau = 0; tau < d.M; ++tau) {
        const double dl = d.imp[static_cast<int64_t>(tau) * d.p_aug + j] - mean;
        bad |= !fix_from_double(dl * dl, v);
        fix_add(a, v);
      }
      sd = sqrt(fix_to_double(a) / static_cast<double>(d.M - 1));
    }
    double z;
    if (sd == 0.0)
      z = (mean == 0.0) ? 0.0 : __longlong_as_double(0x7FF0000000000000ll);
    else
      z = mean / (sd / sqrt(static_cast<double>(d.M)));
    d.s[j] = d.stat == 1 ? mean : z;
    if (bad) atomicOr(&d.status[0], kErrAcc);
  }
}

// u128 -> double, correctly rounded
__device__ __forceinline__ double u128_to_double(u128 v) {
  const uint64_t w[2] = {static_cast<uint64_t>(v), static_cast<uint64_t>(v >> 64)};
  return limbs_to_double(w, 2, 0);
}

__global__ void k_decide(Dev d) {
  __shared__ double smx[1024];
  __shared__ uint32_t scnt[1024];
  double mx = -__longlong_as_double(0x7FF0000000000000ll);
  for (int c = d.p_live + threadIdx.x; c < d.p_aug; c += blockDim.x) mx = fmax(mx, d.s[c]);
  smx[threadIdx.x] = mx;
  __syncthreads();
  for (int s = blockDim.x >> 1; s > 0; s >>= 1) {
    if (threadIdx.x < s) smx[threadIdx.x] = fmax(smx[threadIdx.x], smx[threadIdx.x + s]);
    __syncthreads();
  }
  const double smax = smx[0];
  const int t = d.t;
  if (threadIdx.x == 0) d.smax[t - 1] = smax;
  for (int a = threadIdx.x; a < d.p_live; a += blockDim.x) {
    const int j = d.live[a];
    const double v = d.s[a];
    d.hist[static_cast<int64_t>(t - 1) * d.p + j] = v;
    if (v > smax) d.hits[j] += 1;
  }
  uint32_t m = 0;
  for (int j = threadIdx.x; j < d.p; j += blockDim.x) m += d.state[j] == 0;
  scnt[threadIdx.x] = m;
  __syncthreads();
  for (int s = blockDim.x >> 1; s > 0; s >>= 1) {
    if (threadIdx.x < s) scnt[threadIdx.x] += scnt[threadIdx.x + s];
    __syncthreads();
  }
  const uint32_t mu = scnt[0];
  __syncthreads();
  const double thr = d.alpha / static_cast<double>(mu);
  const u128* row = d.pascal + static_cast<int64_t>(t) * 127;
  uint32_t und = 0;
  for (int j = threadIdx.x; j < d.p; j += blockDim.x) {
    if (d.state[j] != 0) continue;
    const int h = d.hits[j];
    u128 up = 0, lo = 0;
    for (int k = 0; k <= t; ++k) {
      if (k >= h) up += row[k];
      if (k <= h) lo += row[k];
    }
    const double pa = scalbn(u128_to_double(up), -t), pr = scalbn(u128_to_double(lo), -t);
    if (pa < thr)
      d.state[j] = 1;
    else if (pr < thr)
      d.state[j] = -1;
    else
      ++und;
  }
  scnt[threadIdx.x] = und;
  __syncthreads();
  for (int s = blockDim.x >> 1; s > 0; s >>= 1) {
    if (threadIdx.x < s) scnt[threadIdx.x] += scnt[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) d.status[1] = scnt[0];
}

void launch_stats_decide(const Dev& d, cudaStream_t st) {
  k_stats<<<(d.p_aug + 127) / 128, 128, 0, st>>>(d);
  k_decide<<<1, 1024, 0, st>>>(d);
}

// ============================================================ primitives for parity checks
__global__ void k_dbg_philox(const uint32_t* ctr, const uint32_t* key, uint32_t* out, int64_t n) {
  const uint2 k = make_uint2(key[0], key[1]);
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const uint4 o = philox10(make_uint4(ctr[4 * i], ctr[4 * i + 1], ctr[4 * i + 2], ctr[4 * i + 3]), k);
    out[4 * i] = o.x;
    out[4 * i + 1] = o.y;
    out[4 * i + 2] = o.z;
    out[4 * i + 3] = o.w;
  }
}

__global__ void k_dbg_perm(uint32_t n, uint64_t seed, uint32_t w1, uint32_t w2, uint32_t w3,
                           const uint64_t* idx, uint64_t* out, int64_t count) {
  Perm P;
  perm_init(P, n, seed, w1, w2, w3);
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < count;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x)
    out[i] = perm_apply(P, static_cast<uint32_t>(idx[i]));
}

__global__ void k_dbg_u256(const uint64_t* v, double* out, int64_t n) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    uint64_t w[4] = {v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]};
    out[i] = limbs_to_double(w, 4, 0);
  }
}

__global__ void k_dbg_binom(const u128* pascal, const int32_t* t, const int32_t* h, double* pa,
                            double* pr, int64_t n) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int tt = t[i], hh = h[i];
    const u128* row = pascal + static_cast<int64_t>(tt) * 127;
    u128 up = 0, lo = 0;
    for (int k = 0; k <= tt; ++k) {
      if (k >= hh) up += row[k];
      if (k <= hh) lo += row[k];
    }
    pa[i] = scalbn(u128_to_double(up), -tt);
    pr[i] = scalbn(u128_to_double(lo), -tt);
  }
}

static int grid_for(int64_t n) {
  int64_t g = (n + 255) / 256;
  if (g < 1) g = 1;
  if (g > 4096) g = 4096;
  return static_cast<int>(g);
}

void launch_debug_philox(const uint32_t* ctr, const uint32_t* key, uint32_t* out, int64_t n,
                         cudaStream_t st) {
  k_dbg_philox<<<grid_for(n), 256, 0, st>>>(ctr, key, out, n);
}
void launch_debug_perm(uint32_t n, uint64_t seed, uint32_t w1, uint32_t w2, uint32_t w3,
                       const uint64_t* idx, uint64_t* out, int64_t count, cudaStream_t st) {
  k_dbg_perm<<<grid_for(count), 256, 0, st>>>(n, seed, w1, w2, w3, idx, out, count);
}
void launch_debug_u256(const uint64_t* v, double* out, int64_t n, cudaStream_t st) {
  k_dbg_u256<<<grid_for(n), 256, 0, st>>>(v, out, n);
}
void launch_debug_binom(const u128* pascal, const int32_t* t, const int32_t* h, double* pa,
                        double* pr, int64_t n, cudaStream_t st) {
  k_dbg_binom<<<grid_for(n), 256, 0, st>>>(pascal, t, h, pa, pr, n);
}

}  // namespace bgb
