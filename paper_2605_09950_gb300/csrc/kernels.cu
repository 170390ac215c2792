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

#ifndef BORUTA_PERMUT_WALKS
#define BORUTA_PERMUT_WALKS 8  // re-walks of one OOB row advanced together
#endif

namespace bgb {

namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;

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
  uint32_t maxlab = 0, maxbin = 0;
  for (int j = blockIdx.y; j < d.p; j += gridDim.y) {
    const uint8_t* col = d.X + static_cast<int64_t>(j) * d.ld;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < d.N; i += gridDim.x * blockDim.x) {
      const uint32_t b = col[i];
      bad |= b >= static_cast<uint32_t>(d.B);
      maxbin = max(maxbin, b);
    }
  }
  if (maxbin) atomicMax(&d.status[3], maxbin);
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
// X_cur into the augmented matrix: Xaug[a] = X[live[a]] (16-byte copies when
// the caller's columns allow it).  The augmented columns then sit at a fixed
// stride, so every kernel addresses column f as Xaug + f * ldN.
__global__ void k_gather_live(Dev d, int vec) {
  const int a = blockIdx.y;
  const uint8_t* src = d.X + static_cast<int64_t>(d.live[a]) * d.ld;
  uint8_t* dst = d.Xaug + static_cast<int64_t>(a) * d.ldN;
  if (vec) {
    const uint4* s = reinterpret_cast<const uint4*>(src);
    uint4* t = reinterpret_cast<uint4*>(dst);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < d.ldN / 16; i += gridDim.x * blockDim.x) t[i] = s[i];
  } else {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < d.N; i += gridDim.x * blockDim.x) dst[i] = src[i];
  }
}

int launch_gather_live(const Dev& d, cudaStream_t st) {
  // 16-byte path: aligned base, ld a multiple of 16 and at least ldN bytes per column
  const int vec = (reinterpret_cast<uintptr_t>(d.X) % 16 == 0) && (d.ld % 16 == 0) && (d.ld >= d.ldN);
  int bx = ((vec ? d.ldN / 16 : d.N) + 255) / 256;
  if (bx > 16) bx = 16;
  k_gather_live<<<dim3(bx, d.p_live), 256, 0, st>>>(d, vec);
  return 1;
}

// Xaug[p_live + c][i] = X[sigma_c(i)][live[c mod p_live]]; 16 rows per thread, one
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
  uint8_t* dst = d.Xaug + static_cast<int64_t>(d.p_live + c) * d.ldN;
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

int launch_shadow(const Dev& d, cudaStream_t st) {
  int bx = (d.N + 16 * 256 - 1) / (16 * 256);
  if (bx > 32) bx = 32;
  k_shadow<<<dim3(bx, d.n_sha), 256, 0, st>>>(d);
  return 1;
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
      // entry low byte: classification y << 5 | count (count < 32), regression count (< 256)
      wbad |= c > (d.kind == 0 ? 31u : 255u);
      uint32_t tin, tout;
      const uint32_t rin = block_excl_scan(in ? 1u : 0u, &tin, sw);
      const uint32_t rout = block_excl_scan(out ? 1u : 0u, &tout, sw);
      if (in) {
        if (d.kind == 0)
          rows[nin + rin] = (static_cast<uint32_t>(i) << 8) | (static_cast<uint32_t>(d.ycls[i]) << 5) | min(c, 31u);
        else
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

int launch_bootstrap(const Dev& d, int grid, cudaStream_t st) {
  int bx = (d.N + 255) / 256;
  if (bx > 64) bx = 64;
  int by = d.M < 4096 ? d.M : 4096;
  k_boot_count<<<dim3(bx, by), 256, 0, st>>>(d);
  k_boot_compact<<<grid, 256, 0, st>>>(d);
  return 2;
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

int launch_children(const Dev& d, int level, cudaStream_t st) {
  k_count<<<kScanBlocks, 256, 0, st>>>(d, level);
  k_children<<<kScanBlocks, 256, 0, st>>>(d, level);
  return 2;
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
      uint64_t g[kFixLimbs];
      csa_to_fix(d.acc + (static_cast<int64_t>(tau) * d.p_aug + j) * kCsaLimbs, g);
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

int launch_treeimp(const Dev& d, int grid, cudaStream_t st) {
  k_treeimp_norm<<<grid, 256, 0, st>>>(d);
  return 1;
}

// ============================================================ Alg. 3 on OOB rows
// (split, child) of every node of the iteration's trees in one array, so that
// a walk step loads both children's words with two 8-byte loads.
__global__ void k_pack_nodes(Dev d) {
  const uint32_t total = d.lvl_off[d.D] + d.lvl_cnt[d.D];
  for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < total; k += gridDim.x * blockDim.x)
    d.nd_sc[k] = make_uint2(d.nd_split[k], d.nd_child[k]);
}

// Row-major copy of the augmented matrix for the tree walks: Xrow[i][f] =
// Xaug[f][i].  One 64 x 64 tile per block through shared memory: the reads
// run along the rows of a column, the writes along the columns of a row.
__global__ void __launch_bounds__(256) k_transpose_rows(Dev d) {
  __shared__ uint8_t tile[64][65];
  const int tiles_i = (d.N + 63) / 64, tiles_f = (d.p_aug + 63) / 64;
  for (int t = blockIdx.x; t < tiles_i * tiles_f; t += gridDim.x) {
    const int i0 = (t % tiles_i) * 64, f0 = (t / tiles_i) * 64;
    for (int k = threadIdx.x; k < 64 * 64; k += blockDim.x) {
      const int f = k >> 6, i = k & 63;
      if (f0 + f < d.p_aug && i0 + i < d.N) tile[f][i] = d.Xaug[static_cast<int64_t>(f0 + f) * d.ldN + i0 + i];
    }
    __syncthreads();
    for (int k = threadIdx.x; k < 64 * 64; k += blockDim.x) {
      const int i = k >> 6, f = k & 63;
      if (f0 + f < d.p_aug && i0 + i < d.N) d.Xrow[static_cast<int64_t>(i0 + i) * d.ldP + f0 + f] = tile[f][i];
    }
    __syncthreads();
  }
}

// flush_index of the iteration (Alg. 3): one keyed permutation of the rows,
// shared by every feature and tree
__global__ void k_permut_pi(Dev d) {
  __shared__ Perm sp;
  if (threadIdx.x == 0)
    perm_init(sp, static_cast<uint32_t>(d.N), d.seed, 0u, unit_word(d.t, 0u), purpose_word(kPurposePermut, d.job));
  __syncthreads();
  const Perm P = sp;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < static_cast<uint32_t>(d.N);
       i += gridDim.x * blockDim.x)
    d.piv[i] = perm_apply(P, i);
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
    // dl^2 * sum_{n=2..14} (-1)^n dl^(n-2) / (n (n-1)), by Horner
    constexpr float c[13] = {1.0f / 2,   -1.0f / 6,   1.0f / 12,   -1.0f / 20,  1.0f / 30,
                             -1.0f / 42, 1.0f / 56,   -1.0f / 72,  1.0f / 90,   -1.0f / 110,
                             1.0f / 132, -1.0f / 156, 1.0f / 182};
    float s = c[12];
#pragma unroll
    for (int m = 11; m >= 0; --m) s = s * dl + c[m];
    return s * (dl * dl);
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
// The re-walks of a warp's 32 rows are pooled in the warp's shared memory
// and dealt round-robin to its lanes, kWalks at a time per lane, so that a
// lane whose row has few re-walks takes over those of a row with many.
// Work items are (tree, chunk of 128 OOB rows), dealt round-robin to a grid
// of exactly the blocks the GPU holds at once, so no partial last wave.
// PREC: the precision form (0 = FP64 terms, 1 = FP32 terms), a template
// argument so that each instantiation holds one loss routine.
__host__ __device__ inline size_t permut_smem_per_warp(int D) {
  // walk pool: start node and feature << 8 | swapped bin (32 * D each), the
  // owning lane (32 * D bytes), then each lane's row and base leaf
  return static_cast<size_t>(32 * D) * 9 + 64 * 4;
}

template <int PREC>
__global__ void __launch_bounds__(128) k_permut(Dev d) {
  extern __shared__ __align__(16) uint32_t pool[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int cap = 32 * d.D;
  uint32_t* q_node = pool + warp * (permut_smem_per_warp(d.D) / 4);
  uint32_t* q_fx = q_node + cap;
  uint32_t* o_row = q_fx + cap;
  uint32_t* o_leaf = o_row + 32;
  uint8_t* q_own = reinterpret_cast<uint8_t*>(o_leaf + 32);
  const uint32_t chunks = (static_cast<uint32_t>(d.N) + 127u) / 128u;
  const uint64_t items = static_cast<uint64_t>(d.M) * chunks;
  unsigned long long visits = 0;  // nodes whose test a walk applied (the base path and the re-walks)
  constexpr int kWalks = BORUTA_PERMUT_WALKS;
  for (uint64_t item = blockIdx.x; item < items; item += gridDim.x) {
    const int tau = static_cast<int>(item / chunks);
    const uint32_t noob = d.oob_cnt[tau];
    const uint32_t r0 = static_cast<uint32_t>(item - static_cast<uint64_t>(tau) * chunks) * 128u;
    if (r0 >= noob) continue;  // block-uniform
    const uint32_t* oob = d.oob + static_cast<int64_t>(tau) * d.N;
    const uint32_t r = r0 + threadIdx.x;
    uint32_t i = 0u, q = 0u;
    int nw = 0;
    uint32_t wnode[kMaxDepth];  // node at which the swapped row leaves the path
    uint32_t wfx[kMaxDepth];    // feature << 8 | swapped bin
    if (r < noob) {
      i = oob[r];
      const uint32_t pi = d.piv[i];
      const uint8_t* xi = d.Xrow + static_cast<int64_t>(i) * d.ldP;    // the row's bins, row-major
      const uint8_t* xpi = d.Xrow + static_cast<int64_t>(pi) * d.ldP;  // the flush_index row's bins
      // the row's path: node, split word, and the row's own bin at each node;
      // the children's words are loaded with the bin (one round trip a level)
      uint32_t path[kMaxDepth], pw[kMaxDepth];
      uint8_t px[kMaxDepth];
      int depth = 0;
      uint32_t k = static_cast<uint32_t>(tau);
      const uint2 root = d.nd_sc[k];
      uint32_t s = root.x, c = root.y;
      while (depth < kMaxDepth && s != kLeaf) {
        const uint8_t x = xi[s >> 8];
        const uint2 n0 = d.nd_sc[c], n1 = d.nd_sc[c + 1];
        path[depth] = k;
        pw[depth] = s;
        px[depth] = x;
        ++depth;
        const bool right = x > (s & 255u);
        k = c + (right ? 1u : 0u);
        s = right ? n1.x : n0.x;
        c = right ? n1.y : n0.y;
      }
      q = k;
      visits += static_cast<unsigned long long>(depth);
      // the permuted row's bins of every feature on the path, loaded together
      uint8_t xq[kMaxDepth];
      for (int a = 0; a < depth; ++a) xq[a] = xpi[pw[a] >> 8];
      // the re-walks: for each distinct feature f on the path whose swapped
      // value sends the row the other way at some node testing f, the walk
      // restarts at that node's other child
      for (int a = 0; a < depth; ++a) {
        const uint32_t f = pw[a] >> 8;
        bool seen = false;
        for (int b = 0; b < a; ++b) seen |= (pw[b] >> 8) == f;
        if (seen) continue;
        const uint8_t xp = xq[a];
        if (xp == px[a]) continue;  // same value: same leaf
        // The swapped row follows the recorded path until the first node on
        // it that tests f and sends xp the other way; if there is none it
        // reaches the same leaf (loss exactly 0).
        int b = a;
        for (; b < depth; ++b)
          if ((pw[b] >> 8) == f && ((xp > (pw[b] & 255u)) != (px[b] > (pw[b] & 255u)))) break;
        if (b == depth) continue;
        wnode[nw] = d.nd_sc[path[b]].y + ((xp > (pw[b] & 255u)) ? 1u : 0u);
        wfx[nw] = (f << 8) | xp;
        ++nw;
      }
    }
    // pool the warp's re-walks (nw <= depth <= D per lane)
    const uint32_t off = warp_excl_scan_u32(static_cast<uint32_t>(nw), lane);
    const uint32_t W = __shfl_sync(kFull, off + static_cast<uint32_t>(nw), 31);
    for (int j = 0; j < nw; ++j) {
      q_node[off + j] = wnode[j];
      q_fx[off + j] = wfx[j];
      q_own[off + j] = static_cast<uint8_t>(lane);
    }
    o_row[lane] = i;
    o_leaf[lane] = q;
    __syncwarp();
    // kWalks re-walks per lane advance together (independent loads in flight)
    for (uint32_t e0 = 0; e0 < W; e0 += 32u * kWalks) {
      uint32_t wk[kWalks], ws[kWalks], wc[kWalks], fx[kWalks];
      const uint8_t* xr[kWalks];
#pragma unroll
      for (int u = 0; u < kWalks; ++u) {
        const uint32_t e = e0 + static_cast<uint32_t>(u) * 32u + lane;
        wk[u] = 0u;
        ws[u] = kLeaf;
        wc[u] = 0u;
        fx[u] = 0u;
        xr[u] = d.Xrow;
        if (e < W) {
          wk[u] = q_node[e];
          fx[u] = q_fx[e];
          xr[u] = d.Xrow + static_cast<int64_t>(o_row[q_own[e]]) * d.ldP;
        }
      }
#pragma unroll
      for (int u = 0; u < kWalks; ++u)
        if (e0 + static_cast<uint32_t>(u) * 32u + lane < W) {
          const uint2 n = d.nd_sc[wk[u]];
          ws[u] = n.x;
          wc[u] = n.y;
        }
      for (int guard = 0; guard <= kMaxDepth; ++guard) {  // trees are at most kMaxDepth deep
        bool busy = false;
#pragma unroll
        for (int u = 0; u < kWalks; ++u) {
          if (ws[u] == kLeaf) continue;
          busy = true;
          ++visits;
          const uint32_t g = ws[u] >> 8;
          const uint8_t x = (g == (fx[u] >> 8)) ? static_cast<uint8_t>(fx[u] & 255u) : xr[u][g];
          const uint32_t c = wc[u];
          const uint2 n0 = d.nd_sc[c], n1 = d.nd_sc[c + 1];
          const bool right = x > (ws[u] & 255u);
          wk[u] = c + (right ? 1u : 0u);
          ws[u] = right ? n1.x : n0.x;
          wc[u] = right ? n1.y : n0.y;
        }
        if (!busy) break;
      }
      // the losses, unrolled: the leaves' statistics of the kWalks re-walks
      // load together
#pragma unroll
      for (int u = 0; u < kWalks; ++u) {
        const uint32_t e = e0 + static_cast<uint32_t>(u) * 32u + lane;
        if (e >= W) continue;
        const uint32_t qo = o_leaf[q_own[e]];
        if (wk[u] == qo) continue;
        const double L = PREC == 0 ? loss64(d, qo, wk[u]) : static_cast<double>(loss32(d, qo, wk[u]));
        if (!csa_add(d.acc + (static_cast<int64_t>(tau) * d.p_aug + (fx[u] >> 8)) * kCsaLimbs, L))
          atomicOr(&d.status[0], kErrAcc);
      }
    }
    __syncwarp();  // the pool is refilled by the next item
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) visits += __shfl_xor_sync(kFull, visits, off);
  if ((threadIdx.x & 31) == 0 && visits) atomicAdd(&d.counters[3], visits);
}

__global__ void k_permut_final(Dev d) {
  const int64_t total = static_cast<int64_t>(d.M) * d.p_aug;
  for (int64_t g = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; g < total;
       g += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int tau = static_cast<int>(g / d.p_aug);
    const uint32_t n = d.oob_cnt[tau];
    uint64_t a[kFixLimbs];
    csa_to_fix(d.acc + g * kCsaLimbs, a);
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

int launch_permut(const Dev& d, int grid, int walk_grid, cudaStream_t st) {
  k_permut_pi<<<(d.N + 255) / 256 < 1024 ? (d.N + 255) / 256 : 1024, 256, 0, st>>>(d);
  k_pack_nodes<<<grid, 256, 0, st>>>(d);
  const size_t smem = 4 * permut_smem_per_warp(d.D);
  if (d.precision == 0)
    k_permut<0><<<walk_grid, 128, smem, st>>>(d);
  else
    k_permut<1><<<walk_grid, 128, smem, st>>>(d);
  k_permut_final<<<grid, 256, 0, st>>>(d);
  return 4;
}

int launch_transpose(const Dev& d, int grid, cudaStream_t st) {
  k_transpose_rows<<<grid, 256, 0, st>>>(d);
  return 1;
}

size_t permut_smem_bytes(int D) { return 4 * permut_smem_per_warp(D); }

const void* permut_kernel_ptr(int precision) {
  return precision == 0 ? reinterpret_cast<const void*>(&k_permut<0>) : reinterpret_cast<const void*>(&k_permut<1>);
}

// ============================================================ Alg. 3 as printed: all rows, forest
// The model is the whole forest: a row's prediction is the mean over the M
// trees of its leaf's value (class fractions c_k/n, or the leaf mean S/n in
// units of 2^-20).  Per row, the exact sum of the per-tree values (carry-save
// fixed point) is kept in fbase; for a block of rows, facc holds per (row,
// column f) the exact sum over the trees whose leaf changes when the row's
// value of f is read at flush_index of (value of the new leaf - value of the
// old leaf), so base + delta is exactly the sum over every tree of the
// permuted prediction.  Each mean is that exact sum rounded once, then
// divided by M (IEEE), and the per-row losses are summed exactly per column.

__device__ __forceinline__ double leaf_value(const Dev& d, uint32_t q, int k) {
  const double n = static_cast<double>(d.nd_n[q]);
  return d.kind != 0 ? static_cast<double>(d.nd_S[q]) / n
                     : static_cast<double>(d.nd_cnt[static_cast<int64_t>(q) * d.C + k]) / n;
}

// leaf of tree tau for row i (column f, if >= 0, read at row pi instead)
__device__ __forceinline__ uint32_t forest_walk(const Dev& d, int tau, uint32_t i, uint32_t f, uint32_t pi) {
  uint32_t k = static_cast<uint32_t>(tau);
  for (int guard = 0; guard <= kMaxDepth; ++guard) {  // trees are at most kMaxDepth deep
    const uint32_t s = d.nd_split[k];
    if (s == kLeaf) break;
    const uint32_t g = s >> 8;
    const uint8_t x = d.Xrow[static_cast<int64_t>(g == f ? pi : i) * d.ldP + g];
    k = d.nd_child[k] + (x > (s & 255u) ? 1u : 0u);
  }
  return k;
}

__host__ __device__ __forceinline__ int forest_k(const Dev& d) { return d.kind != 0 ? 1 : d.C; }

// one thread per (tree, row): the row's leaf value into its exact base sum
__global__ void k_fperm_base(Dev d) {
  const int K = forest_k(d);
  const int64_t items = static_cast<int64_t>(d.M) * d.N;
  for (int64_t it = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; it < items;
       it += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int tau = static_cast<int>(it / d.N);
    const uint32_t i = static_cast<uint32_t>(it - static_cast<int64_t>(tau) * d.N);
    const uint32_t q = forest_walk(d, tau, i, 0xFFFFFFFFu, 0u);
    for (int k = 0; k < K; ++k)
      if (!csa_add(d.fbase + (static_cast<int64_t>(i) * K + k) * kCsaLimbs, leaf_value(d, q, k)))
        atomicOr(&d.status[0], kErrAcc);
  }
}

// the forest's own prediction per row (the exact sums rounded once, / M)
__global__ void k_fperm_base_mean(Dev d) {
  const int K = forest_k(d);
  const int64_t items = static_cast<int64_t>(d.N) * K;
  for (int64_t it = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; it < items;
       it += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    uint64_t a[kFixLimbs];
    csa_to_fix(d.fbase + it * kCsaLimbs, a);
    d.fbase_mean[it] = fix_to_double(a) / static_cast<double>(d.M);
  }
}

// One thread per (tree, row of the block): the row's path; for each distinct
// column f on it, the leaf reached with f read at flush_index (the walk
// leaves the path at the first node testing f that sends the swapped value
// the other way); a changed leaf adds (new - old) per class to (row, f).
__global__ void k_fperm_delta(Dev d, uint32_t r0, uint32_t rows) {
  const int K = forest_k(d);
  const int64_t items = static_cast<int64_t>(d.M) * rows;
  for (int64_t it = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; it < items;
       it += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int tau = static_cast<int>(it / rows);
    const uint32_t loc = static_cast<uint32_t>(it - static_cast<int64_t>(tau) * rows);
    const uint32_t i = r0 + loc;
    const uint32_t pi = d.piv[i];
    uint32_t pw[kMaxDepth];
    int depth = 0;
    uint32_t k = static_cast<uint32_t>(tau);
    for (uint32_t s = d.nd_split[k]; s != kLeaf && depth < kMaxDepth; s = d.nd_split[k]) {
      const uint8_t x = d.Xrow[static_cast<int64_t>(i) * d.ldP + (s >> 8)];
      pw[depth++] = s;
      k = d.nd_child[k] + (x > (s & 255u) ? 1u : 0u);
    }
    const uint32_t q = k;
    for (int a = 0; a < depth; ++a) {  // a column off the path leaves the leaf unchanged
      const uint32_t f = pw[a] >> 8;
      bool seen = false;
      for (int b = 0; b < a; ++b) seen |= (pw[b] >> 8) == f;
      if (seen) continue;
      const uint32_t q2 = forest_walk(d, tau, i, f, pi);
      if (q2 == q) continue;
      long long* acc = d.facc + ((static_cast<int64_t>(loc) * d.p_aug + f) * K) * kCsaLimbs;
      bool ok = true;
      for (int c = 0; c < K; ++c) {
        ok &= csa_add(acc + c * kCsaLimbs, leaf_value(d, q2, c));
        ok &= csa_add(acc + c * kCsaLimbs, -leaf_value(d, q, c));
      }
      if (!ok) atomicOr(&d.status[0], kErrAcc);
    }
  }
}

// One thread per (row of the block, column): the loss between the forest's
// prediction and its prediction with the column permuted, summed exactly
// per column; the thread clears the (row, column) accumulators it read.
__global__ void k_fperm_loss(Dev d, uint32_t r0, uint32_t rows) {
  const int K = forest_k(d);
  const int64_t items = static_cast<int64_t>(rows) * d.p_aug;
  for (int64_t it = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; it < items;
       it += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const uint32_t loc = static_cast<uint32_t>(it / d.p_aug);
    const uint32_t f = static_cast<uint32_t>(it - static_cast<int64_t>(loc) * d.p_aug);
    const uint32_t i = r0 + loc;
    long long* acc = d.facc + ((static_cast<int64_t>(loc) * d.p_aug + f) * K) * kCsaLimbs;
    double L = 0.0;
    const double eps = d.kl_eps, norm = 1.0 + static_cast<double>(d.C) * eps;
    for (int c = 0; c < K; ++c) {
      bool zero = true;
#pragma unroll
      for (int l = 0; l < kCsaLimbs; ++l) zero &= acc[c * kCsaLimbs + l] == 0;
      if (zero) continue;  // no tree's leaf changed for this class value
      uint64_t a[kFixLimbs], b[kFixLimbs];
      csa_to_fix(d.fbase + (static_cast<int64_t>(i) * K + c) * kCsaLimbs, a);
      csa_to_fix(acc + c * kCsaLimbs, b);
      fix_add(a, b);
      const double perm = fix_to_double(a) / static_cast<double>(d.M);
      const double base = d.fbase_mean[static_cast<int64_t>(i) * K + c];
#pragma unroll
      for (int l = 0; l < kCsaLimbs; ++l) acc[c * kCsaLimbs + l] = 0;
      if (d.kind != 0) {
        const double df = (base - perm) * 0x1p-20;
        L += df * df;
      } else {
        const double pa = (base + eps) / norm, pb = (perm + eps) / norm;
        L += pa * log(pa / pb);
      }
    }
    if (L != 0.0 && !csa_add(d.acc + static_cast<int64_t>(f) * kCsaLimbs, L)) atomicOr(&d.status[0], kErrAcc);
  }
}

// imp[f] = (exact sum over rows of the losses, rounded once) / N
__global__ void k_fperm_final(Dev d) {
  for (int f = blockIdx.x * blockDim.x + threadIdx.x; f < d.p_aug; f += gridDim.x * blockDim.x) {
    uint64_t a[kFixLimbs];
    csa_to_fix(d.acc + static_cast<int64_t>(f) * kCsaLimbs, a);
    d.imp[f] = fix_to_double(a) / static_cast<double>(d.N);
  }
}

int launch_forest_permut(const Dev& d, int grid, cudaStream_t st) {
  int n = 0;
  k_permut_pi<<<(d.N + 255) / 256 < 1024 ? (d.N + 255) / 256 : 1024, 256, 0, st>>>(d);
  cudaMemsetAsync(d.fbase, 0, static_cast<size_t>(d.N) * forest_k(d) * kCsaLimbs * sizeof(long long), st);
  k_fperm_base<<<grid, 256, 0, st>>>(d);
  k_fperm_base_mean<<<grid, 256, 0, st>>>(d);
  n += 3;
  for (uint32_t r0 = 0; r0 < static_cast<uint32_t>(d.N); r0 += d.frows) {
    const uint32_t rows = min(d.frows, static_cast<uint32_t>(d.N) - r0);
    k_fperm_delta<<<grid, 256, 0, st>>>(d, r0, rows);
    k_fperm_loss<<<grid, 256, 0, st>>>(d, r0, rows);
    n += 2;
  }
  k_fperm_final<<<(d.p_aug + 255) / 256, 256, 0, st>>>(d);
  return n + 1;
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

int launch_stats_decide(const Dev& d, cudaStream_t st) {
  k_stats<<<(d.p_aug + 127) / 128, 128, 0, st>>>(d);
  k_decide<<<1, 1024, 0, st>>>(d);
  return 2;
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
