// boruta_quantise: float features -> uint8 quantile bins, on the GPU.
//
// The method consumes binned features (the histogram forest of the fit), and
// the paper does not say how they are binned; the library's reading is
//   bin(x) = min(B - 1, floor(B * rank(x) / N)),  rank(x) = #{values < x},
// so equal values share a bin.  With r_k = ceil(k N / B) (k = 1..B-1) and T_k
// the r_k-th smallest value of the column, floor(B rank / N) >= k exactly
// when rank >= r_k, i.e. when T_k < x; hence bin(x) = #{k : T_k < x}.
//
// One block per column finds all B-1 order statistics at once by bisection
// on the 32-bit order-preserving key of the float: every target keeps an
// interval [lo_k, hi_k] of keys; the intervals stay ordered in k (the targets
// are), so the midpoints are sorted and one sweep over the column counts,
// for every midpoint, the values at or below it (a binary search per value
// into the midpoints plus a prefix sum).  32 sweeps fix every key; a last
// sweep writes the bins.
#include <cstdint>

#include <cuda_runtime.h>

#include "boruta.h"

namespace {

constexpr int kQThreads = 1024;
constexpr int kQTargets = 255;  // B - 1 at most

int qfail(int code, const char* msg);  // below

// order-preserving key of a float (-0 taken as +0); NaN reported by the caller
__device__ __forceinline__ uint32_t fkey(float x) {
  if (x == 0.0f) x = 0.0f;
  const uint32_t u = __float_as_uint(x);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

// number of sorted keys m[0..n) that are < v
__device__ __forceinline__ int count_below(const uint32_t* m, int n, uint32_t v) {
  int lo = 0, hi = n;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (m[mid] < v)
      lo = mid + 1;
    else
      hi = mid;
  }
  return lo;
}

__global__ void __launch_bounds__(kQThreads) k_quantise(const float* X, int64_t ldx, uint32_t N, int64_t p, int B,
                                                        uint8_t* Xb, int64_t ldb, uint32_t* bad) {
  __shared__ uint32_t lo[kQTargets], hi[kQTargets], mid[kQTargets];
  __shared__ uint32_t cnt[kQTargets + 1];
  __shared__ uint32_t rk[kQTargets];
  const int nt = B - 1;
  for (int64_t j = blockIdx.x; j < p; j += gridDim.x) {
    const float* col = X + j * ldx;
    for (int k = threadIdx.x; k < nt; k += blockDim.x) {
      lo[k] = 0u;
      hi[k] = 0xFFFFFFFFu;
      // r_k = ceil(k N / B)
      rk[k] = static_cast<uint32_t>((static_cast<uint64_t>(k + 1) * N + static_cast<uint64_t>(B) - 1) /
                                    static_cast<uint64_t>(B));
    }
    __syncthreads();
    for (int pass = 0; pass < 33; ++pass) {
      for (int k = threadIdx.x; k < nt; k += blockDim.x)
        mid[k] = static_cast<uint32_t>((static_cast<uint64_t>(lo[k]) + hi[k]) >> 1);
      for (int k = threadIdx.x; k <= nt; k += blockDim.x) cnt[k] = 0u;
      __syncthreads();
      // cnt[c] = values whose key lies above exactly c midpoints
      for (uint32_t i = threadIdx.x; i < N; i += blockDim.x) {
        const float x = col[i];
        if (x != x) {
          atomicOr(bad, 1u);
          continue;
        }
        atomicAdd(&cnt[count_below(mid, nt, fkey(x))], 1u);
      }
      __syncthreads();
      if (threadIdx.x == 0) {
        // values <= mid_k = those above fewer than k + 1 midpoints (mid is sorted)
        uint32_t run = 0;
        for (int k = 0; k < nt; ++k) {
          run += cnt[k];
          if (lo[k] < hi[k]) {
            if (run >= rk[k])
              hi[k] = mid[k];
            else
              lo[k] = mid[k] + 1u;
          }
        }
        // keep the intervals ordered in k (T_k <= T_k+1)
        for (int k = 1; k < nt; ++k)
          if (lo[k] < lo[k - 1]) lo[k] = lo[k - 1];
        for (int k = nt - 2; k >= 0; --k)
          if (hi[k] > hi[k + 1]) hi[k] = hi[k + 1];
      }
      __syncthreads();
    }
    // lo[k] = T_k; bin = number of T_k below the value
    uint8_t* out = Xb + j * ldb;
    for (uint32_t i = threadIdx.x; i < N; i += blockDim.x) {
      const float x = col[i];
      out[i] = (x != x) ? 0u : static_cast<uint8_t>(count_below(lo, nt, fkey(x)));
    }
    __syncthreads();
  }
}

}  // namespace

int boruta_noalloc_fail(int code, const char* msg);  // api.cu: records the message

namespace {
int qfail(int code, const char* msg) { return boruta_noalloc_fail(code, msg); }
}  // namespace

extern "C" int boruta_quantise(const float* X, int64_t ldx, int64_t N, int64_t p, int n_bins, uint8_t* Xb,
                               int64_t ldb, void* stream) {
  if (N < 1 || N >= (1ll << 24) || p < 1 || ldx < N || ldb < N || !X || !Xb)
    return qfail(BORUTA_EINVAL, "boruta_quantise: bad sizes or pointers");
  if (n_bins < 2 || n_bins > 256) return qfail(BORUTA_EINVAL, "boruta_quantise: n_bins outside [2, 256]");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  uint32_t* bad = nullptr;
  if (cudaMallocAsync(reinterpret_cast<void**>(&bad), sizeof(uint32_t), st) != cudaSuccess) {
    cudaGetLastError();
    return qfail(BORUTA_ENOMEM, "boruta_quantise: scratch allocation failed");
  }
  uint32_t bad_h = 0;
  cudaMemsetAsync(bad, 0, sizeof(uint32_t), st);
  const int grid = static_cast<int>(p < 4096 ? p : 4096);
  k_quantise<<<grid, kQThreads, 0, st>>>(X, ldx, static_cast<uint32_t>(N), p, n_bins, Xb, ldb, bad);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(&bad_h, bad, sizeof(uint32_t), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFreeAsync(bad, st);
  if (e != cudaSuccess) return qfail(BORUTA_ECUDA, cudaGetErrorString(e));
  if (bad_h) return qfail(BORUTA_EINVAL, "boruta_quantise: NaN in the input");
  return 0;
}
