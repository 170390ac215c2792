// Binomial tails of the Boruta test with no device allocation.
//
// boruta_binom_tails builds its table of binomial coefficients in memory it
// allocates on every call.  Some callers cannot allocate device memory at
// all: a host application whose own caching allocator has reserved the
// GPU's memory, or a latency-critical path where cudaMalloc / cudaFree
// (which may synchronise the device) are not allowed.  For them this file
// keeps the table in a fixed file-scope device array instead.
#include <cstdint>
#include <mutex>

#include "boruta.h"
#include "engine.cuh"

namespace {

using bgb::u128;

constexpr int kMaxRows = 127;  // C(t, k) for 0 <= k <= t <= 126 (max_iter <= 126)

// The whole scratch: 127 x 127 coefficients (258,064 bytes) and one error
// word, 258,080 bytes with the 16-byte alignment of the coefficients.  With
// CUDA's default lazy module loading the array is allocated on a device when
// this file's module is first used there (the first call on that device);
// from then on the device holds it until the process exits.
struct NoAllocScratch {
  u128 tri[kMaxRows * kMaxRows];
  unsigned int bad;  // set when a query asks for t outside [0, 126]
};

static __device__ __align__(256) NoAllocScratch g_noalloc_scratch;
static_assert(sizeof(NoAllocScratch) == 258080, "size stated in boruta.h");

// Device address of the array per device, looked up once per device with
// that device current (in host code the symbol itself is only a stand-in).
constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
NoAllocScratch* g_scratch_ptr[kMaxDevices] = {};

// Pascal's rule, one row per step; thread k owns column k.
__global__ void k_noalloc_pascal(NoAllocScratch* s) {
  const int k = threadIdx.x;
  for (int r = 0; r < kMaxRows; ++r) {
    if (k < kMaxRows) {
      u128 v = 0;
      if (k == 0)
        v = 1;
      else if (k <= r)
        v = s->tri[(r - 1) * kMaxRows + k - 1] + s->tri[(r - 1) * kMaxRows + k];
      s->tri[r * kMaxRows + k] = v;
    }
    __syncthreads();
  }
}

__global__ void k_noalloc_tails(NoAllocScratch* s, const int32_t* t, const int32_t* h, double* pa,
                                double* pr, int64_t n) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int tt = t[i], hh = h[i];
    if (tt < 0 || tt >= kMaxRows) {
      atomicOr(&s->bad, 1u);
      pa[i] = pr[i] = __longlong_as_double(0x7FF8000000000000ll);  // NaN
      continue;
    }
    const u128* row = s->tri + static_cast<int64_t>(tt) * kMaxRows;
    u128 up = 0, lo = 0;
    for (int k = 0; k <= tt; ++k) {
      if (k >= hh) up += row[k];
      if (k <= hh) lo += row[k];
    }
    const uint64_t wu[2] = {static_cast<uint64_t>(up), static_cast<uint64_t>(up >> 64)};
    const uint64_t wl[2] = {static_cast<uint64_t>(lo), static_cast<uint64_t>(lo >> 64)};
    pa[i] = bgb::limbs_to_double(wu, 2, -tt);
    pr[i] = bgb::limbs_to_double(wl, 2, -tt);
  }
}

// Looks up the array's device address and fills the table, once per device.
int setup(cudaStream_t st, NoAllocScratch** out, const char** err) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    *err = "no usable current CUDA device";
    return BORUTA_ECUDA;
  }
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
      *err = "cudaGetSymbolAddress of the no-allocation scratch failed";
      return BORUTA_ECUDA;
    }
    NoAllocScratch* s = static_cast<NoAllocScratch*>(p);
    k_noalloc_pascal<<<1, 128, 0, st>>>(s);
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess) {
      *err = "building the binomial table failed";
      return BORUTA_ECUDA;
    }
    g_scratch_ptr[dev] = s;
  }
  *out = g_scratch_ptr[dev];
  return 0;
}

}  // namespace

int boruta_noalloc_fail(int code, const char* msg);  // api.cu: records the message

extern "C" int boruta_binom_tails_noalloc(const int32_t* t, const int32_t* h, double* p_acc,
                                          double* p_rej, int64_t n, void* stream) {
  if (n < 0) return boruta_noalloc_fail(BORUTA_EINVAL, "n must not be negative");
  if (n > 0 && (!t || !h || !p_acc || !p_rej)) return boruta_noalloc_fail(BORUTA_EINVAL, "NULL pointer");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  NoAllocScratch* s = nullptr;
  const char* err = nullptr;
  int rc = setup(st, &s, &err);
  if (rc) return boruta_noalloc_fail(rc, err);
  if (n == 0) return 0;
  if (cudaMemsetAsync(&s->bad, 0, sizeof(unsigned int), st) != cudaSuccess)
    return boruta_noalloc_fail(BORUTA_ECUDA, "clearing the error word failed");
  int64_t g = (n + 255) / 256;
  if (g > 4096) g = 4096;
  k_noalloc_tails<<<static_cast<int>(g), 256, 0, st>>>(s, t, h, p_acc, p_rej, n);
  unsigned int bad = 0;
  if (cudaGetLastError() != cudaSuccess ||
      cudaMemcpyAsync(&bad, &s->bad, sizeof bad, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return boruta_noalloc_fail(BORUTA_ECUDA, "binomial tails kernel failed");
  if (bad)
    return boruta_noalloc_fail(BORUTA_EINVAL,
                               "t outside [0, 126]: the fixed table holds C(t, k) for t <= 126 only");
  return 0;
}
