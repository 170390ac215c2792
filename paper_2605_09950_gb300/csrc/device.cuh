// Device primitives for the GPU Boruta kernels (sm_103a).
//
//  - Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) and a keyed, cycle-walked
//    8-round Feistel permutation (Black & Rogaway, CT-RSA 2002) with the
//    MurmurHash3 finaliser as round function: the random streams behind the
//    Alg. 1 shuffle, the Alg. 3 flush_index, the bootstrap and the per-node
//    feature sample.
//  - exact unsigned arithmetic up to 256 bits for split-score comparisons;
//  - correctly rounded (ties-to-even) conversion of such integers to double
//    and float;
//  - an exact fixed-point accumulator (384-bit two's complement, LSB 2^-192)
//    so every floating-point sum of the method is formed exactly and rounded
//    once, independent of the order in which threads add their terms.
#pragma once
#include <cstdint>

#include <cuda_runtime.h>

namespace bgb {

// ---------------------------------------------------------------- limits, flags
constexpr int kMaxClasses = 8;
constexpr int kMaxDepth = 30;
constexpr uint32_t kLeaf = 0xFFFFFFFFu;  // split word of a leaf

enum : uint32_t {
  kErrPool = 1u,      // node pool capacity exceeded
  kErrWeight = 2u,    // a bootstrap count exceeded 255
  kErrAcc = 4u,       // an accumulator term outside the fixed-point window
  kErrInput = 16u,    // a bin >= n_bins or a label >= n_classes
};

enum : uint32_t { kPurposeShadow = 1u, kPurposeBoot = 2u, kPurposeMtry = 3u, kPurposePermut = 4u };

// ---------------------------------------------------------------- Philox4x32-10
__device__ __forceinline__ uint4 philox10(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k.x += 0x9E3779B9u;
      k.y += 0xBB67AE85u;
    }
    const uint32_t a = 0xD2511F53u * c.x, ah = __umulhi(0xD2511F53u, c.x);
    const uint32_t b = 0xCD9E8D57u * c.z, bh = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(bh ^ c.y ^ k.x, b, ah ^ c.w ^ k.y, a);
  }
  return c;
}

__device__ __forceinline__ uint2 seed_key(uint64_t seed) {
  return make_uint2(static_cast<uint32_t>(seed), static_cast<uint32_t>(seed >> 32));
}

// 64-bit draw: words 0 and 1 of one Philox block
__device__ __forceinline__ uint64_t draw64(uint64_t seed, uint32_t w0, uint32_t w1, uint32_t w2,
                                           uint32_t w3) {
  const uint4 o = philox10(make_uint4(w0, w1, w2, w3), seed_key(seed));
  return static_cast<uint64_t>(o.x) | (static_cast<uint64_t>(o.y) << 32);
}

__device__ __forceinline__ uint32_t unit_word(int t, uint32_t unit) {
  return (static_cast<uint32_t>(t) << 24) | (unit & 0xFFFFFFu);
}
__device__ __forceinline__ uint32_t purpose_word(uint32_t purpose, uint32_t job) {
  return (purpose << 24) | (job & 0xFFFFFFu);
}

// ---------------------------------------------------------------- Feistel permutation
__device__ __forceinline__ uint32_t murmur_fmix(uint32_t h) {
  h = (h ^ (h >> 16)) * 0x85EBCA6Bu;
  h = (h ^ (h >> 13)) * 0xC2B2AE35u;
  return h ^ (h >> 16);
}

struct Perm {
  uint32_t key[8];
  uint32_t n;     // domain [0, n)
  uint32_t half;  // bits per half
  uint32_t mask;
};

__device__ __forceinline__ void perm_init(Perm& P, uint32_t n, uint64_t seed, uint32_t w1,
                                          uint32_t w2, uint32_t w3) {
  uint32_t half = 1;
  while ((1ull << (2 * half)) < n) ++half;
  P.n = n;
  P.half = half;
  P.mask = (1u << half) - 1u;
  const uint2 k = seed_key(seed);
  const uint4 a = philox10(make_uint4(0u, w1, w2, w3), k);
  const uint4 b = philox10(make_uint4(1u, w1, w2, w3), k);
  P.key[0] = a.x; P.key[1] = a.y; P.key[2] = a.z; P.key[3] = a.w;
  P.key[4] = b.x; P.key[5] = b.y; P.key[6] = b.z; P.key[7] = b.w;
}

__device__ __forceinline__ uint32_t feistel8(const Perm& P, uint32_t x) {
  uint32_t left = x >> P.half, right = x & P.mask;
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    const uint32_t next = left ^ (murmur_fmix(right ^ P.key[r]) & P.mask);
    left = right;
    right = next;
  }
  return (left << P.half) | right;
}

// sigma(i): encrypt, then walk the cycle until the value falls inside [0, n)
__device__ __forceinline__ uint32_t perm_apply(const Perm& P, uint32_t i) {
  if (P.n <= 1u) return i;
  uint32_t x = feistel8(P, i);
  while (x >= P.n) x = feistel8(P, x);
  return x;
}

// ---------------------------------------------------------------- exact integers
typedef unsigned __int128 u128;

struct U192 {  // little-endian limbs
  uint64_t w[3];
};

__device__ __forceinline__ U192 u192_from(u128 v) {
  U192 r;
  r.w[0] = static_cast<uint64_t>(v);
  r.w[1] = static_cast<uint64_t>(v >> 64);
  r.w[2] = 0;
  return r;
}

// a * b as four limbs
__device__ __forceinline__ void mul192x64(const U192& a, uint64_t b, uint64_t out[4]) {
  u128 p = static_cast<u128>(a.w[0]) * b;
  out[0] = static_cast<uint64_t>(p);
  p = static_cast<u128>(a.w[1]) * b + (p >> 64);
  out[1] = static_cast<uint64_t>(p);
  p = static_cast<u128>(a.w[2]) * b + (p >> 64);
  out[2] = static_cast<uint64_t>(p);
  out[3] = static_cast<uint64_t>(p >> 64);
}

__device__ __forceinline__ int cmp_limbs4(const uint64_t a[4], const uint64_t b[4]) {
#pragma unroll
  for (int i = 3; i >= 0; --i) {
    if (a[i] != b[i]) return a[i] > b[i] ? 1 : -1;
  }
  return 0;
}

// sign of num_a/den_a - num_b/den_b (denominators > 0)
__device__ __forceinline__ int frac_cmp(const U192& num_a, uint64_t den_a, const U192& num_b,
                                        uint64_t den_b) {
  uint64_t x[4], y[4];
  mul192x64(num_a, den_b, x);
  mul192x64(num_b, den_a, y);
  return cmp_limbs4(x, y);
}

// value of limbs[0..n) * 2^scale, correctly rounded to double (normal range)
__device__ inline double limbs_to_double(const uint64_t* w, int n, int scale) {
  int top = n - 1;
  while (top >= 0 && w[top] == 0) --top;
  if (top < 0) return 0.0;
  const int msb = top * 64 + 63 - __clzll(static_cast<long long>(w[top]));
  if (msb < 53) return scalbn(static_cast<double>(w[0]), scale);
  const int lo = msb - 63;  // lowest bit of a 64-bit window whose top bit is the msb
  uint64_t win;
  bool sticky = false;
  if (lo >= 0) {
    const int li = lo >> 6, off = lo & 63;
    win = w[li] >> off;
    if (off) {
      if (li + 1 < n) win |= w[li + 1] << (64 - off);
      sticky = (w[li] & ((1ull << off) - 1ull)) != 0;
    }
    for (int i = 0; i < li && !sticky; ++i) sticky = w[i] != 0;
  } else {
    win = w[0] << (-lo);
  }
  uint64_t m = win >> 11;
  const uint64_t rest = win & 0x7FFull;
  sticky = sticky || (rest & 0x3FFull);
  if ((rest & 0x400ull) && (sticky || (m & 1ull))) m += 1;
  return scalbn(static_cast<double>(m), scale + msb - 52);
}

__device__ inline float limbs_to_float(const uint64_t* w, int n, int scale) {
  int top = n - 1;
  while (top >= 0 && w[top] == 0) --top;
  if (top < 0) return 0.0f;
  const int msb = top * 64 + 63 - __clzll(static_cast<long long>(w[top]));
  if (msb < 24) return scalbnf(static_cast<float>(w[0]), scale);
  const int lo = msb - 63;
  uint64_t win;
  bool sticky = false;
  if (lo >= 0) {
    const int li = lo >> 6, off = lo & 63;
    win = w[li] >> off;
    if (off) {
      if (li + 1 < n) win |= w[li + 1] << (64 - off);
      sticky = (w[li] & ((1ull << off) - 1ull)) != 0;
    }
    for (int i = 0; i < li && !sticky; ++i) sticky = w[i] != 0;
  } else {
    win = w[0] << (-lo);
  }
  uint32_t m = static_cast<uint32_t>(win >> 40);
  const uint64_t rest = win & ((1ull << 40) - 1ull);
  sticky = sticky || (rest & ((1ull << 39) - 1ull));
  if ((rest >> 39) && (sticky || (m & 1u))) m += 1;
  return scalbnf(static_cast<float>(m), scale + msb - 23);
}

// ---------------------------------------------------------------- exact accumulation
// Value = (two's complement integer in 6 limbs) * 2^-192.
constexpr int kFixLimbs = 6;
constexpr int kFixShift = 192;

// x as a fixed-point addend.  Bits below 2^-192 are dropped (toward zero);
// returns false (and leaves v zero) for values of magnitude >= 2^190 or non-finite.
__device__ inline bool fix_from_double(double x, uint64_t v[kFixLimbs]) {
#pragma unroll
  for (int i = 0; i < kFixLimbs; ++i) v[i] = 0;
  if (x == 0.0) return true;
  const uint64_t bits = static_cast<uint64_t>(__double_as_longlong(x));
  const bool neg = bits >> 63;
  const int eraw = static_cast<int>((bits >> 52) & 0x7FF);
  if (eraw == 0x7FF) return false;
  uint64_t m = bits & ((1ull << 52) - 1ull);
  int e;
  if (eraw) {
    m |= 1ull << 52;
    e = eraw - 1075;
  } else {
    e = -1074;
  }
  int pos = e + kFixShift;
  if (pos < 0) {
    m = (-pos >= 64) ? 0ull : (m >> (-pos));
    pos = 0;
  }
  if (m == 0) return true;
  if (pos + 53 > 64 * kFixLimbs - 2) return false;
  const int li = pos >> 6, off = pos & 63;
  v[li] = m << off;
  if (off && li + 1 < kFixLimbs) v[li + 1] = m >> (64 - off);
  if (neg) {
    uint64_t carry = 1;
#pragma unroll
    for (int i = 0; i < kFixLimbs; ++i) {
      const uint64_t s = ~v[i] + carry;
      carry = (carry && s == 0) ? 1ull : 0ull;
      v[i] = s;
    }
  }
  return true;
}

__device__ __forceinline__ void fix_add(uint64_t acc[kFixLimbs], const uint64_t v[kFixLimbs]) {
  uint64_t carry = 0;
#pragma unroll
  for (int i = 0; i < kFixLimbs; ++i) {
    const uint64_t s = acc[i] + v[i];
    const uint64_t c1 = s < acc[i];
    const uint64_t s2 = s + carry;
    const uint64_t c2 = s2 < s;
    acc[i] = s2;
    carry = c1 | c2;
  }
}

// round the exact value once
__device__ inline double fix_to_double(const uint64_t acc[kFixLimbs]) {
  uint64_t mag[kFixLimbs];
  const bool neg = acc[kFixLimbs - 1] >> 63;
  uint64_t carry = 1;
#pragma unroll
  for (int i = 0; i < kFixLimbs; ++i) {
    if (neg) {
      const uint64_t s = ~acc[i] + carry;
      carry = (carry && s == 0) ? 1ull : 0ull;
      mag[i] = s;
    } else {
      mag[i] = acc[i];
    }
  }
  const double r = limbs_to_double(mag, kFixLimbs, -kFixShift);
  return neg ? -r : r;
}

__device__ inline float fix_to_float(const uint64_t acc[kFixLimbs]) {
  uint64_t mag[kFixLimbs];
  const bool neg = acc[kFixLimbs - 1] >> 63;
  uint64_t carry = 1;
#pragma unroll
  for (int i = 0; i < kFixLimbs; ++i) {
    if (neg) {
      const uint64_t s = ~acc[i] + carry;
      carry = (carry && s == 0) ? 1ull : 0ull;
      mag[i] = s;
    } else {
      mag[i] = acc[i];
    }
  }
  const float r = limbs_to_float(mag, kFixLimbs, -kFixShift);
  return neg ? -r : r;
}

// ---------------------------------------------------------------- carry-save accumulation
// The same exact value in a form that concurrent adders update without
// reading back: 12 signed 64-bit limbs, limb i weighing 2^(32 i - 192); a
// term adds (or subtracts) its 32-bit chunks to at most three limbs, so no
// carry moves between limbs while terms arrive (a limb absorbs 2^31 terms
// without overflow).  Carries are propagated once, when the sum is read.
constexpr int kCsaLimbs = 12;

// false (nothing added) for magnitudes >= 2^190 or non-finite terms
__device__ inline bool csa_add(long long* acc, double x) {
  if (x == 0.0) return true;
  const uint64_t bits = static_cast<uint64_t>(__double_as_longlong(x));
  const bool neg = bits >> 63;
  const int eraw = static_cast<int>((bits >> 52) & 0x7FF);
  if (eraw == 0x7FF) return false;
  uint64_t m = bits & ((1ull << 52) - 1ull);
  int e;
  if (eraw) {
    m |= 1ull << 52;
    e = eraw - 1075;
  } else {
    e = -1074;
  }
  int pos = e + kFixShift;
  if (pos < 0) {
    m = (-pos >= 64) ? 0ull : (m >> (-pos));
    pos = 0;
  }
  if (m == 0) return true;
  if (pos + 53 > 32 * kCsaLimbs - 2) return false;
  const int li = pos >> 5, off = pos & 31;
  const u128 v = static_cast<u128>(m) << off;
  const uint32_t c[3] = {static_cast<uint32_t>(v), static_cast<uint32_t>(v >> 32),
                         static_cast<uint32_t>(v >> 64)};
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    if (c[q]) {
      const long long s = neg ? -static_cast<long long>(c[q]) : static_cast<long long>(c[q]);
      atomicAdd(reinterpret_cast<unsigned long long*>(acc + li + q), static_cast<unsigned long long>(s));
    }
  }
  return true;
}

// carry-save limbs -> 384-bit two's complement (kFixLimbs u64 limbs)
__device__ inline void csa_to_fix(const long long* acc, uint64_t out[kFixLimbs]) {
  __int128 carry = 0;
  uint32_t w[kCsaLimbs];
#pragma unroll
  for (int i = 0; i < kCsaLimbs; ++i) {
    const __int128 s = carry + static_cast<__int128>(acc[i]);
    w[i] = static_cast<uint32_t>(static_cast<unsigned __int128>(s) & 0xFFFFFFFFu);
    carry = s >> 32;  // arithmetic: keeps the sign
  }
#pragma unroll
  for (int i = 0; i < kFixLimbs; ++i)
    out[i] = static_cast<uint64_t>(w[2 * i]) | (static_cast<uint64_t>(w[2 * i + 1]) << 32);
}

// ---------------------------------------------------------------- warp helpers
__device__ __forceinline__ uint32_t warp_excl_scan_u32(uint32_t v, int lane) {
  uint32_t x = v;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, d);
    if (lane >= d) x += y;
  }
  return x - v;
}

__device__ __forceinline__ long long warp_excl_scan_i64(long long v, int lane) {
  long long x = v;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const long long y = __shfl_up_sync(0xFFFFFFFFu, x, d);
    if (lane >= d) x += y;
  }
  return x - v;
}

__device__ __forceinline__ float warp_max_f(float v) {
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) v = fmaxf(v, __shfl_xor_sync(0xFFFFFFFFu, v, d));
  return v;
}

}  // namespace bgb
