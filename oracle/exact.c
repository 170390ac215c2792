/*
 * Oracle exact arithmetic.  TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 *  - 256-bit unsigned integers (four little-endian 64-bit limbs) for the
 *    exact comparison of split scores, which are ratios of integer
 *    polynomials in the bootstrap-weighted counts;
 *  - correctly rounded (round-half-even) conversion of such integers to
 *    double;
 *  - the exact sum of a list of doubles, rounded once (a wide two's
 *    complement fixed-point accumulator covering the whole double range);
 *  - the binomial tail sums of the Boruta test, exact in 128-bit integers.
 */
#include <math.h>
#include <string.h>

#include "exact.h"

u256 u256_from_u64(uint64_t x) {
  u256 r = {{x, 0, 0, 0}};
  return r;
}

u256 u256_from_u128(unsigned __int128 x) {
  u256 r = {{(uint64_t)x, (uint64_t)(x >> 64), 0, 0}};
  return r;
}

u256 u256_add(u256 a, u256 b) {
  u256 r;
  unsigned __int128 carry = 0;
  for (int i = 0; i < 4; i++) {
    unsigned __int128 s = (unsigned __int128)a.w[i] + b.w[i] + carry;
    r.w[i] = (uint64_t)s;
    carry = s >> 64;
  }
  return r;
}

/* a - b, requires a >= b */
u256 u256_sub(u256 a, u256 b) {
  u256 r;
  uint64_t borrow = 0;
  for (int i = 0; i < 4; i++) {
    uint64_t d = a.w[i] - b.w[i];
    uint64_t b1 = a.w[i] < b.w[i];
    uint64_t d2 = d - borrow;
    uint64_t b2 = d < borrow;
    r.w[i] = d2;
    borrow = b1 | b2;
  }
  return r;
}

/* full product, *overflow set if it does not fit in 256 bits */
u256 u256_mul(u256 a, u256 b, int* overflow) {
  uint64_t full[8] = {0};
  for (int i = 0; i < 4; i++) {
    unsigned __int128 carry = 0;
    for (int j = 0; j < 4; j++) {
      unsigned __int128 cur = (unsigned __int128)a.w[i] * b.w[j] + full[i + j] + carry;
      full[i + j] = (uint64_t)cur;
      carry = cur >> 64;
    }
    full[i + 4] = (uint64_t)carry;
  }
  if (full[4] | full[5] | full[6] | full[7]) *overflow = 1;
  u256 r = {{full[0], full[1], full[2], full[3]}};
  return r;
}

int u256_cmp(u256 a, u256 b) {
  for (int i = 3; i >= 0; i--) {
    if (a.w[i] != b.w[i]) return a.w[i] > b.w[i] ? 1 : -1;
  }
  return 0;
}

/* Correctly rounded value of (limbs as an unsigned integer) * 2^lsb_exp.
 * Round to nearest, ties to even.  Results in the subnormal range are not
 * needed by this program and are not handled specially. */
static double limbs_to_double(const uint64_t* limbs, int nlimbs, int lsb_exp) {
  int top = -1; /* index of the highest set bit */
  for (int i = nlimbs - 1; i >= 0 && top < 0; i--) {
    if (limbs[i]) top = i * 64 + 63 - __builtin_clzll(limbs[i]);
  }
  if (top < 0) return 0.0;
#define BIT(k) ((limbs[(k) >> 6] >> ((k) & 63)) & 1u)
  if (top < 53) { /* fits a double exactly */
    uint64_t m = 0;
    for (int k = top; k >= 0; k--) m = (m << 1) | BIT(k);
    return ldexp((double)m, lsb_exp);
  }
  uint64_t m = 0; /* the 53 leading bits */
  for (int k = top; k > top - 53; k--) m = (m << 1) | BIT(k);
  int cut = top - 53; /* highest discarded bit */
  int round_bit = (int)BIT(cut);
  int sticky = 0;
  for (int k = cut - 1; k >= 0 && !sticky; k--) sticky = (int)BIT(k);
#undef BIT
  if (round_bit && (sticky || (m & 1u))) m += 1;
  /* m may have become 2^53: still exact as a double */
  return ldexp((double)m, lsb_exp + cut + 1);
}

double u256_to_double(u256 a) { return limbs_to_double(a.w, 4, 0); }

int orc_cmp_products(const uint64_t a1[4], const uint64_t b1[4], const uint64_t a2[4],
                     const uint64_t b2[4]) {
  u256 A1, B1, A2, B2;
  memcpy(A1.w, a1, 32);
  memcpy(B1.w, b1, 32);
  memcpy(A2.w, a2, 32);
  memcpy(B2.w, b2, 32);
  int of = 0;
  u256 x = u256_mul(A1, B1, &of);
  u256 y = u256_mul(A2, B2, &of);
  if (of) return 2;
  return u256_cmp(x, y);
}

double orc_u256_to_double(const uint64_t a[4]) { return limbs_to_double(a, 4, 0); }

/* ---- exact summation ----
 * Each double is m * 2^e with |m| < 2^53 and e >= -1074; the accumulator
 * holds sum * 2^ACC_SHIFT as a two's complement integer of ACC_LIMBS limbs,
 * wide enough for any sum of fewer than 2^60 doubles. */
#define ACC_SHIFT 1074
#define ACC_LIMBS 36 /* 2304 bits: 1074 fraction bits + 1024 + 60 headroom + sign */

typedef struct {
  uint64_t w[ACC_LIMBS];
} superacc;

static void acc_add_shifted(superacc* A, uint64_t mag, int shift, int negative) {
  /* add (or subtract) mag * 2^shift, shift >= 0 */
  uint64_t v[ACC_LIMBS];
  memset(v, 0, sizeof v);
  int limb = shift >> 6, off = shift & 63;
  v[limb] = mag << off;
  if (off && limb + 1 < ACC_LIMBS) v[limb + 1] = mag >> (64 - off);
  if (negative) { /* two's complement negation of v */
    unsigned __int128 carry = 1;
    for (int i = 0; i < ACC_LIMBS; i++) {
      unsigned __int128 s = (unsigned __int128)(~v[i]) + carry;
      v[i] = (uint64_t)s;
      carry = s >> 64;
    }
  }
  unsigned __int128 carry = 0;
  for (int i = 0; i < ACC_LIMBS; i++) {
    unsigned __int128 s = (unsigned __int128)A->w[i] + v[i] + carry;
    A->w[i] = (uint64_t)s;
    carry = s >> 64;
  }
}

static void acc_add(superacc* A, double x) {
  if (x == 0.0) return;
  int e;
  double f = frexp(fabs(x), &e); /* |x| = f * 2^e, 0.5 <= f < 1 */
  /* |x| = mant * 2^(e - 53) with mant an integer < 2^53 */
  uint64_t mant = (uint64_t)ldexp(f, 53);
  int exp2 = e - 53;
  int shift = exp2 + ACC_SHIFT;
  if (shift < 0) { /* subnormal inputs: mant carries trailing zeros */
    mant >>= -shift;
    shift = 0;
  }
  acc_add_shifted(A, mant, shift, x < 0);
}

static double acc_round(const superacc* A) {
  int negative = (A->w[ACC_LIMBS - 1] >> 63) & 1u;
  uint64_t mag[ACC_LIMBS];
  memcpy(mag, A->w, sizeof mag);
  if (negative) {
    unsigned __int128 carry = 1;
    for (int i = 0; i < ACC_LIMBS; i++) {
      unsigned __int128 s = (unsigned __int128)(~mag[i]) + carry;
      mag[i] = (uint64_t)s;
      carry = s >> 64;
    }
  }
  double r = limbs_to_double(mag, ACC_LIMBS, -ACC_SHIFT);
  return negative ? -r : r;
}

double exact_sum(const double* x, int64_t n, int64_t stride) {
  superacc A;
  memset(&A, 0, sizeof A);
  for (int64_t i = 0; i < n; i++) acc_add(&A, x[i * stride]);
  return acc_round(&A);
}

double orc_exact_sum(const double* x, int64_t n) { return exact_sum(x, n, 1); }

/* ---- Boruta test (Alg. 1 `test`, read as Kursa's two one-sided binomial
 * tests at 1/2) ----
 * upper = sum_{k=h}^{t} C(t,k), lower = sum_{k=0}^{h} C(t,k), both exact;
 * p_acc = upper / 2^t, p_rej = lower / 2^t (one rounding each). */
void binom_tails(int t, int h, unsigned __int128* upper, unsigned __int128* lower) {
  unsigned __int128 row[128];
  memset(row, 0, sizeof row);
  row[0] = 1;
  for (int r = 1; r <= t; r++) { /* Pascal's rule, row r from row r-1 */
    for (int k = r; k >= 1; k--) row[k] = row[k] + row[k - 1];
  }
  unsigned __int128 up = 0, lo = 0;
  for (int k = 0; k <= t; k++) {
    if (k >= h) up += row[k];
    if (k <= h) lo += row[k];
  }
  *upper = up;
  *lower = lo;
}

double u128_to_double(unsigned __int128 v) {
  uint64_t limbs[2] = {(uint64_t)v, (uint64_t)(v >> 64)};
  return limbs_to_double(limbs, 2, 0);
}

void orc_binom_tails(int t, int h, double* p_acc, double* p_rej, uint64_t upper[2],
                     uint64_t lower[2]) {
  unsigned __int128 up, lo;
  binom_tails(t, h, &up, &lo);
  *p_acc = ldexp(u128_to_double(up), -t);
  *p_rej = ldexp(u128_to_double(lo), -t);
  upper[0] = (uint64_t)up;
  upper[1] = (uint64_t)(up >> 64);
  lower[0] = (uint64_t)lo;
  lower[1] = (uint64_t)(lo >> 64);
}
