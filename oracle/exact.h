/* Oracle-internal exact arithmetic.  TEST INFRASTRUCTURE ONLY (see oracle.h). */
#ifndef BORUTA_ORACLE_EXACT_H
#define BORUTA_ORACLE_EXACT_H
#include "oracle.h"

typedef struct {
  uint64_t w[4]; /* little-endian limbs */
} u256;

u256 u256_from_u64(uint64_t x);
u256 u256_from_u128(unsigned __int128 x);
u256 u256_add(u256 a, u256 b);
u256 u256_sub(u256 a, u256 b);
u256 u256_mul(u256 a, u256 b, int* overflow);
int u256_cmp(u256 a, u256 b);
double u256_to_double(u256 a);
double u128_to_double(unsigned __int128 v);
/* exact sum of x[0], x[stride], ..., x[(n-1)*stride], rounded once */
double exact_sum(const double* x, int64_t n, int64_t stride);
void binom_tails(int t, int h, unsigned __int128* upper, unsigned __int128* lower);

#endif
