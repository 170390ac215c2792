/*
 * Oracle random streams.  TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * The paper draws its randomness from NumPy/CuPy (Alg. 1 shuffle, Alg. 3
 * random.permutation) and from cuML's forest (bootstrap, feature sampling)
 * without fixing a generator.  Both implementations here use one
 * counter-based generator, Philox4x32-10 (Salmon, Moraes, Dror, Shaw,
 * "Parallel random numbers: as easy as 1, 2, 3", SC'11), so that the CPU
 * oracle and the GPU draw identical numbers without sharing code.
 *
 * Counter layout (all streams):  key = (seed lo32, seed hi32)
 *   w0 = draw index, w1 = sub index, w2 = (t << 24) | unit, w3 = (purpose << 24) | job
 *
 * Row permutations (Alg. 1 shuffle of each shadow column, Alg. 3
 * flush_index) and the per-node feature sample use a keyed 8-round balanced
 * Feistel network on [0, 4^h) with cycle walking down to [0, n) (Black &
 * Rogaway, "Ciphers with arbitrary finite domains", CT-RSA 2002).  Round r
 * maps (L, R) -> (R, L xor (fmix32(R xor K_r) & mask)); fmix32 is the
 * MurmurHash3 32-bit finaliser; K_0..K_7 are the 8 words of two Philox
 * calls with w0 = 0 and w0 = 1.
 */
#include "oracle.h"

#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; round++) {
    if (round > 0) { /* key schedule: add the Weyl constants between rounds */
      k0 += PHILOX_W0;
      k1 += PHILOX_W1;
    }
    uint64_t p0 = (uint64_t)PHILOX_M0 * c0;
    uint64_t p1 = (uint64_t)PHILOX_M1 * c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    uint32_t n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

uint32_t orc_fmix32(uint32_t x) {
  x ^= x >> 16;
  x *= 0x85EBCA6Bu;
  x ^= x >> 13;
  x *= 0xC2B2AE35u;
  x ^= x >> 16;
  return x;
}

static uint64_t philox64(uint64_t seed, uint32_t w0, uint32_t w1, uint32_t w2, uint32_t w3) {
  uint32_t ctr[4] = {w0, w1, w2, w3};
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  uint32_t out[4];
  orc_philox4x32_10(ctr, key, out);
  return (uint64_t)out[0] | ((uint64_t)out[1] << 32);
}

/* floor(r * n / 2^64): maps a uniform 64-bit draw onto [0, n). */
static uint64_t scale64(uint64_t r, uint64_t n) {
  return (uint64_t)(((unsigned __int128)r * n) >> 64);
}

typedef struct {
  uint64_t n;
  int h;          /* bits per Feistel half */
  uint32_t mask;
  uint32_t K[8];
} perm_t;

static void perm_init(perm_t* P, uint64_t n, uint64_t seed, uint32_t w1, uint32_t w2,
                      uint32_t w3) {
  P->n = n;
  int h = 1;
  while ((1ull << (2 * h)) < n) h++;
  P->h = h;
  P->mask = (uint32_t)((1ull << h) - 1);
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  for (uint32_t call = 0; call < 2; call++) {
    uint32_t ctr[4] = {call, w1, w2, w3};
    orc_philox4x32_10(ctr, key, &P->K[4 * call]);
  }
}

static uint64_t feistel_once(const perm_t* P, uint64_t x) {
  uint32_t L = (uint32_t)(x >> P->h);
  uint32_t R = (uint32_t)(x & P->mask);
  for (int r = 0; r < 8; r++) {
    uint32_t T = L ^ (orc_fmix32(R ^ P->K[r]) & P->mask);
    L = R;
    R = T;
  }
  return ((uint64_t)L << P->h) | R;
}

static uint64_t perm_apply(const perm_t* P, uint64_t i) {
  if (P->n <= 1) return i;
  uint64_t x = feistel_once(P, i);
  while (x >= P->n) x = feistel_once(P, x); /* cycle walking */
  return x;
}

void orc_perm(uint64_t n, uint64_t seed, uint32_t w1, uint32_t w2, uint32_t w3,
              const uint64_t* idx, uint64_t* out, int64_t count) {
  perm_t P;
  perm_init(&P, n, seed, w1, w2, w3);
  for (int64_t k = 0; k < count; k++) out[k] = perm_apply(&P, idx[k]);
}

/* Bootstrap of tree `tree` in iteration t: N draws with replacement,
 * counts[i] = number of times row i was drawn (0 = out of bag). */
void orc_bootstrap(uint64_t seed, uint32_t job, int t, int tree, int64_t N, uint32_t* counts) {
  for (int64_t i = 0; i < N; i++) counts[i] = 0;
  uint32_t w2 = ((uint32_t)t << 24) | ((uint32_t)tree & 0xFFFFFFu);
  uint32_t w3 = (ORC_P_BOOT << 24) | (job & 0xFFFFFFu);
  for (int64_t d = 0; d < N; d++) {
    uint64_t r = philox64(seed, (uint32_t)d, 0u, w2, w3);
    counts[scale64(r, (uint64_t)N)] += 1;
  }
}

/* Features tried at node `heap` of tree `tree`: the first mtry images of
 * the node's keyed permutation of [0, p_aug). */
void orc_mtry(uint64_t seed, uint32_t job, int t, int tree, uint32_t heap, int64_t p_aug,
              int mtry, uint32_t* feats) {
  perm_t P;
  perm_init(&P, (uint64_t)p_aug, seed, heap, ((uint32_t)t << 24) | ((uint32_t)tree & 0xFFFFFFu),
            (ORC_P_MTRY << 24) | (job & 0xFFFFFFu));
  for (int k = 0; k < mtry; k++) feats[k] = (uint32_t)perm_apply(&P, (uint64_t)k);
}

static int64_t isqrt64(int64_t v) {
  int64_t r = 0;
  while ((r + 1) * (r + 1) <= v) r++;
  return r;
}

/* Breiman's defaults: sqrt(p) for classification, p/3 for regression,
 * taken over the augmented column count of the current iteration. */
int64_t orc_default_mtry(int task, int64_t p_aug) {
  int64_t m = ((task & 1) == ORC_REGRESSION) ? p_aug / 3 : isqrt64(p_aug);
  if (m < 1) m = 1;
  return m;
}

/* Alg. 1: the shadow block starts as a copy of X_cur and is doubled
 * column-wise until it has at least five columns. */
int64_t orc_shadow_count(int64_t p_live) {
  int64_t n = p_live;
  if (n <= 0) return 0;
  while (n < 5) n *= 2;
  return n;
}

/* Alg. 1 shuffle, one row permutation per shadow column:
 * Xsha[c][i] = X[sigma_c(i)][live[c mod p_live]]. */
void orc_shadow(const orc_problem* P, int t, const int32_t* live, int64_t p_live,
                uint8_t* Xsha) {
  int64_t n_sha = orc_shadow_count(p_live);
  for (int64_t c = 0; c < n_sha; c++) {
    perm_t S;
    perm_init(&S, (uint64_t)P->N, P->seed, 0u, ((uint32_t)t << 24) | ((uint32_t)c & 0xFFFFFFu),
              (ORC_P_SHADOW << 24) | (P->job & 0xFFFFFFu));
    const uint8_t* src = P->X + (int64_t)live[c % p_live] * P->ld;
    uint8_t* dst = Xsha + c * P->N;
    for (int64_t i = 0; i < P->N; i++) dst[i] = src[perm_apply(&S, (uint64_t)i)];
  }
}

/* Alg. 3's flush_index: one permutation of the N rows per iteration,
 * shared by every feature and tree.  pi[i] = sigma(i). */
void orc_permut_table(const orc_problem* P, int t, uint64_t* pi) {
  perm_t S;
  perm_init(&S, (uint64_t)P->N, P->seed, 0u, ((uint32_t)t << 24),
            (ORC_P_PERMUT << 24) | (P->job & 0xFFFFFFu));
  for (int64_t i = 0; i < P->N; i++) pi[i] = perm_apply(&S, (uint64_t)i);
}
