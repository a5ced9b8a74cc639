/*
 * Scalar reference ("oracle") for split block Bloom filters
 * (Apple, "Split block Bloom filters", arXiv 2101.01719).
 *
 * TEST INFRASTRUCTURE ONLY: only the tests, the smoke check and the
 * benchmark's CPU-baseline leg load this code.  It is deliberately plain,
 * slow, single-threaded C99 (the *_mt drivers only split work between threads
 * that each run the same scalar code) and shares nothing with the CUDA path.
 *
 * Every function states the definition it follows.  Names refer to the
 * paper's parts: the intro (block selection, multiply-shift hashing into
 * [0,32), one bit per 32-bit lane), the FPR analysis (the Poisson sum) and
 * the appendix figure (block_index, make_mask, add_hash, find_hash).
 *
 * Readings taken where the paper is silent or garbled:
 *  - seed lane order: the appendix initialises a 256-bit vector with four
 *    64-bit elements (hi << 32 | lo); stored little-endian, lane 2j is `lo`
 *    and lane 2j+1 is `hi` of element j.
 *  - the multiply in h_s(x) = floor(s*x / 2^27) is taken modulo 2^32 (the
 *    appendix multiplies 32-bit lanes keeping the low half), so the result
 *    lies in [0,32); the figure's "[0, 31)" comment is a typo for [0, 32).
 *  - make_mask receives the low 32 bits of the 64-bit hash; block_index uses
 *    the high 32 bits.
 *  - an empty filter is all zero bits.
 */
#define _POSIX_C_SOURCE 200809L
#include "sbbf_oracle.h"

#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

/* Eight odd 32-bit multipliers, lane 0..7 (appendix figure; lane order is the
 * little-endian layout of its four 64-bit initialiser elements). */
static const uint32_t kSeed[8] = {
    0x44974d91u, 0x47b6137bu, 0xa2b7289du, 0x8824ad5bu,
    0x2df1424bu, 0x705495c7u, 0x5c6bfb31u, 0x9efc4947u,
};

void oracle_seeds(uint32_t out[8]) {
  for (int i = 0; i < 8; ++i) out[i] = kSeed[i];
}

/* Appendix, block_index: ((hash >> 32) * num_blocks) >> 32.  Both factors
 * are below 2^32, so the 64-bit product cannot overflow. */
uint64_t oracle_block_index(uint64_t hash, uint32_t num_blocks) {
  uint64_t high = hash >> 32;
  uint64_t product = high * (uint64_t)num_blocks;
  return product >> 32;
}

/* Intro: h_{s_i}(x) = floor((s_i * x) / 2^27) with odd seeds s_i, product
 * modulo 2^32 (appendix multiplies 32-bit lanes), giving a bit index in
 * [0,32); appendix make_mask sets that bit in lane i. */
void oracle_make_mask(uint32_t x, uint32_t mask[8]) {
  for (int i = 0; i < 8; ++i) {
    uint32_t product = (uint32_t)(kSeed[i] * x); /* mod 2^32 */
    uint32_t bit = product >> 27;                /* top five bits */
    mask[i] = (uint32_t)1u << bit;
  }
}

/* Appendix, add_hash: OR the mask into the selected 256-bit block. */
static void insert_one(uint32_t *words, uint32_t num_blocks, uint64_t hash) {
  uint64_t b = oracle_block_index(hash, num_blocks);
  uint32_t mask[8];
  oracle_make_mask((uint32_t)hash, mask);
  for (int i = 0; i < 8; ++i) words[8 * b + i] |= mask[i];
}

void oracle_insert(uint32_t *words, uint32_t num_blocks,
                   const uint64_t *hashes, size_t n) {
  for (size_t k = 0; k < n; ++k) insert_one(words, num_blocks, hashes[k]);
}

void oracle_insert_block_range(uint32_t *sub_words, uint32_t num_blocks,
                               const uint64_t *hashes, size_t n,
                               uint64_t lo, uint64_t hi) {
  for (size_t k = 0; k < n; ++k) {
    uint64_t b = oracle_block_index(hashes[k], num_blocks);
    if (b < lo || b >= hi) continue;
    uint32_t mask[8];
    oracle_make_mask((uint32_t)hashes[k], mask);
    for (int i = 0; i < 8; ++i) sub_words[8 * (b - lo) + i] |= mask[i];
  }
}

/* add_hash restricted to several sorted, disjoint block ranges; the output
 * holds the ranges' blocks one after another. */
void oracle_insert_block_ranges(uint32_t *out_words, uint32_t num_blocks,
                                const uint64_t *hashes, size_t n,
                                const uint64_t *lo, const uint64_t *hi,
                                size_t n_ranges) {
  if (n_ranges == 0) return;
  uint64_t *first = (uint64_t *)malloc(n_ranges * sizeof(uint64_t));
  uint64_t acc = 0;
  for (size_t r = 0; r < n_ranges; ++r) {
    first[r] = acc;
    acc += hi[r] - lo[r];
  }
  for (size_t k = 0; k < n; ++k) {
    uint64_t b = oracle_block_index(hashes[k], num_blocks);
    if (b < lo[0]) continue;
    size_t a = 0, z = n_ranges; /* last r with lo[r] <= b: in [a, z) */
    while (z - a > 1) {
      size_t mid = (a + z) / 2;
      if (lo[mid] <= b) a = mid; else z = mid;
    }
    if (b >= hi[a]) continue;
    uint32_t mask[8];
    oracle_make_mask((uint32_t)hashes[k], mask);
    for (int i = 0; i < 8; ++i) out_words[8 * (first[a] + b - lo[a]) + i] |= mask[i];
  }
  free(first);
}

/* Appendix, find_hash: true iff (~block & mask) == 0, i.e. every lane's mask
 * bit is set in the block. */
int oracle_find_one(const uint32_t *words, uint32_t num_blocks,
                    uint64_t hash) {
  uint64_t b = oracle_block_index(hash, num_blocks);
  uint32_t mask[8];
  oracle_make_mask((uint32_t)hash, mask);
  for (int i = 0; i < 8; ++i) {
    if ((~words[8 * b + i] & mask[i]) != 0) return 0;
  }
  return 1;
}

void oracle_find(const uint32_t *words, uint32_t num_blocks,
                 const uint64_t *hashes, size_t n, uint32_t *out_bits) {
  size_t n_out = (n + 31) / 32;
  for (size_t w = 0; w < n_out; ++w) out_bits[w] = 0;
  for (size_t k = 0; k < n; ++k) {
    if (oracle_find_one(words, num_blocks, hashes[k]))
      out_bits[k / 32] |= (uint32_t)1u << (k % 32);
  }
}

void oracle_union(uint32_t *dst, const uint32_t *src, size_t n_words) {
  for (size_t w = 0; w < n_words; ++w) dst[w] |= src[w];
}

/* Several filters in one arena: filter t is the plain filter of
 * num_blocks[t] blocks whose block 0 is arena block base_block[t]. */
uint64_t oracle_multi_insert(uint32_t *arena, const uint64_t *base_block,
                             const uint32_t *num_blocks, uint32_t n_filters,
                             const uint64_t *hashes, const uint32_t *ids,
                             size_t n) {
  uint64_t invalid = 0;
  for (size_t k = 0; k < n; ++k) {
    uint32_t t = ids[k];
    if (t >= n_filters) {
      ++invalid;
      continue;
    }
    insert_one(arena + 8 * base_block[t], num_blocks[t], hashes[k]);
  }
  return invalid;
}

uint64_t oracle_multi_find(const uint32_t *arena, const uint64_t *base_block,
                           const uint32_t *num_blocks, uint32_t n_filters,
                           const uint64_t *hashes, const uint32_t *ids,
                           size_t n, uint32_t *out_bits) {
  uint64_t invalid = 0;
  size_t n_out = (n + 31) / 32;
  for (size_t w = 0; w < n_out; ++w) out_bits[w] = 0;
  for (size_t k = 0; k < n; ++k) {
    uint32_t t = ids[k];
    if (t >= n_filters) {
      ++invalid;
      continue;
    }
    if (oracle_find_one(arena + 8 * base_block[t], num_blocks[t], hashes[k]))
      out_bits[k / 32] |= (uint32_t)1u << (k % 32);
  }
  return invalid;
}

/* FPR analysis: sum_{i>=0} Pois_a(i) * (1 - (1 - 1/32)^i)^8, a = keys per
 * block.  The Poisson weights are formed in log space; the sum is cut where
 * the remaining tail is far below double precision. */
double oracle_fpr_poisson(double a) {
  if (!(a > 0.0)) return 0.0;
  const double q = 1.0 - 1.0 / 32.0;
  size_t i_max = (size_t)(a + 40.0 * sqrt(a + 1.0) + 200.0);
  double sum = 0.0;
  for (size_t i = 0; i <= i_max; ++i) {
    double log_p = (double)i * log(a) - a - lgamma((double)i + 1.0);
    double lane_hit = 1.0 - pow(q, (double)i);
    sum += exp(log_p) * pow(lane_hit, 8.0);
  }
  return sum;
}

double oracle_fpr_standard(double bits_per_key, double k) {
  return pow(1.0 - exp(-k / bits_per_key), k);
}

/* splitmix64 (Steele, Lea, Flood 2014; Vigna's public-domain generator),
 * counter form: state after i+1 steps is seed + (i+1) * golden gamma. */
uint64_t oracle_splitmix64_at(uint64_t seed, uint64_t i) {
  uint64_t z = seed + (i + 1) * UINT64_C(0x9E3779B97F4A7C15);
  z = (z ^ (z >> 30)) * UINT64_C(0xBF58476D1CE4E5B9);
  z = (z ^ (z >> 27)) * UINT64_C(0x94D049BB133111EB);
  return z ^ (z >> 31);
}

void oracle_splitmix64_fill(uint64_t seed, uint64_t start, size_t n,
                            uint64_t *out) {
  for (size_t k = 0; k < n; ++k) out[k] = oracle_splitmix64_at(seed, start + k);
}

/* ---- lane-count variants ----------------------------------------------
 * The design list says four or sixteen lanes would work as well as eight.  A
 * k-lane block is k consecutive 32-bit words; block selection is the
 * appendix block_index over the filter's k-lane blocks, and lane i sets bit
 * (s_i * x mod 2^32) >> 27 of word i, x the low 32 bits of the hash.
 * Readings (the paper names no seeds beyond eight): k = 4 uses lanes 0..3 of
 * the eight appendix seeds; k = 16 uses the eight appendix seeds followed by
 * s_{8+j} = (splitmix64 output j of seed 0 >> 32) | 1, j = 0..7 (odd, as
 * multiply-shift hashing requires). */
uint32_t oracle_seed_k(int i) {
  if (i < 8) return kSeed[i];
  return (uint32_t)(oracle_splitmix64_at(0, (uint64_t)(i - 8)) >> 32) | 1u;
}

static int lanes_ok(int k) { return k == 4 || k == 8 || k == 16; }

int oracle_insert_k(uint32_t *words, uint32_t num_blocks, int k,
                    const uint64_t *hashes, size_t n) {
  if (!lanes_ok(k)) return -1;
  for (size_t j = 0; j < n; ++j) {
    uint64_t b = oracle_block_index(hashes[j], num_blocks);
    uint32_t x = (uint32_t)hashes[j];
    for (int i = 0; i < k; ++i) {
      uint32_t bit = (uint32_t)(oracle_seed_k(i) * x) >> 27;
      words[(uint64_t)k * b + (uint64_t)i] |= (uint32_t)1u << bit;
    }
  }
  return 0;
}

int oracle_find_k(const uint32_t *words, uint32_t num_blocks, int k,
                  const uint64_t *hashes, size_t n, uint32_t *out_bits) {
  if (!lanes_ok(k)) return -1;
  for (size_t w = 0; w < (n + 31) / 32; ++w) out_bits[w] = 0;
  for (size_t j = 0; j < n; ++j) {
    uint64_t b = oracle_block_index(hashes[j], num_blocks);
    uint32_t x = (uint32_t)hashes[j];
    int hit = 1;
    for (int i = 0; i < k; ++i) {
      uint32_t bit = (uint32_t)(oracle_seed_k(i) * x) >> 27;
      if ((words[(uint64_t)k * b + (uint64_t)i] & ((uint32_t)1u << bit)) == 0) hit = 0;
    }
    if (hit) out_bits[j / 32] |= (uint32_t)1u << (j % 32);
  }
  return 0;
}

/* FPR analysis with k lanes: sum_i Pois_a(i) * (1 - (1 - 1/32)^i)^k. */
double oracle_fpr_poisson_k(double a, int k) {
  if (!(a > 0.0)) return 0.0;
  const double q = 1.0 - 1.0 / 32.0;
  size_t i_max = (size_t)(a + 40.0 * sqrt(a + 1.0) + 200.0);
  double sum = 0.0;
  for (size_t i = 0; i <= i_max; ++i) {
    double log_p = (double)i * log(a) - a - lgamma((double)i + 1.0);
    sum += exp(log_p) * pow(1.0 - pow(q, (double)i), (double)k);
  }
  return sum;
}

/* ---- key hashing --------------------------------------------------------
 * The paper hashes each key once to 64 bits and fixes no hash function.
 * Parquet, one of the adopters the paper lists, uses XXH64 with seed 0; this
 * is XXH64 as its published specification defines it (Y. Collet, "xxHash
 * fast digest algorithm", XXH64): four accumulators over 32-byte stripes for
 * inputs of 32 bytes or more, then the length, then 8-, 4- and 1-byte tail
 * steps, then the final avalanche.  Input bytes are read little-endian. */
#define XP1 UINT64_C(0x9E3779B185EBCA87)
#define XP2 UINT64_C(0xC2B2AE3D27D4EB4F)
#define XP3 UINT64_C(0x165667B19E3779F9)
#define XP4 UINT64_C(0x85EBCA77C2B2AE63)
#define XP5 UINT64_C(0x27D4EB2F165667C5)

static uint64_t xrotl(uint64_t x, int r) { return (x << r) | (x >> (64 - r)); }

static uint64_t read_le(const uint8_t *p, int bytes) {
  uint64_t v = 0;
  for (int i = bytes - 1; i >= 0; --i) v = (v << 8) | p[i];
  return v;
}

static uint64_t xround(uint64_t acc, uint64_t lane) {
  acc += lane * XP2;
  acc = xrotl(acc, 31);
  return acc * XP1;
}

static uint64_t xmerge(uint64_t acc, uint64_t v) {
  acc ^= xround(0, v);
  return acc * XP1 + XP4;
}

uint64_t oracle_xxh64(const void *data, size_t len, uint64_t seed) {
  const uint8_t *p = (const uint8_t *)data;
  size_t i = 0;
  uint64_t acc;
  if (len >= 32) {
    uint64_t v1 = seed + XP1 + XP2, v2 = seed + XP2, v3 = seed, v4 = seed - XP1;
    for (; i + 32 <= len; i += 32) {
      v1 = xround(v1, read_le(p + i, 8));
      v2 = xround(v2, read_le(p + i + 8, 8));
      v3 = xround(v3, read_le(p + i + 16, 8));
      v4 = xround(v4, read_le(p + i + 24, 8));
    }
    acc = xrotl(v1, 1) + xrotl(v2, 7) + xrotl(v3, 12) + xrotl(v4, 18);
    acc = xmerge(acc, v1);
    acc = xmerge(acc, v2);
    acc = xmerge(acc, v3);
    acc = xmerge(acc, v4);
  } else {
    acc = seed + XP5;
  }
  acc += (uint64_t)len;
  for (; i + 8 <= len; i += 8) {
    acc ^= xround(0, read_le(p + i, 8));
    acc = xrotl(acc, 27) * XP1 + XP4;
  }
  if (i + 4 <= len) {
    acc ^= read_le(p + i, 4) * XP1;
    acc = xrotl(acc, 23) * XP2 + XP3;
    i += 4;
  }
  for (; i < len; ++i) {
    acc ^= (uint64_t)p[i] * XP5;
    acc = xrotl(acc, 11) * XP1;
  }
  acc ^= acc >> 33;
  acc *= XP2;
  acc ^= acc >> 29;
  acc *= XP3;
  acc ^= acc >> 32;
  return acc;
}

void oracle_xxh64_fixed(const void *keys, size_t key_bytes, size_t n,
                        uint64_t seed, uint64_t *out) {
  const uint8_t *p = (const uint8_t *)keys;
  for (size_t k = 0; k < n; ++k) out[k] = oracle_xxh64(p + k * key_bytes, key_bytes, seed);
}

void oracle_xxh64_var(const uint8_t *data, const uint64_t *offsets, size_t n,
                      uint64_t seed, uint64_t *out) {
  for (size_t k = 0; k < n; ++k)
    out[k] = oracle_xxh64(data + offsets[k], (size_t)(offsets[k + 1] - offsets[k]), seed);
}

/* Parquet's block layout.  Parquet lists its eight salts in the order the
 * paper's text prints the appendix constants, which swaps each pair of the
 * appendix's little-endian lane order: Parquet lane i uses the multiplier of
 * appendix lane i ^ 1.  The same keys therefore give the same blocks with
 * words 2j and 2j+1 exchanged; this maps one layout to the other (the map is
 * its own inverse). */
void oracle_swap_lane_pairs(const uint32_t *in, size_t n_words, uint32_t *out) {
  for (size_t w = 0; w < n_words; ++w) out[w] = in[w ^ 1];
}

/* ---- verification digest (a checking aid; not part of the method) -------
 * The filter's words, read as 64-bit units (unit u holds word 2u in its low
 * half and word 2u+1 in its high half, the little-endian pairing), are split
 * into ranges of range_blocks blocks: range r holds the blocks
 * [r * range_blocks, min(num_blocks, (r + 1) * range_blocks)).  `words` may
 * start at block first_block of a larger filter (a multiple of range_blocks,
 * so that callers can split the work at range boundaries): unit indexes are
 * then those of the whole filter and r counts from the slice's first range.
 * For each range:
 *   digest[r]  = sum over the range's units u of splitmix64 output u of the
 *                stream seeded with the unit's value, mod 2^64;
 *   bits[r]    = number of set bits in the range;
 *   partial[r] = number of its blocks holding both an all-zero lane and a
 *                non-zero lane.
 * Every insert sets one bit in each lane of its block (the make_mask step),
 * and a union ORs whole blocks, so partial is 0 for any filter built by them. */
void oracle_range_digest(const uint32_t *words, uint64_t first_block,
                         uint64_t num_blocks, int lanes, uint64_t range_blocks,
                         uint64_t *digest, uint64_t *bits, uint64_t *partial) {
  const uint64_t n_ranges = (num_blocks + range_blocks - 1) / range_blocks;
  for (uint64_t r = 0; r < n_ranges; ++r) {
    digest[r] = 0;
    bits[r] = 0;
    partial[r] = 0;
  }
  for (uint64_t b = 0; b < num_blocks; ++b) {
    const uint64_t r = b / range_blocks;
    const uint32_t *blk = words + b * (uint64_t)lanes;
    int zero_lanes = 0;
    for (int i = 0; i < lanes; ++i) {
      uint32_t w = blk[i];
      if (w == 0) ++zero_lanes;
      while (w) { /* one pass per set bit: clear the lowest */
        bits[r] += 1;
        w &= w - 1u;
      }
    }
    if (zero_lanes > 0 && zero_lanes < lanes) ++partial[r];
    for (int i = 0; i < lanes; i += 2) {
      const uint64_t u = ((first_block + b) * (uint64_t)lanes + (uint64_t)i) / 2;
      const uint64_t v = (uint64_t)blk[i] | ((uint64_t)blk[i + 1] << 32);
      digest[r] += oracle_splitmix64_at(v, u);
    }
  }
}

int oracle_num_cores(void) {
  long c = sysconf(_SC_NPROCESSORS_ONLN);
  return c > 0 ? (int)c : 1;
}

/* ---- timing drivers: same scalar code, disjoint pieces per thread ---- */

struct find_job {
  const uint32_t *words;
  uint32_t num_blocks;
  const uint64_t *hashes;
  size_t n;
  uint32_t *out_bits;
};

static void *find_worker(void *arg) {
  struct find_job *j = (struct find_job *)arg;
  oracle_find(j->words, j->num_blocks, j->hashes, j->n, j->out_bits);
  return NULL;
}

int oracle_find_mt(const uint32_t *words, uint32_t num_blocks,
                   const uint64_t *hashes, size_t n, uint32_t *out_bits,
                   int n_threads) {
  if (n_threads < 1) n_threads = 1;
  size_t groups = (n + 31) / 32;
  if ((size_t)n_threads > groups) n_threads = groups > 0 ? (int)groups : 1;
  pthread_t *tid = (pthread_t *)calloc((size_t)n_threads, sizeof(pthread_t));
  struct find_job *job =
      (struct find_job *)calloc((size_t)n_threads, sizeof(struct find_job));
  for (int t = 0; t < n_threads; ++t) {
    size_t g0 = groups * (size_t)t / (size_t)n_threads;
    size_t g1 = groups * (size_t)(t + 1) / (size_t)n_threads;
    size_t k0 = 32 * g0, k1 = 32 * g1 < n ? 32 * g1 : n;
    job[t].words = words;
    job[t].num_blocks = num_blocks;
    job[t].hashes = hashes + k0;
    job[t].n = k1 > k0 ? k1 - k0 : 0;
    job[t].out_bits = out_bits + g0;
    pthread_create(&tid[t], NULL, find_worker, &job[t]);
  }
  for (int t = 0; t < n_threads; ++t) pthread_join(tid[t], NULL);
  free(tid);
  free(job);
  return n_threads;
}

struct insert_job {
  uint32_t *words;
  uint32_t num_blocks;
  const uint64_t *hashes;
  size_t n;
  uint64_t lo, hi;
};

static void *insert_worker(void *arg) {
  struct insert_job *j = (struct insert_job *)arg;
  oracle_insert_block_range(j->words + 8 * j->lo, j->num_blocks, j->hashes,
                            j->n, j->lo, j->hi);
  return NULL;
}

int oracle_insert_mt(uint32_t *words, uint32_t num_blocks,
                     const uint64_t *hashes, size_t n, int n_threads) {
  if (n_threads < 1) n_threads = 1;
  if ((uint32_t)n_threads > num_blocks) n_threads = (int)num_blocks;
  pthread_t *tid = (pthread_t *)calloc((size_t)n_threads, sizeof(pthread_t));
  struct insert_job *job =
      (struct insert_job *)calloc((size_t)n_threads, sizeof(struct insert_job));
  for (int t = 0; t < n_threads; ++t) {
    job[t].words = words;
    job[t].num_blocks = num_blocks;
    job[t].hashes = hashes;
    job[t].n = n;
    job[t].lo = (uint64_t)num_blocks * (uint64_t)t / (uint64_t)n_threads;
    job[t].hi = (uint64_t)num_blocks * (uint64_t)(t + 1) / (uint64_t)n_threads;
    pthread_create(&tid[t], NULL, insert_worker, &job[t]);
  }
  for (int t = 0; t < n_threads; ++t) pthread_join(tid[t], NULL);
  free(tid);
  free(job);
  return n_threads;
}
