/*
 * Scalar reference ("oracle") for split block Bloom filters (Apple,
 * "Split block Bloom filters", arXiv 2101.01719).
 *
 * TEST INFRASTRUCTURE ONLY.  This header and sbbf_oracle.c are used by the
 * test suite, by the smoke check and by the benchmark's CPU-baseline leg.
 * The product library (the CUDA path) never includes, links or calls it, and
 * it shares no header, table or helper with that path.
 *
 * Layout (shared by convention only, restated independently on each side):
 *   a filter of B blocks is B*8 little-endian uint32 words; block b occupies
 *   words [8b, 8b+8); lane i of block b is word 8b+i; bit j of a lane is
 *   (1u << j).  This is how the appendix figure stores one __m256i per block.
 *
 * Lookup results are packed LSB-first: bit (k % 32) of word (k / 32) is the
 * answer for hash k; bits past the last hash are zero.
 */
#ifndef SBBF_ORACLE_H
#define SBBF_ORACLE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Appendix figure, block_index: high 32 bits of the hash, range-reduced to
 * [0, num_blocks) by a 32x32->64 multiply and a 32-bit right shift. */
uint64_t oracle_block_index(uint64_t hash, uint32_t num_blocks);

/* Intro (multiply-shift hashing into [0,32)) and appendix figure, make_mask:
 * mask[i] = 1 << ((s_i * x mod 2^32) >> 27) for the eight odd seeds s_i. */
void oracle_make_mask(uint32_t x, uint32_t mask[8]);

/* The eight seeds in lane order 0..7 (copied out for tests). */
void oracle_seeds(uint32_t out[8]);

/* Appendix figure, add_hash, applied to hashes[0..n) in order. */
void oracle_insert(uint32_t *words, uint32_t num_blocks,
                   const uint64_t *hashes, size_t n);

/* add_hash restricted to blocks in [lo, hi): keys whose block falls outside
 * are skipped; sub_words holds blocks lo..hi-1 (word 8*(b-lo)+i). */
void oracle_insert_block_range(uint32_t *sub_words, uint32_t num_blocks,
                               const uint64_t *hashes, size_t n,
                               uint64_t lo, uint64_t hi);

/* add_hash restricted to n_ranges sorted, disjoint block ranges
 * [lo[r], hi[r]); out_words holds the ranges' blocks one after another. */
void oracle_insert_block_ranges(uint32_t *out_words, uint32_t num_blocks,
                                const uint64_t *hashes, size_t n,
                                const uint64_t *lo, const uint64_t *hi,
                                size_t n_ranges);

/* Appendix figure, find_hash for one hash: 1 iff every mask bit is set. */
int oracle_find_one(const uint32_t *words, uint32_t num_blocks, uint64_t hash);

/* find_hash over hashes[0..n) into a packed bitmask of (n+31)/32 words. */
void oracle_find(const uint32_t *words, uint32_t num_blocks,
                 const uint64_t *hashes, size_t n, uint32_t *out_bits);

/* Word-wise OR of src into dst (union of two filters with equal B). */
void oracle_union(uint32_t *dst, const uint32_t *src, size_t n_words);

/* Several filters in one word arena.  Filter t holds num_blocks[t] blocks
 * starting at block base_block[t] of the arena.  A hash with ids[k] >=
 * n_filters is skipped (insert) or answers 0 (find); the return value counts
 * such hashes. */
uint64_t oracle_multi_insert(uint32_t *arena, const uint64_t *base_block,
                             const uint32_t *num_blocks, uint32_t n_filters,
                             const uint64_t *hashes, const uint32_t *ids,
                             size_t n);
uint64_t oracle_multi_find(const uint32_t *arena, const uint64_t *base_block,
                           const uint32_t *num_blocks, uint32_t n_filters,
                           const uint64_t *hashes, const uint32_t *ids,
                           size_t n, uint32_t *out_bits);

/* False positive rate approximation (FPR analysis): sum over i of the
 * Poisson(a) probability of i keys in a block times (1-(1-1/32)^i)^8. */
double oracle_fpr_poisson(double a);

/* Standard Bloom filter FPR (1 - e^{-k/bits_per_key})^k, for the paper's
 * comparison claims only. */
double oracle_fpr_standard(double bits_per_key, double k);

/* splitmix64 (Steele, Lea, Flood, OOPSLA 2014) in counter form: output i of
 * the stream seeded with `seed` is mix(seed + (i+1)*0x9E3779B97F4A7C15). */
uint64_t oracle_splitmix64_at(uint64_t seed, uint64_t i);
void oracle_splitmix64_fill(uint64_t seed, uint64_t start, size_t n,
                            uint64_t *out);

/* Multi-threaded drivers used only to time the oracle on all host cores.
 * They call the scalar functions above on disjoint pieces of the work:
 * lookups by contiguous chunks of 32-hash groups, inserts by block range.
 * The return value is the number of threads actually used. */
int oracle_find_mt(const uint32_t *words, uint32_t num_blocks,
                   const uint64_t *hashes, size_t n, uint32_t *out_bits,
                   int n_threads);
int oracle_insert_mt(uint32_t *words, uint32_t num_blocks,
                     const uint64_t *hashes, size_t n, int n_threads);

/* Lane-count variants (k = 4, 8 or 16 lanes per block; the design list says
 * four or sixteen work as well).  A k-lane block is k words; lane i uses
 * seed oracle_seed_k(i): the appendix seeds for i < 8, and for k = 16
 * lanes 8..15 use (splitmix64(seed 0) output i-8 >> 32) | 1.  Return -1 for
 * any other k. */
uint32_t oracle_seed_k(int i);
int oracle_insert_k(uint32_t *words, uint32_t num_blocks, int k,
                    const uint64_t *hashes, size_t n);
int oracle_find_k(const uint32_t *words, uint32_t num_blocks, int k,
                  const uint64_t *hashes, size_t n, uint32_t *out_bits);
double oracle_fpr_poisson_k(double a, int k);

/* XXH64 of len bytes (published xxHash specification).  The paper hashes
 * each key once and fixes no hash; Parquet's split block filters use XXH64,
 * seed 0. */
uint64_t oracle_xxh64(const void *data, size_t len, uint64_t seed);
/* XXH64 of n fixed-width keys of key_bytes bytes each, stored back to back. */
void oracle_xxh64_fixed(const void *keys, size_t key_bytes, size_t n,
                        uint64_t seed, uint64_t *out);
/* XXH64 of n variable-length keys: key k is data[offsets[k], offsets[k+1]). */
void oracle_xxh64_var(const uint8_t *data, const uint64_t *offsets, size_t n,
                      uint64_t seed, uint64_t *out);

/* Parquet block layout: out word w = in word (w ^ 1) (Parquet lists the
 * salts in the paper text's order, pairwise swapped against the appendix's
 * little-endian lane order). */
void oracle_swap_lane_pairs(const uint32_t *in, size_t n_words, uint32_t *out);

/* Verification digest over block ranges (a checking aid, not part of the
 * method).  Range r holds blocks [r*range_blocks, min(num_blocks,
 * (r+1)*range_blocks)); digest[r] = sum mod 2^64 over the range's 64-bit units
 * u (words 2u | 2u+1 << 32) of splitmix64 output u seeded with the unit's
 * value; bits[r] = set bits; partial[r] = blocks with both a zero and a
 * non-zero lane.  Arrays hold ceil(num_blocks / range_blocks) entries;
 * lanes is 4, 8 or 16 and range_blocks >= 1.  words may be the slice of a
 * filter starting at block first_block (a multiple of range_blocks); unit
 * indexes are the whole filter's and ranges count from the slice's first. */
void oracle_range_digest(const uint32_t *words, uint64_t first_block,
                         uint64_t num_blocks, int lanes, uint64_t range_blocks,
                         uint64_t *digest, uint64_t *bits, uint64_t *partial);

/* Number of online host cores. */
int oracle_num_cores(void);

#ifdef __cplusplus
}
#endif
#endif
