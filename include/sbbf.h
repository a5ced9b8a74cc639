/*
 * sbbf.h -- C ABI of a GB300 (sm_103a) library for split block Bloom filters
 * (J. Apple, "Split block Bloom filters", arXiv 2101.01719).
 *
 * The method (paper, intro and appendix figure):
 *   - a filter is an array of num_blocks 256-bit blocks, all zero when empty;
 *   - a 64-bit hash h selects block b = ((h >> 32) * num_blocks) >> 32
 *     (appendix, block_index);
 *   - the low 32 bits x of h give one bit per 32-bit lane i = 0..7 of that
 *     block: bit ((s_i * x mod 2^32) >> 27), s_i eight fixed odd seeds
 *     (intro, multiply-shift hashing into [0,32); appendix, make_mask);
 *   - insert ORs those eight bits into the block (appendix, add_hash);
 *     lookup answers true iff all eight are set (appendix, find_hash);
 *   - there is no delete (intro).
 *
 * Memory layout of a filter in device memory: num_blocks * 32 bytes, 256-byte
 * aligned when the library allocates it; block b is bytes [32b, 32b+32) and
 * lane i of block b is the little-endian uint32 at byte 32b + 4i (the layout
 * of one 256-bit vector per block in the appendix figure).
 *
 * Lookup results are packed LSB-first: bit (k % 32) of uint32 word (k / 32)
 * answers hash k; bits past the last hash are written as zero.  An output
 * buffer for n hashes holds (n + 31) / 32 words.
 *
 * Conventions for every entry point:
 *   - pointers named d_* are device pointers on the current CUDA device,
 *     owned by the caller unless stated otherwise; h_* are host pointers;
 *   - work is enqueued on the caller's stream `stream` (NULL: the legacy
 *     default stream) and is asynchronous unless stated otherwise; the call
 *     returns once the work is enqueued;
 *   - hashes are hash values, not keys: hashing a key is the caller's step
 *     (intro: the key is hashed once to pick the block);
 *   - calls return a status code and never abort; SBBF_ECUDA means a CUDA
 *     runtime call failed, and sbbf_last_cuda_error() gives its code;
 *   - concurrent inserts into one filter from several streams are safe (the
 *     kernels OR atomically, and OR is order-independent); a lookup that
 *     overlaps an insert into the same filter may see any subset of the
 *     overlapping insert's bits.
 */
#ifndef SBBF_H
#define SBBF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Same object as cudaStream_t / CUstream; NULL is the legacy default stream. */
typedef struct CUstream_st *sbbf_stream_t;

typedef enum sbbf_status {
  SBBF_OK = 0,
  SBBF_EINVAL = 1,   /* invalid argument (NULL pointer with n > 0, zero
                        blocks, mismatched filters, filter on another device) */
  SBBF_ENOMEM = 2,   /* device or host allocation failed */
  SBBF_ECUDA = 3,    /* a CUDA runtime call or launch failed */
  SBBF_EBUSY = 4,    /* admission refused: budget or slots exhausted */
  SBBF_ETIMEOUT = 5, /* a device-side wait reached its deadline */
  SBBF_ERANGE = 6    /* a size exceeds a stated maximum */
} sbbf_status;

/* Static string naming a status code. */
const char *sbbf_status_string(int status);

/* The cudaError_t value behind the last SBBF_ECUDA returned on this host
 * thread (0 if none). */
int sbbf_last_cuda_error(void);

/* Library version, (major << 16) | minor. */
uint32_t sbbf_version(void);

/* ------------------------------------------------------------------------
 * Single filter
 * ---------------------------------------------------------------------- */

typedef struct sbbf_filter sbbf_t;

/* Create an empty filter of num_blocks 256-bit blocks on the current device.
 * The library allocates and zero-fills num_blocks * 32 bytes (synchronously)
 * and owns them.  num_blocks is 32-bit as in the appendix's block_index, so
 * a filter holds at most 2^32 - 1 blocks (128 GiB).
 * Errors: SBBF_EINVAL (num_blocks == 0 or out == NULL), SBBF_ENOMEM,
 * SBBF_ECUDA. */
sbbf_status sbbf_create(uint32_t num_blocks, sbbf_t **out);

/* Wrap caller-owned device memory d_words (num_blocks * 32 bytes, 32-byte
 * aligned, e.g. a framework tensor) as a filter without copying or clearing
 * it.  The memory must outlive the handle; sbbf_destroy frees only the
 * handle.  Errors: SBBF_EINVAL (NULL, zero blocks, misaligned). */
sbbf_status sbbf_wrap(uint32_t *d_words, uint32_t num_blocks, sbbf_t **out);

/* Copy h_words (num_blocks * 8 uint32 in the layout above) into a new
 * library-owned filter (synchronous).  Errors as sbbf_create. */
sbbf_status sbbf_create_from_host(const uint32_t *h_words, uint32_t num_blocks,
                                  sbbf_t **out);

/* Free a filter (synchronises the device first if it owns memory).
 * NULL is a no-op. */
sbbf_status sbbf_destroy(sbbf_t *f);

/* Number of blocks (0 for NULL). */
uint32_t sbbf_num_blocks(const sbbf_t *f);

/* Device address and size in bytes of the filter words. */
sbbf_status sbbf_device_words(const sbbf_t *f, uint32_t **d_words,
                              size_t *bytes);

/* Reset every bit to zero (enqueued on stream). */
sbbf_status sbbf_clear(sbbf_t *f, sbbf_stream_t stream);

/* Insert d_hashes[0..n) (appendix add_hash for each).  d_hashes is any
 * 8-byte aligned device array; 16-byte alignment takes the vector path.
 * Duplicates and any order give the same filter.  n == 0 is a no-op.
 * Errors: SBBF_EINVAL (f NULL, d_hashes NULL with n > 0, misaligned),
 * SBBF_ECUDA (launch). */
sbbf_status sbbf_insert_hashes(sbbf_t *f, const uint64_t *d_hashes, size_t n,
                               sbbf_stream_t stream);

/* Look up d_hashes[0..n) (appendix find_hash for each) into the packed
 * bitmask d_out_bits of (n + 31) / 32 words (caller-owned, 4-byte aligned).
 * Errors as sbbf_insert_hashes; d_out_bits NULL with n > 0 is SBBF_EINVAL. */
sbbf_status sbbf_find_hashes(const sbbf_t *f, const uint64_t *d_hashes,
                             size_t n, uint32_t *d_out_bits,
                             sbbf_stream_t stream);

/* dst |= src word by word: afterwards dst answers true for every hash either
 * filter held.  Not in the paper; meaningful only for equal num_blocks (the
 * seeds are fixed).  Errors: SBBF_EINVAL (NULL or num_blocks differ). */
sbbf_status sbbf_union(sbbf_t *dst, const sbbf_t *src, sbbf_stream_t stream);

/* Copy the filter words to host memory h_words of at least
 * num_blocks * 32 bytes; synchronises the stream before returning.
 * Errors: SBBF_EINVAL (NULL or bytes too small), SBBF_ECUDA. */
sbbf_status sbbf_copy_to_host(const sbbf_t *f, uint32_t *h_words, size_t bytes,
                              sbbf_stream_t stream);

/* ------------------------------------------------------------------------
 * Host-buffer path: copies, kernels and result copies pipelined in chunks.
 * ---------------------------------------------------------------------- */

typedef struct sbbf_host_pipe sbbf_host_pipe_t;

/* Staging for host-buffer calls: two device buffers of chunk_hashes hashes
 * (chunk_hashes a positive multiple of 64) and their result words, plus the
 * streams and events that overlap host->device copies, kernels and
 * device->host copies.  Allocates device memory (synchronous).
 * Errors: SBBF_EINVAL, SBBF_ENOMEM, SBBF_ECUDA. */
sbbf_status sbbf_host_pipe_create(size_t chunk_hashes, sbbf_host_pipe_t **out);
sbbf_status sbbf_host_pipe_destroy(sbbf_host_pipe_t *p);

/* Insert / look up hashes held in HOST memory (pinned memory overlaps copies
 * with kernels; pageable memory works but serialises).  The call returns when
 * every result is in h_out_bits ((n + 31) / 32 words, host memory), i.e. it
 * is synchronous.  Kernels and copies are ordered after prior work on
 * `stream`.  Errors as the device-pointer forms. */
sbbf_status sbbf_insert_hashes_host(sbbf_t *f, sbbf_host_pipe_t *p,
                                    const uint64_t *h_hashes, size_t n,
                                    sbbf_stream_t stream);
sbbf_status sbbf_find_hashes_host(const sbbf_t *f, sbbf_host_pipe_t *p,
                                  const uint64_t *h_hashes, size_t n,
                                  uint32_t *h_out_bits, sbbf_stream_t stream);

/* ------------------------------------------------------------------------
 * Synthetic inputs (not part of the method): splitmix64 in counter form,
 * Steele, Lea and Flood, OOPSLA 2014.  Output i of the stream with `seed` is
 * mix(seed + (i + 1) * 0x9E3779B97F4A7C15).
 * ---------------------------------------------------------------------- */

/* d_out[k] = output (start + k) of the stream, k in [0, n). */
sbbf_status sbbf_fill_splitmix64(uint64_t *d_out, size_t n, uint64_t seed,
                                 uint64_t start, sbbf_stream_t stream);

/* Query stream mixing members and fresh hashes.  For k in [0, n), j =
 * start + k and r = output j of member_seed: if (r >> 32) < member_threshold
 * the query is output (ins_start + (((r & 0xffffffff) * n_inserted) >> 32))
 * of ins_seed (a previously inserted hash), else output j of fresh_seed.
 * Errors: SBBF_EINVAL if n_inserted == 0 while member_threshold > 0. */
sbbf_status sbbf_fill_queries(uint64_t *d_out, size_t n, uint64_t start,
                              uint64_t ins_seed, uint64_t ins_start,
                              uint64_t n_inserted, uint64_t fresh_seed,
                              uint64_t member_seed, uint64_t member_threshold,
                              sbbf_stream_t stream);

/* Number of set bits in the packed bitmask d_bits over its first n bits,
 * written to *d_count (uint64, device) -- used to count lookup hits. */
sbbf_status sbbf_count_bits(const uint32_t *d_bits, size_t n,
                            unsigned long long *d_count, sbbf_stream_t stream);

#ifdef __cplusplus
}
#endif
#endif /* SBBF_H */
