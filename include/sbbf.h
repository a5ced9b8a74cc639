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

/* Lane-count variants.  The paper uses eight 32-bit lanes per block to fill a
 * 256-bit SIMD register and notes that four or sixteen lanes would work too
 * (design list, footnote).  A filter of `lanes` = 4, 8 or 16 has blocks of
 * `lanes` consecutive 32-bit words (16, 32 or 64 bytes); block selection is
 * the appendix block_index over its num_blocks blocks, and lane i of the
 * block sets bit (s_i * x mod 2^32) >> 27 of word i (x the hash's low 32
 * bits).  Lanes 0..7 use the appendix seeds; lanes 8..15 (lanes = 16) use
 * the odd constants 0xe220a839, 0x6e789e6b, 0x06c45d19, 0xf88bb8a9,
 * 0x1b39896b, 0x53cb9f0d, 0x2c829abf, 0xc584133b ((splitmix64 output j of
 * seed 0 >> 32) | 1; the paper names only eight seeds).  Filters of 4 or 16
 * lanes support the single-filter calls (insert, find, keys, union, clear,
 * copy, host pipe, serialization); they never take the partitioned path,
 * and Parquet export wants 8 lanes.  Memory: num_blocks * lanes * 4 bytes.
 * Errors: SBBF_EINVAL (lanes not 4, 8 or 16, else as sbbf_create /
 * sbbf_wrap). */
sbbf_status sbbf_create_lanes(uint32_t num_blocks, uint32_t lanes, sbbf_t **out);
sbbf_status sbbf_wrap_lanes(uint32_t *d_words, uint32_t num_blocks,
                            uint32_t lanes, sbbf_t **out);

/* 32-bit lanes per block of f (0 for NULL). */
uint32_t sbbf_lanes(const sbbf_t *f);

/* Copy h_words (num_blocks * 8 uint32 in the layout above) into a new
 * library-owned filter (synchronous).  Errors as sbbf_create. */
sbbf_status sbbf_create_from_host(const uint32_t *h_words, uint32_t num_blocks,
                                  sbbf_t **out);

/* Free a filter (synchronises the device first if it owns memory).
 * NULL is a no-op. */
sbbf_status sbbf_destroy(sbbf_t *f);

/* Number of blocks (0 for NULL). */
uint32_t sbbf_num_blocks(const sbbf_t *f);

/* Device address and size in bytes of the filter words (num_blocks * lanes *
 * 4 bytes). */
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

/* How sbbf_insert_hashes and sbbf_find_hashes process a batch.
 * Partitioned: the hashes are first grouped by filter slice (2^17 to 2^20
 * consecutive blocks, 4 to 32 MiB) into a scratch buffer, then processed
 * slice by slice with each slice prefetched into L2, which turns random DRAM
 * accesses into L2 hits for filters larger than L2; a lookup's answers are
 * then moved back to the hashes' order.  Results are identical either way
 * (inserts commute; a lookup's answer is set at its original position), for
 * any input: hashes that crowd one slice far beyond its share are redone by
 * the unpartitioned path.  The scratch -- about 8.6 bytes per hash for
 * inserts and 11 for lookups (processed in pieces of at most 2^34 and 2^31
 * hashes), plus per slice 4 bytes per SM and, for lookups, 4 bytes per SM
 * and per 2^16 hashes -- is allocated with cudaMalloc (synchronous) when a
 * batch needs more than the filter holds, kept by the filter and freed by
 * sbbf_destroy; partitioned calls on one filter must therefore be ordered on
 * one stream.
 * Region passes (no scratch): the filter's blocks are split into P equal
 * ranges of at most 64 MiB and the call runs P kernels over all the hashes,
 * each inserting or answering only the hashes whose block lies in its range
 * (a lookup's first pass writes every answer word, the later ones OR their
 * bits in with atomics, so the answers of one call must not be read before
 * its last pass ends -- the stream orders that).  Each pass finds its
 * blocks in L2, for filters somewhat larger than what L2 keeps under random
 * access.
 *   SBBF_PARTITION_AUTO (default): lookups of at least 8Mi hashes into
 *     filters of more than 84 MiB and at most 192 MiB take region passes
 *     (two or three); otherwise partition batches of at least 4Mi hashes
 *     (inserts) or 8Mi (lookups) when the filter holds at least 96 MiB
 *     (inserts) or more than 128 MiB (lookups) and the batch has at least
 *     0.25 hashes per block (inserts) or 0.6 (lookups) -- the measured
 *     break-evens; if the scratch cannot be allocated, run unpartitioned;
 *   SBBF_PARTITION_OFF: never partition, no region passes;
 *   SBBF_PARTITION_ON: always partition (SBBF_ENOMEM if no scratch);
 *   SBBF_PARTITION_REGIONS: inserts and lookups of hashes (sbbf_*_hashes
 *     and the staged host-buffer calls) by region passes whenever the filter
 *     spans more than one region.
 * Host-buffer calls that read the hashes in place from host memory (direct
 * mode) never take region passes: each pass would read them again.
 * Filters of 4 or 16 lanes never partition or take region passes.  Lookups
 * of 4- or 8-byte raw keys take region passes as hashes do (every pass
 * hashes its keys again); lookups of byte strings take none (where hashes
 * would, they run unpartitioned).
 * Errors: SBBF_EINVAL (NULL filter or unknown mode). */
enum {
  SBBF_PARTITION_AUTO = 0,
  SBBF_PARTITION_OFF = 1,
  SBBF_PARTITION_ON = 2,
  SBBF_PARTITION_REGIONS = 3
};
sbbf_status sbbf_set_partitioning(sbbf_t *f, int mode);

/* Whether a batch of n hashes takes the partitioned path under the filter's
 * current mode: for sbbf_insert_hashes / sbbf_insert_keys / sbbf_insert_bytes
 * (lookup = 0) or the matching lookups (lookup != 0).  The answer is the
 * decision before any scratch allocation (in automatic mode a failed
 * allocation still falls back to the unpartitioned path).  A partitioned
 * insert runs three kernels per piece of at most 2^34 hashes (scatter,
 * slice-ordered insert, crowded ranges), a partitioned lookup four per piece
 * of at most 2^31 hashes (scatter, slice-ordered lookup, answers back to key
 * order, crowded ranges); raw keys add one hashing kernel.  *applies is set to 1 or 0.
 * Errors: SBBF_EINVAL (NULL filter or applies). */
sbbf_status sbbf_partition_applies(const sbbf_t *f, size_t n, int lookup, int *applies);

/* Number of region passes (one kernel each) an insert (lookup = 0) or a
 * lookup (lookup != 0) of n hashes by sbbf_insert_hashes / sbbf_find_hashes
 * (and of n fixed-width keys by sbbf_find_keys) takes under the filter's
 * mode, in *passes (1: a single pass, unpartitioned or partitioned).
 * Errors: SBBF_EINVAL (NULL filter or passes). */
sbbf_status sbbf_region_passes(const sbbf_t *f, size_t n, int lookup, uint32_t *passes);

/* Outcome of the device-side waits of the partitioned calls on f since the
 * last query.  The partitioned passes stream each CTA's hashes through
 * shared memory with asynchronous bulk copies and wait for each copy on an
 * mbarrier with a time limit (2 s; a copy takes microseconds).  If a wait
 * runs out, the CTA records bit 1 in the filter's device status word and
 * reads its remaining hashes with plain loads -- the call's results stay
 * exact; before the CTA exits it waits, with the same limit, for every copy
 * still outstanding, and records bit 2 if one never completed (the results
 * of that call are then not guaranteed).  This call synchronises `stream`
 * (order it after the calls to check), reads the word and clears it.
 * Returns SBBF_OK when no wait ran out, SBBF_ETIMEOUT when one did.
 * Errors: SBBF_EINVAL (NULL filter), SBBF_ECUDA. */
sbbf_status sbbf_device_status(sbbf_t *f, sbbf_stream_t stream);

/* Sets `bits` in f's device status word on `stream`, as a timed-out device
 * wait does; for testing the reporting of sbbf_device_status without making
 * a device wait run out.  Errors: SBBF_EINVAL (NULL filter or one not on
 * the current device), SBBF_ENOMEM / SBBF_ECUDA (allocating the word). */
sbbf_status sbbf_record_device_status(sbbf_t *f, uint32_t bits, sbbf_stream_t stream);

/* Look up d_hashes[0..n) (appendix find_hash for each) into the packed
 * bitmask d_out_bits of (n + 31) / 32 words (caller-owned, 4-byte aligned).
 * Errors as sbbf_insert_hashes; d_out_bits NULL with n > 0 is SBBF_EINVAL. */
sbbf_status sbbf_find_hashes(const sbbf_t *f, const uint64_t *d_hashes,
                             size_t n, uint32_t *d_out_bits,
                             sbbf_stream_t stream);

/* dst |= src word by word: afterwards dst answers true for every hash either
 * filter held.  Not in the paper; meaningful only for equal num_blocks and
 * lanes (the seeds are fixed).  Errors: SBBF_EINVAL (NULL, num_blocks or
 * lanes differ). */
sbbf_status sbbf_union(sbbf_t *dst, const sbbf_t *src, sbbf_stream_t stream);

/* Copy the filter words to host memory h_words of at least
 * num_blocks * lanes * 4 bytes; synchronises the stream before returning.
 * Errors: SBBF_EINVAL (NULL or bytes too small), SBBF_ECUDA. */
sbbf_status sbbf_copy_to_host(const sbbf_t *f, uint32_t *h_words, size_t bytes,
                              sbbf_stream_t stream);

/* ------------------------------------------------------------------------
 * Serialization (not in the paper; the systems it lists as adopters store
 * filters).  Both formats are synchronous and go through host memory.
 *
 * Native checkpoint format: a 64-byte little-endian header, then the filter
 * words in the layout above.
 *   bytes  0..3   'S' 'B' 'B' 'F'
 *   bytes  4..7   u32 format version, 1
 *   bytes  8..11  u32 lanes (4, 8 or 16)
 *   bytes 12..15  u32 num_blocks
 *   bytes 16..23  u64 layout digest: XXH64 (seed 0) of the lanes' seeds as
 *                 little-endian uint32, lane 0 first (detects a filter built
 *                 with other seeds or another lane order)
 *   bytes 24..31  u64 payload bytes, num_blocks * lanes * 4
 *   bytes 32..39  u64 XXH64 (seed 0) of the payload
 *   bytes 40..63  zero
 * ---------------------------------------------------------------------- */

/* Bytes sbbf_serialize writes for f (0 for NULL). */
size_t sbbf_serialized_size(const sbbf_t *f);

/* Write f into h_buf (host memory, at least sbbf_serialized_size(f) bytes)
 * after the work already on `stream`.  Errors: SBBF_EINVAL (NULL, buffer too
 * small), SBBF_ECUDA. */
sbbf_status sbbf_serialize(const sbbf_t *f, void *h_buf, size_t bytes,
                           sbbf_stream_t stream);

/* Create a library-owned filter on the current device from a native buffer.
 * Errors: SBBF_EINVAL (bad magic, version, lanes, digest, sizes, nonzero
 * reserved bytes, truncated buffer or checksum mismatch), SBBF_ENOMEM,
 * SBBF_ECUDA. */
sbbf_status sbbf_deserialize(const void *h_buf, size_t bytes, sbbf_t **out);

/* Parquet's Bloom-filter format: a Thrift compact-protocol BloomFilterHeader
 * {1: i32 numBytes; 2: algorithm = BLOCK; 3: hash = XXHASH; 4: compression =
 * UNCOMPRESSED} followed by numBytes of bitset.  Parquet's blocks are eight
 * little-endian uint32 words, but it lists the eight seeds in the order the
 * paper's text prints the appendix constants, which exchanges words 2j and
 * 2j+1 of every block relative to this library's lane order (the appendix's
 * little-endian order); export and import make that exchange.  Parquet hashes
 * values with XXH64 seed 0 (sbbf_insert_keys / sbbf_insert_bytes with seed
 * 0 insert the same hashes).  numBytes must be a positive multiple of 32 below
 * 2^31 (Parquet writers use powers of two up to 128 MiB; readers may require
 * a power of two). */

/* The header for a bitset of num_bytes bytes: its length in *header_len and,
 * if h_out is not NULL, its bytes in h_out (cap bytes).  Host only.
 * Errors: SBBF_EINVAL (num_bytes not a positive multiple of 32 below 2^31,
 * cap too small). */
sbbf_status sbbf_parquet_header(uint64_t num_bytes, uint8_t *h_out, size_t cap,
                                size_t *header_len);

/* Parse a header at h_buf (bytes available): the bitset size and the header
 * length.  Unknown fields are skipped.  Host only.  Errors: SBBF_EINVAL
 * (malformed or truncated header, an algorithm, hash or compression other
 * than BLOCK / XXHASH / UNCOMPRESSED, numBytes not a positive multiple of
 * 32). */
sbbf_status sbbf_parquet_parse_header(const uint8_t *h_buf, size_t bytes,
                                      uint64_t *num_bytes, size_t *header_len);

/* Bytes sbbf_export_parquet writes for f (0 for NULL, lanes != 8 or a filter
 * of 2 GiB or more). */
size_t sbbf_parquet_size(const sbbf_t *f);

/* Write header and bitset of f to h_buf; *written (may be NULL) receives the
 * byte count.  Errors: SBBF_EINVAL (NULL, lanes != 8, buffer too small,
 * filter too large), SBBF_ECUDA. */
sbbf_status sbbf_export_parquet(const sbbf_t *f, uint8_t *h_buf, size_t bytes,
                                size_t *written, sbbf_stream_t stream);

/* Create a library-owned 8-lane filter of numBytes / 32 blocks from a
 * Parquet Bloom filter at h_buf; *consumed (may be NULL) receives header +
 * bitset bytes.  Errors: as sbbf_parquet_parse_header, SBBF_EINVAL if the
 * bitset is truncated, SBBF_ENOMEM, SBBF_ECUDA. */
sbbf_status sbbf_import_parquet(const uint8_t *h_buf, size_t bytes,
                                sbbf_t **out, size_t *consumed);

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

/* How a pipe moves the data of a call.
 *   SBBF_PIPE_AUTO (default): direct when every host buffer of the call is
 *     page-locked memory mapped into the device's address space (e.g.
 *     cudaHostAlloc / cudaHostRegister memory, torch pin_memory), else staged;
 *   SBBF_PIPE_COPY: always staged: chunked cudaMemcpyAsync to the pipe's
 *     device buffers, overlapped with the kernels on two streams;
 *   SBBF_PIPE_DIRECT: the kernels read the hashes from, and write the result
 *     bits to, the host buffers in place through the device mapping (on a
 *     Grace-Blackwell node over NVLink-C2C); calls whose buffers are not
 *     mapped return SBBF_EINVAL.
 * Results are identical in every mode.  Errors: SBBF_EINVAL (NULL, unknown
 * mode). */
enum { SBBF_PIPE_AUTO = 0, SBBF_PIPE_COPY = 1, SBBF_PIPE_DIRECT = 2 };
sbbf_status sbbf_host_pipe_set_mode(sbbf_host_pipe_t *p, int mode);

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
 * Keys hashed on the device (the step before the method: the paper hashes a
 * key once to 64 bits before block selection, intro, and fixes no hash
 * function).  The hash is XXH64 of the key's bytes with the caller's seed
 * (Y. Collet's published xxHash specification).  Parquet's split block
 * filters hash with XXH64, seed 0, so with seed 0 these calls insert the
 * hashes a Parquet writer inserts.
 *
 * Fixed-width keys: d_keys holds n keys of key_bytes = 4 or 8 bytes each
 * (a uint32 or uint64 array, aligned to key_bytes); key k is hashed as its
 * key_bytes little-endian bytes.  Variable-length keys (byte strings): key k
 * is d_data[d_offsets[k] .. d_offsets[k+1]), d_offsets n + 1 non-decreasing
 * uint64 (8-byte aligned; not checked against the size of d_data), d_data
 * any alignment.
 * Errors: SBBF_EINVAL (key_bytes not 4 or 8, NULL with n > 0, misaligned),
 * SBBF_ECUDA.
 * ---------------------------------------------------------------------- */

/* d_hashes[k] = XXH64(key k, seed) for k in [0, n) (d_hashes 8-byte
 * aligned). */
sbbf_status sbbf_hash_keys(const void *d_keys, uint32_t key_bytes, size_t n,
                           uint64_t seed, uint64_t *d_hashes,
                           sbbf_stream_t stream);
sbbf_status sbbf_hash_bytes(const uint8_t *d_data, const uint64_t *d_offsets,
                            size_t n, uint64_t seed, uint64_t *d_hashes,
                            sbbf_stream_t stream);

/* Insert / look up keys with the hash computed inside the insert and lookup
 * kernels (no hash array in memory).  The filter and the result bits equal
 * those of sbbf_hash_keys (or sbbf_hash_bytes) followed by
 * sbbf_insert_hashes / sbbf_find_hashes.  A batch that takes the partitioned
 * path (sbbf_set_partitioning) is hashed into the filter's scratch first,
 * which then grows by 8 bytes per key. */
sbbf_status sbbf_insert_keys(sbbf_t *f, const void *d_keys, uint32_t key_bytes,
                             size_t n, uint64_t seed, sbbf_stream_t stream);
sbbf_status sbbf_find_keys(const sbbf_t *f, const void *d_keys,
                           uint32_t key_bytes, size_t n, uint64_t seed,
                           uint32_t *d_out_bits, sbbf_stream_t stream);
sbbf_status sbbf_insert_bytes(sbbf_t *f, const uint8_t *d_data,
                              const uint64_t *d_offsets, size_t n,
                              uint64_t seed, sbbf_stream_t stream);
sbbf_status sbbf_find_bytes(const sbbf_t *f, const uint8_t *d_data,
                            const uint64_t *d_offsets, size_t n, uint64_t seed,
                            uint32_t *d_out_bits, sbbf_stream_t stream);

/* ------------------------------------------------------------------------
 * Serving: resident filters, requests arriving over time, continuous batching
 * under a device-memory budget (not in the paper).
 *
 * A scheduler thread owned by the server forms launch windows from the
 * requests that have arrived (filters in the order of their oldest queued
 * request, each filter's requests in arrival order, bounded by requests and
 * hashes per window), admits a filter's requests only when the filter is
 * resident within the budget (evicting the least recently used filter with
 * no queued requests, else the least recently used, to pinned host memory),
 * and runs all requests of a window in one launch while the next window is
 * being formed.  Results equal serial replay in
 * arrival order: a lookup sees exactly the inserts on its filter that arrived
 * before it (per filter, runs of inserts and runs of lookups execute as
 * ordered phases).
 * ---------------------------------------------------------------------- */

typedef struct sbbf_server sbbf_server_t;

typedef struct sbbf_server_config {
  uint64_t budget_bytes;         /* device bytes for resident filters plus the
                                    device-resident buffers of admitted requests */
  uint32_t max_window_requests;  /* requests per launch window (slots) */
  uint32_t max_inflight_windows; /* windows enqueued on the GPU at once */
  uint64_t max_window_keys;      /* hashes per window (a larger single request
                                    still forms a window of its own) */
  uint64_t max_pending_requests; /* submitted, not yet admitted; beyond it
                                    submit returns SBBF_EBUSY */
} sbbf_server_config_t;

typedef struct sbbf_request {
  uint32_t op;                   /* SBBF_OP_INSERT or SBBF_OP_FIND */
  uint32_t filter;               /* id from sbbf_server_add_filter */
  uint64_t n;                    /* hashes */
  const uint64_t *d_hashes;      /* device or pinned host memory, 8-byte
                                    aligned, owned by the caller, unchanged
                                    until the request completes */
  uint32_t *d_out_bits;          /* lookups: (n + 31) / 32 words (device or
                                    pinned host), written by completion */
} sbbf_request_t;

typedef struct sbbf_server_stats {
  uint64_t windows, launches, phases, requests, keys;
  uint64_t admissions, evictions, writebacks, admission_waits;
  uint64_t resident_bytes;
} sbbf_server_stats_t;

/* Start a server (its stream and scheduler thread) on the current device.
 * Errors: SBBF_EINVAL (zero limits), SBBF_ENOMEM, SBBF_ECUDA. */
sbbf_status sbbf_server_create(const sbbf_server_config_t *cfg,
                               sbbf_server_t **out);
/* Finish all submitted requests, stop the thread and free everything. */
sbbf_status sbbf_server_destroy(sbbf_server_t *s);

/* Register an empty filter of num_blocks blocks (not yet resident). */
sbbf_status sbbf_server_add_filter(sbbf_server_t *s, uint32_t num_blocks,
                                   uint32_t *id);

/* Enqueue a request (thread-safe, non-blocking).  *ticket identifies it.
 * Errors: SBBF_EINVAL, SBBF_EBUSY (queue full, or the filter plus the
 * request's device buffers exceed the whole budget), or the server's sticky
 * device error. */
sbbf_status sbbf_server_submit(sbbf_server_t *s, const sbbf_request_t *r,
                               uint64_t *ticket);
/* *done = 1 once the request's results are in place. */
sbbf_status sbbf_server_poll(sbbf_server_t *s, uint64_t ticket, int *done);
/* Block until the request completes or timeout_ns passes (0: no limit).
 * Errors: SBBF_ETIMEOUT, SBBF_EINVAL, a device error. */
sbbf_status sbbf_server_wait(sbbf_server_t *s, uint64_t ticket,
                             uint64_t timeout_ns);
/* Block until no request is pending or running (timeout_ns 0: no limit). */
sbbf_status sbbf_server_drain(sbbf_server_t *s, uint64_t timeout_ns);

/* Insert d_hashes[0..n) into filter id outside any window (set-up before
 * serving; drains first; synchronous). */
sbbf_status sbbf_server_prefill(sbbf_server_t *s, uint32_t id,
                                const uint64_t *d_hashes, size_t n);
/* Copy filter id's words to host memory (drains first; synchronous). */
sbbf_status sbbf_server_copy_filter(sbbf_server_t *s, uint32_t id,
                                    uint32_t *h_words, size_t bytes);
sbbf_status sbbf_server_stats(sbbf_server_t *s, sbbf_server_stats_t *out);

/* Client-side replay: submit reqs[i] at arrival_ns[i] nanoseconds after the
 * call starts (waiting for the clock; on a full queue, retrying), then wait
 * for all; latency_ns[i] = completion - arrival.  Synchronous. */
sbbf_status sbbf_server_replay(sbbf_server_t *s, const sbbf_request_t *reqs,
                               const uint64_t *arrival_ns, size_t n,
                               uint64_t *latency_ns);
/* The same arrivals served one plain launch per request, in arrival order,
 * on the server's filters and stream (the scheduler is paused meanwhile):
 * the serial baseline for the batched server. */
sbbf_status sbbf_server_replay_serial(sbbf_server_t *s,
                                      const sbbf_request_t *reqs,
                                      const uint64_t *arrival_ns, size_t n,
                                      uint64_t *latency_ns);

/* ------------------------------------------------------------------------
 * Allocation-free lookup (the paper has no counterpart: it is an interface
 * for callers that must not allocate device memory on this path -- a serving
 * loop bound to a fixed device-memory budget, a framework whose caching
 * allocator owns the device memory, or a latency-critical caller that cannot
 * afford the device synchronisation of cudaFree).
 * ---------------------------------------------------------------------- */

/* Largest n_filters sbbf_multi_find_noalloc accepts. */
#define SBBF_NOALLOC_MAX_FILTERS 65536u

/* Tagged-form lookup (as sbbf_multi_find) over caller-owned memory, with no
 * cudaMalloc, cudaFree or other allocating call.
 *   d_arena        the filters' words, filter t at block offset
 *                  d_num_blocks[0] + ... + d_num_blocks[t-1] (the layout of
 *                  sbbf_multi_create), 32-byte aligned, at least
 *                  sum(d_num_blocks) * 32 bytes (not checked);
 *   d_num_blocks   n_filters uint32 sizes in device memory; a filter of 0
 *                  blocks answers 0 and counts its keys as invalid;
 *   d_hashes, d_ids, n, d_out_bits   as sbbf_multi_find;
 *   d_invalid_count  device uint64 receiving the number of keys whose id is
 *                  >= n_filters or names an empty filter (NULL: not reported).
 * Its scratch (directory and counter) is one static device array of
 * 256 + 16 * SBBF_NOALLOC_MAX_FILTERS bytes held by every GPU that loads the
 * library until the process exits; each call overwrites it, so calls that
 * overlap on the GPU race: issue them in order on one stream.  The first call
 * on a device looks up that array's device address (with the device
 * current); make that first call before any stream capture.  Asynchronous.
 * Errors: SBBF_ERANGE (n_filters > SBBF_NOALLOC_MAX_FILTERS), SBBF_EINVAL
 * (n_filters == 0, NULL or misaligned pointers), SBBF_ECUDA. */
sbbf_status sbbf_multi_find_noalloc(const uint32_t *d_arena,
                                    const uint32_t *d_num_blocks,
                                    uint32_t n_filters, const uint64_t *d_hashes,
                                    const uint32_t *d_ids, size_t n,
                                    uint32_t *d_out_bits,
                                    unsigned long long *d_invalid_count,
                                    sbbf_stream_t stream);

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

/* Query streams for several filters in the segment layout: query k (global
 * index, k in [0, n)) belongs to the filter t with d_q_offsets[t] <= k <
 * d_q_offsets[t+1]; with r = output k of member_seed it is a member when
 * (r >> 32) < member_threshold and filter t has inserted keys, namely output
 * (d_ins_offsets[t] + (((r & 0xffffffff) * n_t) >> 32)) of ins_seed with
 * n_t = d_ins_offsets[t+1] - d_ins_offsets[t]; otherwise output k of
 * fresh_seed.  Offsets as for the segment form (n_filters + 1 entries each).
 */
sbbf_status sbbf_fill_segment_queries(uint64_t *d_out, size_t n,
                                      const uint64_t *d_q_offsets,
                                      const uint64_t *d_ins_offsets,
                                      uint32_t n_filters, uint64_t ins_seed,
                                      uint64_t fresh_seed, uint64_t member_seed,
                                      uint64_t member_threshold,
                                      sbbf_stream_t stream);

/* d_ids[k] = the filter t with d_offsets[t] <= k < d_offsets[t+1], k < n. */
sbbf_status sbbf_fill_segment_ids(uint32_t *d_ids, size_t n,
                                  const uint64_t *d_offsets, uint32_t n_filters,
                                  sbbf_stream_t stream);

/* Number of set bits in the packed bitmask d_bits over its first n bits,
 * written to *d_count (uint64, device) -- used to count lookup hits. */
sbbf_status sbbf_count_bits(const uint32_t *d_bits, size_t n,
                            unsigned long long *d_count, sbbf_stream_t stream);

/* ------------------------------------------------------------------------
 * Verification digest (a checking aid; not part of the method).
 *
 * Compares filters, or a filter and a host copy, range by range without
 * moving the words.  d_words holds num_blocks blocks of `lanes` 32-bit words
 * (the layout above; 16-byte aligned, device memory), read as 64-bit units:
 * unit u is word 2u in its low half and word 2u+1 in its high half.  Range r
 * holds the blocks [r * range_blocks, min(num_blocks, (r + 1) *
 * range_blocks)), r < n_ranges = ceil(num_blocks / range_blocks), and gets
 *   d_digest[r]  = sum mod 2^64 over its units u of splitmix64 output u of the
 *                  stream seeded with the unit's value (the generator above),
 *   d_bits[r]    = number of set bits,
 *   d_partial[r] = number of its blocks with both an all-zero lane and a
 *                  non-zero lane.
 * An insert sets one bit in every lane of its block (the paper's make_mask)
 * and a union ORs whole blocks, so d_partial is 0 in every range of a filter
 * built by them.  The three arrays (device, n_ranges entries each, owned by
 * the caller) are zeroed on the stream and then filled by one kernel reading
 * every word once; the result does not depend on the launch's schedule.
 * Errors: SBBF_EINVAL for lanes not 4, 8 or 16, range_blocks == 0, a NULL
 * output, num_blocks > 2^40, or (num_blocks > 0) a NULL or unaligned
 * d_words.  num_blocks == 0 enqueues nothing. */
sbbf_status sbbf_range_digest(const uint32_t *d_words, uint64_t num_blocks,
                              uint32_t lanes, uint64_t range_blocks,
                              unsigned long long *d_digest,
                              unsigned long long *d_bits,
                              unsigned long long *d_partial,
                              sbbf_stream_t stream);

/* ------------------------------------------------------------------------
 * Many filters in one arena (batched form; not in the paper).
 *
 * Filter t of a set is the plain filter of num_blocks[t] blocks whose block 0
 * is arena block base[t] = num_blocks[0] + ... + num_blocks[t-1]; each filter
 * keeps the paper's block selection (with its own num_blocks) and mask, so a
 * filter's words equal those of a single filter given the same hashes.
 *
 * Keys name their filter in one of two forms:
 *   tagged:   d_ids[k] is key k's filter (uint32); a key whose id is
 *             >= n_filters is skipped by inserts, answers 0 in lookups and is
 *             counted (see sbbf_multi_invalid_count); it never faults;
 *   segments: keys are grouped by filter: filter t's keys are
 *             d_hashes[d_offsets[t] .. d_offsets[t+1]) with d_offsets a device
 *             array of n_filters + 1 non-decreasing uint64, d_offsets[0] = 0
 *             and d_offsets[n_filters] = n.  Offsets that break this contract
 *             assign keys to unspecified filters of the set but never access
 *             memory outside the arena.
 * Lookup answers are packed by key index k over the whole batch, exactly as
 * for a single filter.  Each batch is one persistent launch whatever the
 * number of filters.
 * ---------------------------------------------------------------------- */

typedef struct sbbf_multi_set sbbf_multi_t;

enum { SBBF_OP_INSERT = 0, SBBF_OP_FIND = 1 };
enum { SBBF_FORM_SEGMENTS = 0, SBBF_FORM_TAGGED = 1 };

/* Create n_filters empty filters with h_num_blocks[t] >= 1 blocks each
 * (host array) in one library-owned, zero-filled device arena (synchronous).
 * Errors: SBBF_EINVAL (NULL, n_filters == 0, a zero size), SBBF_ENOMEM,
 * SBBF_ECUDA. */
sbbf_status sbbf_multi_create(const uint32_t *h_num_blocks, uint32_t n_filters,
                              sbbf_multi_t **out);
sbbf_status sbbf_multi_destroy(sbbf_multi_t *m);
uint32_t sbbf_multi_num_filters(const sbbf_multi_t *m);

/* First arena block and size of filter id.  Errors: SBBF_EINVAL. */
sbbf_status sbbf_multi_filter_info(const sbbf_multi_t *m, uint32_t id,
                                   uint64_t *base_block, uint32_t *num_blocks);

/* Device address and byte size of the whole arena. */
sbbf_status sbbf_multi_device_words(const sbbf_multi_t *m, uint32_t **d_words,
                                    size_t *bytes);

sbbf_status sbbf_multi_clear(sbbf_multi_t *m, sbbf_stream_t stream);

/* Copy the whole arena (total blocks * 32 bytes) to host memory h_words of
 * at least that many bytes; synchronises the stream.  Errors: SBBF_EINVAL,
 * SBBF_ECUDA. */
sbbf_status sbbf_multi_copy_to_host(const sbbf_multi_t *m, uint32_t *h_words,
                                    size_t bytes, sbbf_stream_t stream);

/* Tagged form.  d_hashes 8-byte aligned, d_ids 4-byte aligned, n keys. */
sbbf_status sbbf_multi_insert(sbbf_multi_t *m, const uint64_t *d_hashes,
                              const uint32_t *d_ids, size_t n,
                              sbbf_stream_t stream);
sbbf_status sbbf_multi_find(const sbbf_multi_t *m, const uint64_t *d_hashes,
                            const uint32_t *d_ids, size_t n,
                            uint32_t *d_out_bits, sbbf_stream_t stream);

/* Segment form (d_offsets 8-byte aligned, n = d_offsets[n_filters]). */
sbbf_status sbbf_multi_insert_segments(sbbf_multi_t *m, const uint64_t *d_hashes,
                                       const uint64_t *d_offsets, size_t n,
                                       sbbf_stream_t stream);
sbbf_status sbbf_multi_find_segments(const sbbf_multi_t *m,
                                     const uint64_t *d_hashes,
                                     const uint64_t *d_offsets, size_t n,
                                     uint32_t *d_out_bits, sbbf_stream_t stream);

/* Per-filter form: one plain single-filter launch per non-empty filter, with
 * HOST offsets h_offsets[0..n_filters] (same contract as d_offsets).  The
 * same results as the segment form; for lookups every h_offsets[t] must be a
 * multiple of 32 so that each filter's answers start a fresh output word
 * (SBBF_EINVAL otherwise).  This is the launch-per-filter baseline that the
 * batched form is measured against. */
sbbf_status sbbf_multi_insert_each(sbbf_multi_t *m, const uint64_t *d_hashes,
                                   const uint64_t *h_offsets,
                                   sbbf_stream_t stream);
sbbf_status sbbf_multi_find_each(const sbbf_multi_t *m, const uint64_t *d_hashes,
                                 const uint64_t *h_offsets, uint32_t *d_out_bits,
                                 sbbf_stream_t stream);

/* Number of tagged keys with an invalid id seen since the last call; resets
 * the count.  Synchronises the stream.  Errors: SBBF_EINVAL, SBBF_ECUDA. */
sbbf_status sbbf_multi_invalid_count(sbbf_multi_t *m, uint64_t *count,
                                     sbbf_stream_t stream);

/* Launch shape used for (op, form): CTA size (128/256/512), lanes per key
 * (1 or 8), loads in flight per warp (1/2/4) and, for lookups, whether block
 * loads bypass L1 allocation (0/1; ignored for inserts).  Shapes never
 * change results, only speed. */
sbbf_status sbbf_multi_get_tuning(const sbbf_multi_t *m, int op, int form,
                                  int *threads, int *lanes, int *unroll,
                                  int *l1_bypass);
sbbf_status sbbf_multi_set_tuning(sbbf_multi_t *m, int op, int form,
                                  int threads, int lanes, int unroll,
                                  int l1_bypass);

/* Autotune (op, form) on a prefix (at most 2^24 keys) of a real batch:
 * every candidate shape runs on the sample, its result (lookup bits, or the
 * arena words it inserts into a scratch copy of the touched filters) is
 * compared with the default shape's result and discarded on any difference;
 * the fastest verified shape is kept for the set and cached per (GPU, op,
 * form, size class).  The set's filters are not modified.  d_offsets_or_ids
 * is the batch's d_offsets (segments) or d_ids (tagged).  *best_ms (may be
 * NULL) receives the winner's sample time, or -1 when the cache answered.
 * Synchronous.  Errors: SBBF_EINVAL, SBBF_ENOMEM (scratch), SBBF_ECUDA. */
sbbf_status sbbf_multi_tune(sbbf_multi_t *m, int op, int form,
                            const uint64_t *d_hashes,
                            const void *d_offsets_or_ids, size_t n,
                            sbbf_stream_t stream, float *best_ms);

/* A CUDA graph holding one batched segment-form insert followed by one
 * batched segment-form lookup on the set, with the set's current tuned
 * shapes (tune before creating it).  Each launch updates the two kernels'
 * arguments in the instantiated graph and launches it on stream: inserts of
 * the batch land before its lookups run.  Either part may be empty
 * (n_ins == 0 or n_q == 0). */
typedef struct sbbf_multi_graph sbbf_multi_graph_t;
sbbf_status sbbf_multi_graph_create(sbbf_multi_t *m, sbbf_multi_graph_t **out);
sbbf_status sbbf_multi_graph_destroy(sbbf_multi_graph_t *g);
sbbf_status sbbf_multi_graph_launch(sbbf_multi_graph_t *g,
                                    const uint64_t *d_ins,
                                    const uint64_t *d_ins_offsets, size_t n_ins,
                                    const uint64_t *d_q,
                                    const uint64_t *d_q_offsets, size_t n_q,
                                    uint32_t *d_out_bits, sbbf_stream_t stream);

/* ------------------------------------------------------------------------
 * One filter sharded by block range over several devices.
 *
 * The appendix's block_index sends every hash to exactly one block, so a
 * filter of B blocks split into contiguous block ranges is the same filter:
 * shard s of G owns global blocks [s P, min(B, (s + 1) P)), P = ceil(B / G),
 * held as a filter of its own (sbbf_create with hi - lo blocks), and a hash
 * belongs to the shard that owns its block.  A batch on one device is
 * routed (sbbf_shard_route), exchanged with the other devices by the
 * caller's collective library (an all-to-all of the routed hashes, with the
 * per-shard counts), inserted or looked up on the local range
 * (sbbf_shard_insert / sbbf_shard_find), and for lookups the answer words go
 * back by the reverse all-to-all and are put in query order
 * (sbbf_shard_unpermute).  The results equal those of the unsharded filter
 * bit for bit.
 * ---------------------------------------------------------------------- */

/* The global block range [*lo, *hi) of shard `shard` of n_shards (empty when
 * the filter has fewer blocks than shards need).  Pure arithmetic; no device
 * is needed.  Errors: SBBF_EINVAL (num_blocks or n_shards 0, n_shards above
 * 1024, shard >= n_shards, NULL out pointers). */
sbbf_status sbbf_shard_range(uint32_t num_blocks, uint32_t n_shards, uint32_t shard,
                             uint32_t *lo, uint32_t *hi);

/* Entries sbbf_shard_route may write to d_routed / d_perm: n, plus 31 per
 * shard when padding. */
size_t sbbf_shard_routed_capacity(size_t n, uint32_t n_shards, int pad);

/* Device scratch bytes sbbf_shard_route needs (per SM and shard). */
size_t sbbf_shard_route_scratch_bytes(size_t n, uint32_t n_shards);

/* Groups d_hashes[0..n) (device, 8-byte aligned, n < 2^32) by owner shard
 * of a num_blocks-block filter split n_shards ways: owner 0's hashes first,
 * then owner 1's, ...; d_routed[i] is a hash and d_perm[i] its index in
 * d_hashes.  d_counts[s] (device, n_shards uint64) receives the number of
 * entries of owner s's group.  With pad != 0 every group is padded to a
 * multiple of 32 entries with a hash of the owner's first block and
 * d_perm = 0xFFFFFFFF, so that a group's lookup answers are whole 32-bit
 * words; padding is for lookups only (an insert of a padding hash would set
 * bits).  The order within a group is not specified.  d_routed and d_perm
 * hold sbbf_shard_routed_capacity(n, n_shards, pad) entries; d_scratch
 * (device, 8-byte aligned) holds sbbf_shard_route_scratch_bytes bytes.
 * Asynchronous on stream.  Errors: SBBF_EINVAL (sizes, NULL, alignment,
 * n_shards above 1024), SBBF_ECUDA. */
sbbf_status sbbf_shard_route(const uint64_t *d_hashes, size_t n, uint32_t num_blocks,
                             uint32_t n_shards, int pad, uint64_t *d_routed, uint32_t *d_perm,
                             uint64_t *d_counts, void *d_scratch, size_t scratch_bytes,
                             sbbf_stream_t stream);

/* Insert d_hashes[0..n) into f, the shard holding global blocks
 * [lo, lo + sbbf_num_blocks(f)) of a num_blocks-block filter (appendix
 * add_hash at block block_index(h, num_blocks) - lo); hashes whose block
 * lies outside the range are skipped.  f has 8 lanes.  Errors: SBBF_EINVAL
 * (NULL, other lane count, a range past num_blocks, misaligned), SBBF_ECUDA. */
sbbf_status sbbf_shard_insert(sbbf_t *f, uint32_t num_blocks, uint32_t lo,
                              const uint64_t *d_hashes, size_t n, sbbf_stream_t stream);

/* Look up d_hashes[0..n) in shard f (as sbbf_shard_insert) into the packed
 * bitmask d_out_bits ((n + 31) / 32 words); hashes outside the range answer
 * 0.  Errors as sbbf_shard_insert; d_out_bits NULL or not 4-byte aligned is
 * SBBF_EINVAL. */
sbbf_status sbbf_shard_find(const sbbf_t *f, uint32_t num_blocks, uint32_t lo,
                            const uint64_t *d_hashes, size_t n, uint32_t *d_out_bits,
                            sbbf_stream_t stream);

/* Answers back to query order: zeroes d_out_bits ((n + 31) / 32 words) and
 * sets bit d_perm[i] for every set bit i of d_routed_bits (answers of the
 * n_routed routed entries) whose d_perm is not padding.  Errors:
 * SBBF_EINVAL (NULL with a nonzero size, misaligned), SBBF_ECUDA. */
sbbf_status sbbf_shard_unpermute(const uint32_t *d_routed_bits, const uint32_t *d_perm,
                                 size_t n_routed, size_t n, uint32_t *d_out_bits,
                                 sbbf_stream_t stream);

#ifdef __cplusplus
}
#endif
#endif /* SBBF_H */
