// Block-range partitioned inserts and lookups for filters larger than L2.
//
// A random 32-byte block of a filter far larger than L2 costs a DRAM access
// of at least 64 bytes, and DRAM serves only ~40 G random accesses per
// second, whereas the same block in L2 costs one L1/L2 request.  So for a
// large batch the keys are first grouped by filter slice -- 2^shift
// consecutive blocks, 4 to 32 MiB (see slice_shift) -- and then processed
// slice by slice, in order:
//   1. count: the keys are split into one contiguous range per CTA; each CTA
//      histograms its range by slice in shared memory and stores its row;
//   2. scan (one CTA): slice totals, slice start offsets, and for every
//      (CTA, slice) the output position where that CTA's keys of the slice
//      begin -- so the scatter needs no global atomics and its output order
//      is the same on every run;
//   3. scatter: each CTA streams its range in tiles through shared memory
//      (double-buffered bulk copies, cp.async.bulk with an mbarrier, the next
//      tile arriving while the current one is processed), counting-sorts the
//      tile by slice there and writes each slice's run at its own cursor, so
//      consecutive threads write consecutive addresses;
//   4. insert or look up the slice-ordered keys with the in-order dynamic
//      tile schedule; every claimed tile bulk-prefetches into L2 the filter
//      bytes of the keys a slice ahead, so the filter is read from DRAM
//      sequentially and hit in L2 when the keys arrive;
//   5. lookups only: the answers, written in slice order, go back to key
//      order one sub-range of positions at a time, each in shared memory.
// Inserts commute (OR), so the order within a slice does not matter and the
// filter equals the unpartitioned insert bit for bit; lookups keep each key's
// original position (written by the scatter) and answer exactly as the
// unpartitioned lookup.
#include <cuda_runtime.h>

#include <cstdint>

#include "sbbf.h"
#include "sbbf_device.cuh"
#include "sbbf_host.cuh"
#include "sbbf_kernels.cuh"

namespace sbbf {
sbbf_status launch_clear(uint32_t* dst, uint64_t n_words, cudaStream_t s);

namespace {

constexpr int kMinSliceShift = 17;       // 2^17 blocks (4 MiB) per slice
constexpr int kMaxSliceShift = 20;       // 2^20 blocks (32 MiB) per slice
constexpr uint32_t kTargetSlices = 512;
constexpr uint32_t kMaxSlices = 4096;    // num_blocks < 2^32 at the largest slice
constexpr uint32_t kFewSlices = 32;      // ballot counting up to this many slices
constexpr int kPartThreads = 1024;

__device__ __forceinline__ uint32_t slice_of(uint64_t h, uint32_t nb, int shift) {
  return block_of(h, nb) >> shift;
}

__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

constexpr int kCountThreads = 1024;

// Adds 1 to bins[p] for every valid lane's p.  With few bins (kFew) a warp
// counts each bin with one ballot; with many, lanes rarely collide and add
// directly.
template <bool kFew>
__device__ __forceinline__ void count_warp(unsigned* bins, uint32_t n_slices, bool v, uint32_t p) {
  if (kFew) {
    for (uint32_t b = 0; b < n_slices; ++b) {
      const unsigned m = __ballot_sync(0xFFFFFFFFu, v && p == b);
      if (m && lane_id() == static_cast<unsigned>(__ffs(m) - 1)) atomicAdd(&bins[b], __popc(m));
    }
  } else if (v) {
    atomicAdd(&bins[p], 1u);
  }
}

// Rank of this lane's key among the keys of the same bin (claims ranks from
// the shared counter ranks[p]).
template <bool kFew>
__device__ __forceinline__ unsigned rank_warp(unsigned* ranks, uint32_t n_slices, bool v,
                                              uint32_t p) {
  if (kFew) {
    unsigned mine = 0;
    for (uint32_t b = 0; b < n_slices; ++b) {
      const unsigned m = __ballot_sync(0xFFFFFFFFu, v && p == b);
      if (!m) continue;
      const int leader = __ffs(m) - 1;
      unsigned first = 0;
      if (lane_id() == static_cast<unsigned>(leader)) first = atomicAdd(&ranks[b], __popc(m));
      first = __shfl_sync(0xFFFFFFFFu, first, leader);
      if (v && p == b) mine = first + __popc(m & lanemask_lt());
    }
    return mine;
  }
  return v ? atomicAdd(&ranks[p], 1u) : 0u;
}

// Keys [c * R, min(n, (c + 1) * R)) belong to CTA c of the count and scatter
// passes.  R is a multiple of 32: a range starts 16-byte aligned whenever the
// array does, and a lookup's result words split between ranges without
// sharing a word.
__host__ __device__ __forceinline__ uint64_t range_keys(uint64_t n, uint32_t ctas) {
  const uint64_t r = (n + ctas - 1) / ctas;
  return (r + 31) & ~31ull;
}

// Lookups map answers back to key order by sub-range: kSubKeys consecutive
// positions of a CTA's range (a multiple of every scatter tile).  The scatter
// records its slice cursors at each sub-range start, so the keys of sub-range
// u of CTA c that fall in slice q sit at sorted positions
// [marks[c][u][q], marks[c][u + 1][q]); a key's original position is then
// stored as its 16-bit offset within its sub-range.
constexpr uint32_t kSubKeys = 1u << 16;

__host__ __device__ __forceinline__ uint32_t sub_ranges(uint64_t range) {
  return static_cast<uint32_t>((range + kSubKeys - 1) / kSubKeys);
}

// ---- bulk copies into shared memory ------------------------------------------

constexpr uint64_t kWaitNs = 2000ull * 1000 * 1000;  // a tile copy is microseconds

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Polls the mbarrier phase with the given parity; false after kWaitNs.
__device__ __forceinline__ bool wait_phase(uint32_t bar, uint32_t parity) {
  const uint64_t t0 = global_ns();
  for (;;) {
    uint32_t done;
    asm volatile(
        "{ .reg .pred p; mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2; "
        "selp.u32 %0, 1, 0, p; }"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
    if (global_ns() - t0 > kWaitNs) return false;
  }
}

// One thread: copy `bytes` (a multiple of 16, 16-byte aligned ends) from
// global src to shared dst, completing on mbarrier bar (armed here; a
// zero-byte copy just arrives).
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  if (bytes == 0) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
    return;
  }
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
  asm volatile(
      "cp.async.bulk.shared::cta.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}

// hist[c * n_slices + p] = keys of CTA c's range that fall in slice p.  The
// range streams through shared memory in tiles of kCountTile keys,
// double-buffered bulk copies like the scatter's (plain loads when the key
// array is not 16-byte aligned or a copy did not complete in time), so the
// histogram atomics of one tile overlap the copy of the next.
constexpr uint32_t kCountTile = 8192;

template <bool kFew>
__global__ void __launch_bounds__(kCountThreads, 1)
    count_kernel(const uint64_t* __restrict__ hashes, uint64_t n, uint32_t nb, int shift,
                 uint32_t n_slices, uint64_t range, unsigned* __restrict__ hist) {
  extern __shared__ __align__(16) unsigned long long smem[];
  uint64_t* s_buf0 = reinterpret_cast<uint64_t*>(smem);
  uint64_t* s_buf1 = s_buf0 + kCountTile;
  unsigned* s_cnt = reinterpret_cast<unsigned*>(s_buf1 + kCountTile);
  __shared__ __align__(8) unsigned long long s_bar[2];
  for (uint32_t i = threadIdx.x; i < n_slices; i += blockDim.x) s_cnt[i] = 0;
  const uint64_t pol = policy_evict_first();
  const uint64_t a = static_cast<uint64_t>(blockIdx.x) * range;
  const uint64_t b = a + range < n ? a + range : n;
  const uint64_t n_tiles = a < b ? (b - a + kCountTile - 1) / kCountTile : 0;
  bool bulk = (reinterpret_cast<uintptr_t>(hashes) & 15) == 0 && n_tiles > 0;
  const uint32_t bar0 = smem_u32(&s_bar[0]), bar1 = smem_u32(&s_bar[1]);
  if (threadIdx.x == 0 && bulk) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar0) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar1) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  auto issue = [&](uint64_t t) {
    const uint64_t t0 = a + t * kCountTile;
    const uint64_t m = b - t0 < kCountTile ? b - t0 : kCountTile;
    bulk_load((t & 1) ? s_buf1 : s_buf0, hashes + t0, static_cast<uint32_t>((m & ~1ull) * 8),
              (t & 1) ? bar1 : bar0);
  };
  if (threadIdx.x == 0 && bulk) issue(0);
  uint32_t parity = 0;
  for (uint64_t t = 0; t < n_tiles; ++t) {
    const uint64_t t0 = a + t * kCountTile;
    const uint32_t m = static_cast<uint32_t>(b - t0 < kCountTile ? b - t0 : kCountTile);
    const int cur = static_cast<int>(t & 1);
    uint64_t* s_in = cur ? s_buf1 : s_buf0;
    if (bulk) {
      if (threadIdx.x == 0 && t + 1 < n_tiles) issue(t + 1);
      const bool ok = wait_phase(cur ? bar1 : bar0, (parity >> cur) & 1);
      parity ^= 1u << cur;
      bulk = __syncthreads_and(ok);
      if (bulk && (m & 1) && threadIdx.x == 0) s_in[m - 1] = load_key1(hashes + t0 + m - 1, pol);
      __syncthreads();
    }
    for (uint32_t j0 = 0; j0 < m; j0 += blockDim.x) {
      const uint32_t j = j0 + threadIdx.x;
      const bool v = j < m;
      const uint64_t key = !v ? 0 : bulk ? s_in[j] : load_key1(hashes + t0 + j, pol);
      count_warp<kFew>(s_cnt, n_slices, v, v ? slice_of(key, nb, shift) : 0u);
    }
    __syncthreads();  // this buffer's readers are done before it is refilled
  }
  for (uint32_t i = threadIdx.x; i < n_slices; i += blockDim.x)
    hist[static_cast<uint64_t>(blockIdx.x) * n_slices + i] = s_cnt[i];
}

// From the per-CTA histograms of `ctas` CTAs: offsets[0..n_slices] (slice
// starts in the sorted array, exclusive scan of the slice totals) and
// base[c * n_slices + p] = offsets[p] + keys of slice p in the ranges of CTAs
// before c.  One CTA.
__global__ void __launch_bounds__(1024)
    scan_kernel(const unsigned* __restrict__ hist, uint32_t ctas, uint32_t n_slices,
                unsigned long long* __restrict__ offsets, unsigned long long* __restrict__ base) {
  __shared__ unsigned long long warp_total[32];
  __shared__ unsigned long long carry;
  const unsigned lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (uint32_t start = 0; start < n_slices; start += blockDim.x) {
    const uint32_t t = start + threadIdx.x;
    unsigned long long v = 0;
    if (t < n_slices)
      for (uint32_t c = 0; c < ctas; ++c) v += hist[static_cast<uint64_t>(c) * n_slices + t];
    unsigned long long x = v;
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long y = __shfl_up_sync(0xFFFFFFFFu, x, o);
      if (lane >= static_cast<unsigned>(o)) x += y;
    }
    if (lane == 31) warp_total[warp] = x;
    __syncthreads();
    if (warp == 0) {
      unsigned long long s = warp_total[lane];
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xFFFFFFFFu, s, o);
        if (lane >= static_cast<unsigned>(o)) s += y;
      }
      warp_total[lane] = s;
    }
    __syncthreads();
    const unsigned long long before = carry + (warp > 0 ? warp_total[warp - 1] : 0ull) + x - v;
    if (t < n_slices) {
      offsets[t] = before;
      unsigned long long run = before;
      for (uint32_t c = 0; c < ctas; ++c) {
        base[static_cast<uint64_t>(c) * n_slices + t] = run;
        run += hist[static_cast<uint64_t>(c) * n_slices + t];
      }
    }
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) carry += warp_total[31];
    __syncthreads();
  }
  if (threadIdx.x == 0) offsets[n_slices] = carry;
}

// Exclusive scan of vals[0..n) in place over the CTA (n <= 8 * blockDim);
// each thread scans up to 8 consecutive entries, then the per-thread sums
// are scanned with warp shuffles.  Callers synchronise before the call; it
// ends with a barrier.
__device__ __forceinline__ void cta_exclusive_scan(unsigned* vals, uint32_t n, unsigned* warp_sums) {
  const uint32_t per = (n + blockDim.x - 1) / blockDim.x;
  const uint32_t a = threadIdx.x * per, b = a + per < n ? a + per : n;
  unsigned sum = 0;
  for (uint32_t i = a; i < b; ++i) sum += vals[i];
  const unsigned lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned x = sum;
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned y = __shfl_up_sync(0xFFFFFFFFu, x, o);
    if (lane >= static_cast<unsigned>(o)) x += y;
  }
  if (lane == 31) warp_sums[warp] = x;
  __syncthreads();
  if (warp == 0) {
    const unsigned nw = blockDim.x >> 5;
    unsigned w = lane < nw ? warp_sums[lane] : 0u;
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned y = __shfl_up_sync(0xFFFFFFFFu, w, o);
      if (lane >= static_cast<unsigned>(o)) w += y;
    }
    if (lane < nw) warp_sums[lane] = w;
  }
  __syncthreads();
  unsigned run = (warp > 0 ? warp_sums[warp - 1] : 0u) + x - sum;
  for (uint32_t i = a; i < b; ++i) {
    const unsigned v = vals[i];
    vals[i] = run;
    run += v;
  }
  __syncthreads();
}

// Shared memory of the scatter: two input tiles, the sorted tile, the
// per-slice output cursors (u64) and counts / run starts / rank cursors
// (u32), and the tile positions of the sorted keys (u16, lookups only).
__host__ __device__ constexpr size_t scatter_smem_bytes(uint32_t tile, uint32_t n_slices,
                                                        bool with_index) {
  return 3ull * 8 * tile + 12ull * n_slices + (with_index ? 2ull * tile : 0);
}

// Keys into slice order.  CTA c streams its range in tiles of kT keys: each
// key claims its rank among the tile's keys of its slice with one shared
// atomic (so the counters end as the slice counts), the counts are scanned
// in place into run starts, a key goes to run start + rank in the sorted
// tile, and each slice's run is written at the CTA's cursor for that slice
// (from the scan), kept during the tile as cursor minus run start so that a
// key's output position is one add.  Tile t+1 is bulk-copied into the other buffer while
// tile t is processed.  The copies need a 16-byte aligned key array; with
// any other alignment, or if a copy ever failed to complete in time, the
// CTA reads the keys straight from global memory instead.  Lookups (kIndex)
// also write each key's original position, as its 16-bit offset within its
// sub-range, and the cursors at every sub-range start (and after the last
// tile) to marks[c][u][q], `rows` rows per CTA.
template <bool kFew, bool kIndex, uint32_t kT>
__global__ void __launch_bounds__(kPartThreads, 1)
    scatter_kernel(const uint64_t* __restrict__ hashes, uint64_t n, uint32_t nb, int shift,
                   uint32_t n_slices, uint64_t range, const unsigned long long* __restrict__ base,
                   uint64_t* __restrict__ out, uint16_t* __restrict__ out_idx,
                   uint32_t* __restrict__ marks, uint32_t rows) {
  static_assert(kSubKeys % kT == 0, "a sub-range is a whole number of tiles");
  static_assert(kT % kPartThreads == 0 && kT <= 8192, "whole keys per thread; 13-bit ranks");
  constexpr uint32_t kPer = kT / kPartThreads;  // launched with kPartThreads threads
  extern __shared__ __align__(16) unsigned long long smem[];
  uint64_t* s_buf0 = reinterpret_cast<uint64_t*>(smem);
  uint64_t* s_buf1 = s_buf0 + kT;
  uint64_t* s_sorted = s_buf1 + kT;
  unsigned long long* s_cursor = reinterpret_cast<unsigned long long*>(s_sorted + kT);
  unsigned* s_cnt = reinterpret_cast<unsigned*>(s_cursor + n_slices);
  uint16_t* s_pos = reinterpret_cast<uint16_t*>(s_cnt + n_slices);  // kIndex
  __shared__ unsigned warp_sums[32];
  __shared__ __align__(8) unsigned long long s_bar[2];

  const uint64_t a = static_cast<uint64_t>(blockIdx.x) * range;
  if (a >= n) return;  // the whole CTA: nothing of the key array is ours
  const uint64_t b = a + range < n ? a + range : n;
  const uint64_t n_tiles = (b - a + kT - 1) / kT;
  for (uint32_t i = threadIdx.x; i < n_slices; i += blockDim.x) {
    s_cursor[i] = base[static_cast<uint64_t>(blockIdx.x) * n_slices + i];
    s_cnt[i] = 0;
  }
  bool bulk = (reinterpret_cast<uintptr_t>(hashes) & 15) == 0;  // uniform over the CTA
  const uint32_t bar0 = smem_u32(&s_bar[0]), bar1 = smem_u32(&s_bar[1]);
  if (threadIdx.x == 0 && bulk) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar0) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar1) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  // thread 0 starts the copy of tile t (its even-length head; an odd last
  // key is loaded after the wait)
  auto issue = [&](uint64_t t) {
    const uint64_t t0 = a + t * kT;
    const uint64_t m = b - t0 < kT ? b - t0 : kT;
    bulk_load((t & 1) ? s_buf1 : s_buf0, hashes + t0, static_cast<uint32_t>((m & ~1ull) * 8),
              (t & 1) ? bar1 : bar0);
  };
  if (threadIdx.x == 0 && bulk) issue(0);
  uint32_t parity = 0;  // bit i: phase parity expected next on buffer i
  const uint64_t pol = policy_evict_first();

  uint32_t* my_marks = kIndex ? marks + static_cast<uint64_t>(blockIdx.x) * rows * n_slices
                              : nullptr;
  for (uint64_t t = 0; t < n_tiles; ++t) {
    const uint64_t t0 = a + t * kT;
    const uint32_t m = static_cast<uint32_t>(b - t0 < kT ? b - t0 : kT);
    const int cur = static_cast<int>(t & 1);
    uint64_t* s_in = cur ? s_buf1 : s_buf0;
    // offset of the tile's first key within its sub-range
    const uint32_t sub_off = static_cast<uint32_t>((t % (kSubKeys / kT)) * kT);
    if (kIndex && sub_off == 0) {  // cursors are true cursors between tiles
      uint32_t* row = my_marks + (t / (kSubKeys / kT)) * n_slices;
      for (uint32_t i = threadIdx.x; i < n_slices; i += blockDim.x)
        row[i] = static_cast<uint32_t>(s_cursor[i]);
    }
    if (bulk) {
      // the other buffer's last reader finished at the previous tile's end
      if (threadIdx.x == 0 && t + 1 < n_tiles) issue(t + 1);
      // an odd last key lies past the copied span: stored before the barrier
      if ((m & 1) && threadIdx.x == 0) s_in[m - 1] = load_key1(hashes + t0 + m - 1, pol);
      const bool ok = wait_phase(cur ? bar1 : bar0, (parity >> cur) & 1);
      parity ^= 1u << cur;
      bulk = __syncthreads_and(ok);  // all threads agree; on failure never use the buffers again
    }
    const bool from_smem = bulk;
    auto key_at = [&](uint32_t j) -> uint64_t {
      return from_smem ? s_in[j] : load_key1(hashes + t0 + j, pol);
    };
    // each key claims its rank among the tile's keys of its slice (the
    // counters end as the slice counts); slice and rank stay in registers
    uint32_t qr[kPer];  // slice << 13 | rank
#pragma unroll
    for (uint32_t i = 0; i < kPer; ++i) {
      const uint32_t j = i * kPartThreads + threadIdx.x;
      const bool v = j < m;
      const uint32_t q = v ? slice_of(key_at(j), nb, shift) : 0u;
      qr[i] = (q << 13) | rank_warp<kFew>(s_cnt, n_slices, v, q);
    }
    __syncthreads();
    cta_exclusive_scan(s_cnt, n_slices, warp_sums);  // counts -> run starts (ends with a barrier)
    for (uint32_t i = threadIdx.x; i < n_slices; i += blockDim.x) s_cursor[i] -= s_cnt[i];
#pragma unroll
    for (uint32_t i = 0; i < kPer; ++i) {
      const uint32_t j = i * kPartThreads + threadIdx.x;
      if (j < m) {
        const unsigned at = s_cnt[qr[i] >> 13] + (qr[i] & 0x1FFFu);  // run start + rank
        s_sorted[at] = key_at(j);
        if (kIndex) s_pos[at] = static_cast<uint16_t>(j);
      }
    }
    __syncthreads();
    for (uint32_t j = threadIdx.x; j < m; j += blockDim.x) {
      const uint64_t key = s_sorted[j];
      const unsigned long long pos = s_cursor[slice_of(key, nb, shift)] + j;
      if (pos < n) {  // in range unless the input changed between the passes
        out[pos] = key;
        if (kIndex) out_idx[pos] = static_cast<uint16_t>(sub_off + s_pos[j]);
      }
    }
    __syncthreads();
    // the cursor advances by the run's length: cursor - start + end
    for (uint32_t i = threadIdx.x; i < n_slices; i += blockDim.x)
      s_cursor[i] += i + 1 < n_slices ? s_cnt[i + 1] : m;
    __syncthreads();  // every run end is read before the counters are cleared
    for (uint32_t i = threadIdx.x; i < n_slices; i += blockDim.x) s_cnt[i] = 0;
    __syncthreads();
  }
  if (kIndex) {
    uint32_t* row = my_marks + static_cast<uint64_t>(sub_ranges(b - a)) * n_slices;
    for (uint32_t i = threadIdx.x; i < n_slices; i += blockDim.x)
      row[i] = static_cast<uint32_t>(s_cursor[i]);
  }
}

// Prefetches bytes [lo, hi) of the filter words into L2 (16-byte multiples);
// the lanes of the calling warp split the range into bulk prefetches of at
// most 16 KiB.
__device__ __forceinline__ void prefetch_bytes(const uint32_t* words, uint64_t lo, uint64_t hi) {
  constexpr uint64_t kChunk = 16 * 1024;
  const char* base = reinterpret_cast<const char*>(words);
  for (uint64_t off = lo + static_cast<uint64_t>(lane_id()) * kChunk; off < hi; off += 32 * kChunk) {
    const uint64_t sz = hi - off < kChunk ? hi - off : kChunk;
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(base + off),
                 "r"(static_cast<uint32_t>(sz))
                 : "memory");
  }
}

// Streaming prefetch by key position.  Slice q holds sorted positions
// [offsets[q], offsets[q+1]) and filter blocks [q << shift, ...); the
// position p of slice q is mapped to byte
//   slice_lo + floor((p - first) * slice_bytes / keys / 32) * 32
// so consecutive position ranges map to consecutive, disjoint byte ranges and
// every byte of every slice that holds keys is covered exactly once.  A warp
// prefetches the bytes of positions [p0, p1) (any number of slices).
__device__ __forceinline__ uint64_t position_byte(uint32_t nb, int shift, uint32_t q,
                                                  uint64_t first, uint64_t keys, uint64_t p) {
  const uint64_t b0 = static_cast<uint64_t>(q) << shift;
  const uint64_t b1 = b0 + (1ull << shift) < nb ? b0 + (1ull << shift) : nb;
  const uint64_t blocks = b1 - b0;
  // (p - first) * blocks / keys without overflow: both factors < 2^32 here
  // unless keys is large, so split the quotient
  const uint64_t d = p - first;
  const uint64_t blk = (d / keys) * blocks + ((d % keys) * blocks) / keys;
  return 32 * (b0 + blk);
}

__device__ __forceinline__ void prefetch_positions(const uint32_t* words, uint32_t nb, int shift,
                                                   const unsigned long long* __restrict__ offsets,
                                                   uint32_t n_slices, uint64_t p0, uint64_t p1) {
  const uint64_t n = offsets[n_slices];
  if (p0 >= n) return;
  if (p1 > n) p1 = n;
  uint32_t lo = 0, hi = n_slices;  // last q with offsets[q] <= p0
  while (hi - lo > 1) {
    const uint32_t mid = (lo + hi) >> 1;
    if (offsets[mid] <= p0) lo = mid; else hi = mid;
  }
  for (uint32_t q = lo; q < n_slices && offsets[q] < p1; ++q) {
    const uint64_t first = offsets[q], last = offsets[q + 1];
    if (last == first) continue;
    const uint64_t a = p0 > first ? p0 : first, b = p1 < last ? p1 : last;
    if (a >= b) continue;
    prefetch_bytes(words, position_byte(nb, shift, q, first, last - first, a),
                   position_byte(nb, shift, q, first, last - first, b));
  }
}

// Distance, in sorted positions, that the streaming prefetch runs ahead of
// the newest claimed tile: one whole slice of keys (the largest), so a
// slice's blocks are all in L2 before its first key is processed, plus half
// the window of keys in flight, for the prefetches to land.  The L2
// footprint is then about one slice plus 1.5 windows of filter bytes.  One
// warp computes it (all lanes return the same value).
__device__ __forceinline__ uint64_t prefetch_ahead(const unsigned long long* __restrict__ offsets,
                                                   uint32_t n_slices, uint64_t window) {
  unsigned long long k_max = 0;
  for (uint32_t q = lane_id(); q < n_slices; q += 32) {
    const unsigned long long k = offsets[q + 1] - offsets[q];
    k_max = k > k_max ? k : k_max;
  }
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long v = __shfl_xor_sync(0xFFFFFFFFu, k_max, o);
    k_max = v > k_max ? v : k_max;
  }
  return k_max + window / 2;
}

// Rounds of 64-key groups per warp per tile (a launch argument, 1..8; even
// for lookups).  The host picks it from the filter bytes per key: the window
// of keys in flight (CTAs x tile) times that is held near 24 MiB, so window
// and prefetch fit in L2 with a slice; dense batches get long tiles (fewer
// claims of the shared tile counter), sparse ones short tiles.
constexpr int kMaxSlicedRounds = 8;

// Slice-ordered insert with the in-order dynamic tile schedule.  Every tile
// at position a0 prefetches the filter bytes of positions [a0 + ahead,
// a0 + ahead + tile) (see prefetch_ahead), so each block is read from DRAM
// once, sequentially, before its keys arrive.  At launch the CTAs split the
// prefetch of positions [0, ahead).
__global__ void __launch_bounds__(256)
    sliced_insert_kernel(uint32_t* __restrict__ words, uint32_t nb, int shift,
                         const uint64_t* __restrict__ keys, uint64_t n,
                         const unsigned long long* __restrict__ offsets, uint32_t n_slices,
                         unsigned long long* __restrict__ tiles, int rounds) {
  __shared__ unsigned long long s_tile;
  const unsigned wpc = blockDim.x >> 5, wic = threadIdx.x >> 5;
  const uint64_t n_groups = (n + 63) >> 6;
  const uint64_t groups_per_tile = static_cast<uint64_t>(wpc) * rounds;
  const uint64_t keys_per_tile = groups_per_tile * 64;
  const uint64_t pol = policy_evict_first();
  OneFilter res{nb};
  uint64_t ahead = 0;
  if (wic == 0) {
    ahead = prefetch_ahead(offsets, n_slices, keys_per_tile * gridDim.x);
    const uint64_t share = (ahead + gridDim.x - 1) / gridDim.x;
    prefetch_positions(words, nb, shift, offsets, n_slices, blockIdx.x * share,
                       (blockIdx.x + 1) * share);
  }
  for (;;) {
    if (threadIdx.x == 0) s_tile = atomicAdd(tiles, 1ull);
    __syncthreads();
    const uint64_t g0 = s_tile * groups_per_tile;
    __syncthreads();
    if (g0 >= n_groups) break;
    if (wic == 0)
      prefetch_positions(words, nb, shift, offsets, n_slices, g0 * 64 + ahead,
                         g0 * 64 + ahead + keys_per_tile);
    for (int r = 0; r < rounds; ++r) {
      const uint64_t g = g0 + static_cast<uint64_t>(r) * wpc + wic;
      if (g < n_groups) insert_group8(words, res, HashInput(keys), n, pol, g);
    }
  }
}

// Bits of x (16 bits) at the even positions and of y at the odd positions
// of a 32-bit word.
__device__ __forceinline__ uint32_t spread16(uint32_t x) {
  x = (x | (x << 8)) & 0x00FF00FFu;
  x = (x | (x << 4)) & 0x0F0F0F0Fu;
  x = (x | (x << 2)) & 0x33333333u;
  return (x | (x << 1)) & 0x55555555u;
}

__device__ __forceinline__ uint32_t interleave16(uint32_t x, uint32_t y) {
  return spread16(x) | (spread16(y) << 1);
}

// Slice-ordered lookups of keys[0..n), with the same schedule and streaming
// prefetch as the sliced insert.  The answers are written in sorted order,
// packed like the unpartitioned lookup's (bit k of the pair of words 2g, 2g+1
// answers sorted position 64g + k); unscatter_kernel moves them to the keys'
// original positions.
__global__ void __launch_bounds__(256, 4)
    sliced_find_kernel(const uint32_t* __restrict__ words, uint32_t nb, int shift,
                       const uint64_t* __restrict__ keys, uint64_t n,
                       const unsigned long long* __restrict__ offsets, uint32_t n_slices,
                       unsigned long long* __restrict__ tiles, uint32_t* __restrict__ sorted_bits,
                       int rounds) {
  __shared__ unsigned long long s_tile;
  const unsigned wpc = blockDim.x >> 5, wic = threadIdx.x >> 5, lane = lane_id();
  const uint64_t n_groups = (n + 63) >> 6;
  const uint64_t groups_per_tile = static_cast<uint64_t>(wpc) * rounds;
  const uint64_t keys_per_tile = groups_per_tile * 64;
  const uint64_t pk = policy_evict_first();
  // block loads at evict-last priority: the near die then keeps its copies of
  // lines that live in the other die's memory, which halved the requests
  // crossing the die-to-die fabric on a 2 GiB filter (50.2M against 100.8M
  // for 128M keys) and cut the pass from 0.83 to 0.74 ms at the same DRAM
  // reads (evict-normal loads measured 4-5% slower overall)
  const uint64_t pf = policy_evict_last();
  uint64_t ahead = 0;
  if (wic == 0) {
    ahead = prefetch_ahead(offsets, n_slices, keys_per_tile * gridDim.x);
    const uint64_t share = (ahead + gridDim.x - 1) / gridDim.x;
    prefetch_positions(words, nb, shift, offsets, n_slices, blockIdx.x * share,
                       (blockIdx.x + 1) * share);
  }
  for (;;) {
    if (threadIdx.x == 0) s_tile = atomicAdd(tiles, 1ull);
    __syncthreads();
    const uint64_t g0 = s_tile * groups_per_tile;
    __syncthreads();
    if (g0 >= n_groups) break;
    if (wic == 0)
      prefetch_positions(words, nb, shift, offsets, n_slices, g0 * 64 + ahead,
                         g0 * 64 + ahead + keys_per_tile);
    // two rounds per step: four block loads per lane in flight before any test
    for (int r = 0; r < rounds; r += 2) {
      uint64_t k[2], h[2][2];
      uint32_t w[2][2][8];
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const uint64_t g = g0 + static_cast<uint64_t>(r + u) * wpc + wic;
        k[u] = g * 64 + 2 * lane;  // >= n past the last group
        HashInput(keys).pair(k[u], n, pk, h[u][0], h[u][1]);
      }
#pragma unroll
      for (int u = 0; u < 2; ++u) {
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          if (k[u] + e < n) {
            load_block_na(words + 8ull * block_of(h[u][e], nb), pf, w[u][e]);
          } else {
#pragma unroll
            for (int i = 0; i < 8; ++i) w[u][e][i] = 0;
          }
        }
      }
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        // bit l of b0 / b1: key 2l / 2l + 1 of the group
        const uint32_t b0 = __ballot_sync(
            0xFFFFFFFFu, k[u] < n && block_has(w[u][0], static_cast<uint32_t>(h[u][0])));
        const uint32_t b1 = __ballot_sync(
            0xFFFFFFFFu, k[u] + 1 < n && block_has(w[u][1], static_cast<uint32_t>(h[u][1])));
        const uint64_t g = g0 + static_cast<uint64_t>(r + u) * wpc + wic;
        if (lane == 0 && g < n_groups)
          *reinterpret_cast<uint2*>(sorted_bits + 2 * g) =
              make_uint2(interleave16(b0 & 0xFFFFu, b1 & 0xFFFFu), interleave16(b0 >> 16, b1 >> 16));
      }
    }
  }
}

// Answers back into key order.  CTA (c, u) owns the original positions
// [lo, hi): sub-range u of scatter CTA c's key range.  The scatter put the
// keys of that sub-range that fall in slice q at sorted positions
// [marks[c][u][q], marks[c][u + 1][q]).  The CTA lists the answer words that
// overlap these runs (shared memory holds each run's bounds and the list
// offset of its first word); a lane takes one word, masks it to its run, and
// for each found key -- each set bit -- loads the key's offset within the
// sub-range and sets its bit in a shared-memory copy of the sub-range's
// result words, four bits per round so that their loads overlap.  The words
// are then stored whole: every result word belongs to exactly one CTA, so there are
// no global atomics and no zeroing pass.  Positions and runs are clamped to
// their buffers, so keys that changed between the passes give wrong answers,
// never an access out of bounds.
constexpr int kUnscatterThreads = 512;

__host__ __device__ constexpr size_t unscatter_smem_bytes(uint32_t n_slices) {
  return 4ull * (kSubKeys / 32) + 4ull * 3 * n_slices;
}

__global__ void __launch_bounds__(kUnscatterThreads)
    unscatter_kernel(const uint32_t* __restrict__ sorted_bits, const uint16_t* __restrict__ idx,
                     const uint32_t* __restrict__ marks, uint64_t n, uint64_t range, uint32_t rows,
                     uint32_t n_slices, uint32_t* __restrict__ out) {
  extern __shared__ __align__(16) uint32_t s_mem[];
  uint32_t* s_out = s_mem;                           // result words of the sub-range
  uint32_t* s_lo = s_out + kSubKeys / 32;            // run q: sorted positions [s_lo, s_hi)
  uint32_t* s_hi = s_lo + n_slices;
  uint32_t* s_item = s_hi + n_slices;                // list offset of run q's first word
  __shared__ unsigned warp_sums[32];
  __shared__ uint32_t s_last;
  const uint32_t subs = rows - 1;
  const uint32_t c = blockIdx.x / subs, u = blockIdx.x % subs;
  const uint64_t a = static_cast<uint64_t>(c) * range;
  const uint64_t end = a + range < n ? a + range : n;
  const uint64_t lo = a + static_cast<uint64_t>(u) * kSubKeys;
  if (lo >= end) return;  // the whole CTA
  const uint64_t hi = lo + kSubKeys < end ? lo + kSubKeys : end;
  const uint32_t span = static_cast<uint32_t>(hi - lo);
  const uint32_t n_words = (span + 31) / 32;
  const uint32_t* m0 = marks + (static_cast<uint64_t>(c) * rows + u) * n_slices;
  const uint32_t* m1 = m0 + n_slices;
  for (uint32_t i = threadIdx.x; i < n_words; i += blockDim.x) s_out[i] = 0;
  for (uint32_t q = threadIdx.x; q < n_slices; q += blockDim.x) {
    const uint32_t p1 = static_cast<uint32_t>(m1[q] < n ? m1[q] : n);
    const uint32_t p0 = m0[q] < p1 ? m0[q] : p1;
    s_lo[q] = p0;
    s_hi[q] = p1;
    const uint32_t words = p1 > p0 ? ((p1 - 1) >> 5) - (p0 >> 5) + 1 : 0u;
    s_item[q] = words;  // scanned next
    if (q == n_slices - 1) s_last = words;
  }
  __syncthreads();
  cta_exclusive_scan(s_item, n_slices, warp_sums);
  const uint32_t items = s_item[n_slices - 1] + s_last;
  const unsigned lane = threadIdx.x & 31;
  for (uint32_t i0 = threadIdx.x & ~31u; i0 < items; i0 += blockDim.x) {
    const uint32_t i = i0 + lane;
    uint32_t bits = 0, base = 0;
    if (i < items) {
      uint32_t l = 0, r = n_slices;  // the run holding item i: last q with s_item[q] <= i
      while (r - l > 1) {
        const uint32_t mid = (l + r) >> 1;
        if (s_item[mid] <= i) l = mid; else r = mid;
      }
      const uint32_t w = (s_lo[l] >> 5) + (i - s_item[l]);
      base = 32 * w;
      const uint32_t from = s_lo[l] > base ? s_lo[l] - base : 0u;
      const uint32_t to = s_hi[l] - base < 32 ? s_hi[l] - base : 32u;
      const uint32_t mask = (to == 32 ? 0xFFFFFFFFu : (1u << to) - 1) & ~((1u << from) - 1);
      bits = __ldg(sorted_bits + w) & mask;
    }
    while (__any_sync(0xFFFFFFFFu, bits != 0)) {
      uint32_t j[4];
      bool has[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        has[e] = bits != 0;
        const uint32_t p = base + (has[e] ? __ffs(bits) - 1 : 0u);
        bits &= bits - 1;
        j[e] = has[e] ? __ldg(idx + p) : 0u;  // offset within the sub-range
      }
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        if (has[e] && j[e] < span) atomicOr(&s_out[j[e] >> 5], 1u << (j[e] & 31));
      }
    }
  }
  __syncthreads();
  uint32_t* dst = out + lo / 32;
  for (uint32_t i = threadIdx.x; i < n_words; i += blockDim.x) dst[i] = s_out[i];
}

inline uint64_t align256(uint64_t x) { return (x + 255) & ~255ull; }

// Tile rounds for a sliced launch of `grid` CTAs of 8 warps over n keys into
// a filter of `filter_bytes`: the largest power of two (at least `min_rounds`,
// at most kMaxSlicedRounds) whose window of keys times filter bytes per key
// stays within 24 MiB.
int sliced_rounds(unsigned grid, uint64_t n, uint64_t filter_bytes, int min_rounds) {
  const double bytes_per_key = static_cast<double>(filter_bytes) / static_cast<double>(n);
  const double window_keys = 24.0 * 1024 * 1024 / bytes_per_key;
  int r = min_rounds;
  while (r < kMaxSlicedRounds && 2.0 * r * grid * 8 * 64 <= window_keys) r *= 2;
  return r;
}

// Dynamic shared memory a CTA may use on this architecture (227 KB), less a
// margin for the kernel's static shared memory.
constexpr size_t kSmemBudget = 227 * 1024 - 512;

// Scatter tile size: 8192 keys while three tiles, the index and the slice
// tables fit, else 4096.
uint32_t scatter_tile(uint32_t n_slices, bool with_index) {
  return scatter_smem_bytes(8192, n_slices, with_index) <= kSmemBudget ? 8192u : 4096u;
}

// CTAs of the count and scatter passes (one per SM; both use the same key
// ranges).
uint32_t partition_ctas() { return static_cast<uint32_t>(sm_count()); }

uint32_t slices_at(uint32_t num_blocks, int shift) {
  return static_cast<uint32_t>((static_cast<uint64_t>(num_blocks) + (1ull << shift) - 1) >> shift);
}

// Smallest slice shift lookups may take: 4 MiB, or larger until at most 1024
// slices (the scatter's shared-memory tables).
int lookup_min_shift(uint32_t num_blocks) {
  int shift = kMinSliceShift;
  while (shift < kMaxSliceShift && slices_at(num_blocks, shift) > 1024) ++shift;
  return shift;
}

int find_occupancy() {
  static const int occ = occupancy(sliced_find_kernel, 256);
  return occ;
}

// The slice stream keeps its reads exact while a slice plus 1.5 windows of
// filter bytes stay below ~48 MiB of L2 (measured on a 2 GiB filter: 62 MB
// live, 5.85 GB of DRAM reads for 3.5 GB of keys and filter; 46 MB, 4.31 GB).
constexpr double kLiveBytes = 48.0 * 1024 * 1024;

// Slice shift, grid and tile rounds of a partitioned lookup of n keys.  A
// slice's blocks stay in L2 from its prefetch until its last key is
// processed, so a slice plus the keys in flight (and those prefetched ahead)
// must fit there, while the scatter of positions pays for every extra slice
// (shorter runs): lookups take the largest slice (at most 32 MiB, no smaller than
// lookup_min_shift) within the live-set budget.  When even that slice leaves
// too little room -- sparse batches, many filter bytes per key -- the grid
// shrinks (to one CTA per SM at least) until the window fits beside it.
struct FindPlan {
  int shift;
  unsigned grid;
  int rounds;
};

FindPlan find_plan(uint32_t num_blocks, uint64_t n) {
  const double per_key = 32.0 * num_blocks / static_cast<double>(n);
  unsigned grid = grid_for((n + 63) / 64, 8, find_occupancy());
  const int rounds = sliced_rounds(grid, n, 32ull * num_blocks, 2);
  const double keys_per_cta = 8.0 * rounds * 64;
  const double window = grid * keys_per_cta * per_key;
  const int floor_shift = lookup_min_shift(num_blocks);
  int shift = kMaxSliceShift;
  while (shift > floor_shift && 32.0 * static_cast<double>(1ull << shift) + 1.5 * window > kLiveBytes)
    --shift;
  const double room = (kLiveBytes - 32.0 * static_cast<double>(1ull << shift)) / 1.5;
  if (window > room) {
    const double cap = room / per_key / keys_per_cta;
    const unsigned floor_grid = static_cast<unsigned>(sm_count());
    unsigned g = cap < grid ? static_cast<unsigned>(cap) : grid;
    grid = g > floor_grid ? g : (floor_grid < grid ? floor_grid : grid);
  }
  return {shift, grid, rounds};
}

// Blocks per slice, 2^shift.  For inserts slices get smaller as long as the
// partition's fan-out stays near kTargetSlices (the scatter's runs per tile
// shrink with more slices), between 4 and 32 MiB: measured 67.6 against
// 60.3 G inserts/s on a 2 GiB filter.  Lookups: find_plan.
int slice_shift(uint32_t num_blocks, uint64_t n, bool lookup) {
  if (lookup) return find_plan(num_blocks, n).shift;
  int shift = kMinSliceShift;
  while (shift < kMaxSliceShift && slices_at(num_blocks, shift) > kTargetSlices) ++shift;
  return shift;
}

}  // namespace

// Scratch bytes for a partitioned insert (or, with_index, lookup) of n keys
// into num_blocks blocks.
uint64_t partition_scratch_bytes(uint32_t num_blocks, uint64_t n, bool with_index) {
  // lookups: the most slices their rule can pick, so any piece fits
  const uint64_t s = with_index ? slices_at(num_blocks, lookup_min_shift(num_blocks))
                                : slices_at(num_blocks, slice_shift(num_blocks, n, false));
  const uint64_t g = partition_ctas();
  uint64_t bytes = align256(4 * g * s) + align256(8 * g * s) + align256(8 * (s + 1)) + 256 +
                   align256(8 * n);
  if (with_index) {
    const uint64_t rows = sub_ranges(range_keys(n, static_cast<uint32_t>(g))) + 1;
    bytes += align256(2 * n) + align256(8 * ((n + 63) / 64)) + align256(4 * g * rows * s);
  }
  return bytes;
}

// Largest batch a partitioned lookup handles in one pass (32-bit sorted
// positions in the scatter's cursors and marks).
constexpr uint64_t kMaxIndexedKeys = 1ull << 31;

namespace {

struct PartScratch {
  unsigned* hist;                  // [ctas][n_slices]
  unsigned long long* base;        // [ctas][n_slices]
  unsigned long long* offsets;     // [n_slices + 1]
  unsigned long long* tiles;       // dynamic-schedule counter
  uint64_t* sorted;                // [n]
  uint16_t* idx;                   // [n] offset of the original position in its sub-range
  uint32_t* sorted_bits;           // [2 * ceil(n / 64)] answers in sorted order (lookups)
  uint32_t* marks;                 // [ctas][rows][n_slices] sub-range cursors (lookups)
  uint32_t rows;
};

PartScratch carve(void* scratch, uint32_t ctas, uint32_t n_slices, uint64_t n) {
  PartScratch r;
  char* p = static_cast<char*>(scratch);
  const uint64_t cells = static_cast<uint64_t>(ctas) * n_slices;
  r.hist = reinterpret_cast<unsigned*>(p);
  p += align256(4 * cells);
  r.base = reinterpret_cast<unsigned long long*>(p);
  p += align256(8 * cells);
  r.offsets = reinterpret_cast<unsigned long long*>(p);
  p += align256(8 * (n_slices + 1));
  r.tiles = reinterpret_cast<unsigned long long*>(p);
  p += 256;
  r.sorted = reinterpret_cast<uint64_t*>(p);
  p += align256(8 * n);
  r.idx = reinterpret_cast<uint16_t*>(p);
  p += align256(2 * n);
  r.sorted_bits = reinterpret_cast<uint32_t*>(p);
  p += align256(8 * ((n + 63) / 64));
  r.marks = reinterpret_cast<uint32_t*>(p);
  r.rows = sub_ranges(range_keys(n, ctas)) + 1;
  return r;
}

template <bool kFew, bool kIndex, uint32_t kT>
sbbf_status launch_scatter(const uint64_t* hashes, uint64_t n, uint32_t nb, int shift,
                           uint32_t n_slices, uint64_t range, uint32_t ctas, const PartScratch& ps,
                           cudaStream_t s) {
  const size_t smem = scatter_smem_bytes(kT, n_slices, kIndex);
  static const cudaError_t attr = cudaFuncSetAttribute(
      scatter_kernel<kFew, kIndex, kT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
      static_cast<int>(kSmemBudget));
  if (attr != cudaSuccess) return record_cuda(attr);
  scatter_kernel<kFew, kIndex, kT><<<ctas, kPartThreads, smem, s>>>(
      hashes, n, nb, shift, n_slices, range, ps.base, ps.sorted, kIndex ? ps.idx : nullptr,
      kIndex ? ps.marks : nullptr, ps.rows);
  return launch_status();
}

// Steps 1-3: per-CTA counts, offsets and bases, and the slice-ordered keys
// (and positions).
sbbf_status partition(const uint64_t* hashes, uint64_t n, uint32_t num_blocks, int shift,
                      uint32_t n_slices, const PartScratch& ps, bool with_index, cudaStream_t s) {
  const bool few = n_slices <= kFewSlices;
  const uint32_t ctas = partition_ctas();
  const uint64_t range = range_keys(n, ctas);
  const size_t count_smem = 16ull * kCountTile + 4ull * n_slices;
  static const bool count_attr = [] {
    cudaFuncSetAttribute(count_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         static_cast<int>(kSmemBudget));
    cudaFuncSetAttribute(count_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         static_cast<int>(kSmemBudget));
    return true;
  }();
  (void)count_attr;
  if (few)
    count_kernel<true><<<ctas, kCountThreads, count_smem, s>>>(hashes, n, num_blocks, shift,
                                                              n_slices, range, ps.hist);
  else
    count_kernel<false><<<ctas, kCountThreads, count_smem, s>>>(hashes, n, num_blocks, shift,
                                                               n_slices, range, ps.hist);
  sbbf_status st = launch_status();
  if (st != SBBF_OK) return st;
  scan_kernel<<<1, 1024, 0, s>>>(ps.hist, ctas, n_slices, ps.offsets, ps.base);
  if ((st = launch_status()) != SBBF_OK) return st;
  const bool big = scatter_tile(n_slices, with_index) == 8192;
  const auto args = [&](auto launch) {
    return launch(hashes, n, num_blocks, shift, n_slices, range, ctas, ps, s);
  };
  if (few)
    return with_index ? args(launch_scatter<true, true, 8192>)
                      : args(launch_scatter<true, false, 8192>);
  if (with_index)
    return big ? args(launch_scatter<false, true, 8192>) : args(launch_scatter<false, true, 4096>);
  return big ? args(launch_scatter<false, false, 8192>) : args(launch_scatter<false, false, 4096>);
}

}  // namespace

// Partitioned insert (see the file comment).  `scratch` holds at least
// partition_scratch_bytes(num_blocks, n, false) bytes of device memory.
sbbf_status launch_insert_partitioned(uint32_t* words, uint32_t num_blocks, const uint64_t* hashes,
                                      uint64_t n, void* scratch, cudaStream_t s) {
  SBBF_TRACE_NAMED("sbbf_partitioned_insert");
  if (n == 0) return SBBF_OK;
  const int shift = slice_shift(num_blocks, n, false);
  const uint32_t n_slices = slices_at(num_blocks, shift);
  if (n_slices == 0 || n_slices > kMaxSlices) return SBBF_EINVAL;
  const PartScratch ps = carve(scratch, partition_ctas(), n_slices, n);
  sbbf_status st = partition(hashes, n, num_blocks, shift, n_slices, ps, false, s);
  if (st != SBBF_OK) return st;
  SBBF_CUDA(cudaMemsetAsync(ps.tiles, 0, 8, s));
  static int occ_ins = occupancy(sliced_insert_kernel, 256);
  const unsigned grid = grid_for((n + 63) / 64, 8, occ_ins);
  const int rounds = sliced_rounds(grid, n, 32ull * num_blocks, 1);
  sliced_insert_kernel<<<grid, 256, 0, s>>>(words, num_blocks, shift, ps.sorted, n, ps.offsets,
                                            n_slices, ps.tiles, rounds);
  return launch_status();
}

// Partitioned lookup of d_hashes[0..n) into the packed bitmask d_out (the
// same bits as the unpartitioned lookup; every word of the answer is
// written).  `scratch` holds at least partition_scratch_bytes(num_blocks,
// min(n, 2^31), true) bytes; batches larger than 2^31 keys run in pieces of
// 2^31 (a multiple of 32).
sbbf_status launch_find_partitioned(const uint32_t* words, uint32_t num_blocks,
                                    const uint64_t* hashes, uint64_t n, uint32_t* d_out,
                                    void* scratch, cudaStream_t s) {
  SBBF_TRACE_NAMED("sbbf_partitioned_find");
  if (n == 0) return SBBF_OK;
  for (uint64_t off = 0; off < n; off += kMaxIndexedKeys) {
    const uint64_t m = n - off < kMaxIndexedKeys ? n - off : kMaxIndexedKeys;
    const FindPlan plan = find_plan(num_blocks, m);
    const uint32_t n_slices = slices_at(num_blocks, plan.shift);
    if (n_slices == 0 || n_slices > kMaxSlices) return SBBF_EINVAL;
    const uint32_t ctas = partition_ctas();
    const PartScratch ps = carve(scratch, ctas, n_slices, m);
    sbbf_status st = partition(hashes + off, m, num_blocks, plan.shift, n_slices, ps, true, s);
    if (st != SBBF_OK) return st;
    SBBF_CUDA(cudaMemsetAsync(ps.tiles, 0, 8, s));
    static const cudaError_t attr = cudaFuncSetAttribute(
        unscatter_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(kSmemBudget));
    if (attr != cudaSuccess) return record_cuda(attr);
    sliced_find_kernel<<<plan.grid, 256, 0, s>>>(words, num_blocks, plan.shift, ps.sorted, m,
                                                 ps.offsets, n_slices, ps.tiles, ps.sorted_bits,
                                                 plan.rounds);
    if ((st = launch_status()) != SBBF_OK) return st;
    unscatter_kernel<<<ctas * (ps.rows - 1), kUnscatterThreads, unscatter_smem_bytes(n_slices),
                       s>>>(ps.sorted_bits, ps.idx, ps.marks, m, range_keys(m, ctas), ps.rows,
                            n_slices, d_out + off / 32);
    if ((st = launch_status()) != SBBF_OK) return st;
  }
  return SBBF_OK;
}

}  // namespace sbbf

sbbf_status sbbf_partition_applies(const sbbf_t* f, size_t n, int lookup, int* applies) {
  if (!f || !applies) return SBBF_EINVAL;
  (void)lookup;  // the same rule for inserts and lookups
  *applies = sbbf::want_partition(f, n) ? 1 : 0;
  return SBBF_OK;
}
