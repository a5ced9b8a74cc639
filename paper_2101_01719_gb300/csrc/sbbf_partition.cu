// Block-range partitioned inserts and lookups for filters larger than L2.
//
// A random 32-byte block of a filter far larger than L2 costs a DRAM access
// of at least 64 bytes, and DRAM serves only ~40 G random accesses per
// second, whereas the same block in L2 costs one L1/L2 request.  So for a
// large batch the keys are first grouped by filter slice -- 2^shift
// consecutive blocks, 4 to 32 MiB (see insert_shift, find_plan) -- and then
// processed slice by slice, in order:
//   1. scatter: the keys are split into one contiguous range per CTA (one
//      CTA per SM); each CTA streams its range through shared memory in
//      8192-key tiles (double-buffered bulk copies, cp.async.bulk with an
//      mbarrier, the next tile arriving while the current one is
//      processed), counting-sorts each tile by slice there and appends each
//      slice's run to its bucket for that slice, so consecutive threads write
//      consecutive addresses.  Bucket (q, c) of slice q and CTA c holds
//      positions [(q C + c) cap, (q C + c + 1) cap) of the slice-ordered
//      array (C CTAs), where cap is the expected number of keys of one
//      (slice, CTA) pair plus six standard deviations, so the buckets are
//      placed by formula and no counting pass over the keys precedes the
//      scatter.  Each CTA records how full its buckets are; a CTA whose keys
//      overflow one of its buckets drops the overflow and is marked spilled.
//   2. insert or look up the slice-ordered keys with the in-order dynamic
//      tile schedule, skipping the unfilled end of each bucket; every
//      claimed tile bulk-prefetches into L2 the filter bytes of the keys a
//      slice ahead, so the filter is read from DRAM sequentially and hit in
//      L2 when the keys arrive;
//   3. lookups only: the answers, written in slice order, go back to key
//      order one sub-range of positions at a time, each in shared memory;
//   4. spilled CTAs (an input that crowds one slice far beyond its share;
//      uniformly distributed hashes essentially never do) have their whole
//      key range redone by the random-access path: inserts again (OR is
//      idempotent), lookups rewrite that range's result words.  So every
//      input gives the exact result, and a crowded one only costs time.
// Inserts commute (OR), so the order within a slice does not matter and the
// filter equals the unpartitioned insert bit for bit; lookups keep each key's
// original position (written by the scatter) and answer exactly as the
// unpartitioned lookup.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "sbbf.h"
#include "sbbf_device.cuh"
#include "sbbf_host.cuh"
#include "sbbf_kernels.cuh"

namespace sbbf {

namespace {

constexpr int kMinSliceShift = 17;       // 2^17 blocks (4 MiB) per slice
constexpr int kMaxSliceShift = 20;       // 2^20 blocks (32 MiB) per slice
constexpr uint32_t kTargetSlices = 512;
constexpr uint32_t kMaxSlices = 4096;    // num_blocks < 2^32 at the largest slice
// Ranking by warp match up to this many slices, by one shared atomic per key
// above.  Measured on 1e9 lookups / 100M inserts (16M batches): at 8 slices
// (256 MiB, lookups) 118 G/s with atomics against 107 with matches, at 16
// and 32 slices 120 / 121 against 94 / 84, inserts at 16 and 32 slices 78 /
// 77 against 64 / 59; at 2 and 3 slices matches win (110 / 113 against 88 /
// 109).  An earlier ranking by one ballot per slice ran 49 G/s at 16 slices.
constexpr uint32_t kFewSlices = 4;
constexpr int kPartThreads = 1024;  // one scatter CTA per SM

// Scatter tiles: 12288 keys where the slice tables leave room in shared
// memory (longer runs per slice and a third less per-tile work), else 8192.
// Lookups map answers back to key order by sub-range, a whole number of
// tiles of at most 2^16 keys (16-bit offsets): five tiles of 12288 or eight
// of 8192.
template <uint32_t kT>
struct TileShape {
  static_assert(kT == 8192 || kT == 12288, "the two tile sizes");
  static constexpr uint32_t kPer = kT / kPartThreads;  // keys per thread
  static constexpr uint32_t kSub = kT == 12288 ? 5 * kT : 8 * kT;
  static_assert(kSub <= 65536 && kSub % 32 == 0, "16-bit offsets; whole result words");
};
constexpr uint32_t kMaxSubKeys = 65536;

__device__ __forceinline__ uint32_t slice_of(uint64_t h, uint32_t nb, int shift) {
  return block_of(h, nb) >> shift;
}

__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// Rank of this lane's key among the keys of the same bin (claims ranks from
// the shared counter ranks[p]).  With few bins (kFew) many lanes share a bin:
// the lanes of each distinct bin find one another with one match, and their
// lowest lane claims the group's ranks with one atomic.  With many bins lanes
// rarely collide and count directly.
template <bool kFew>
__device__ __forceinline__ unsigned rank_warp(unsigned* ranks, bool v, uint32_t p) {
  if (kFew) {
    const unsigned m = __match_any_sync(0xFFFFFFFFu, v ? p : 0xFFFFFFFFu);
    const int leader = __ffs(m) - 1;
    unsigned first = 0;
    if (v && lane_id() == static_cast<unsigned>(leader)) first = atomicAdd(&ranks[p], __popc(m));
    first = __shfl_sync(0xFFFFFFFFu, first, leader);
    return v ? first + __popc(m & lanemask_lt()) : 0u;
  }
  return v ? atomicAdd(&ranks[p], 1u) : 0u;
}

// Keys [c * R, min(n, (c + 1) * R)) belong to CTA c of the scatter.  R is a
// multiple of 32: a range starts 16-byte aligned whenever the array does,
// and a lookup's result words split between ranges without sharing a word.
__host__ __device__ __forceinline__ uint64_t range_keys(uint64_t n, uint32_t ctas) {
  const uint64_t r = (n + ctas - 1) / ctas;
  return (r + 31) & ~31ull;
}

// Sub-ranges: sub_keys consecutive positions of a CTA's range.  The scatter
// records its bucket cursors at each sub-range start, so the keys of
// sub-range u of CTA c that fall in slice q sit at sorted positions
// [marks[c][u][q], marks[c][u + 1][q]); a key's original position is then
// stored as its 16-bit offset within its sub-range.
__host__ __device__ __forceinline__ uint32_t sub_ranges(uint64_t range, uint32_t sub_keys) {
  return static_cast<uint32_t>((range + sub_keys - 1) / sub_keys);
}

// Where the slice-ordered keys go: bucket (q, c) -- slice q, scatter CTA c --
// holds positions [base(q, c), base(q, c) + cap); slice q's buckets are
// consecutive, so slice q spans positions [q * slice_positions(), ...).
struct Buckets {
  uint32_t ctas;
  uint32_t n_slices;
  uint64_t cap;  // a multiple of 64, below 2^31
  __host__ __device__ __forceinline__ uint64_t base(uint32_t q, uint32_t c) const {
    return (static_cast<uint64_t>(q) * ctas + c) * cap;
  }
  __host__ __device__ __forceinline__ uint64_t slice_positions() const {
    return static_cast<uint64_t>(ctas) * cap;
  }
  __host__ __device__ __forceinline__ uint64_t positions() const {
    return slice_positions() * n_slices;
  }
};

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

// Waits for the mbarrier phase with the given parity; false after kWaitNs.
// try_wait suspends the thread in hardware for a while when the phase is not
// complete yet, so waiting threads do not take issue slots from the others.
__device__ __forceinline__ bool wait_phase(uint32_t bar, uint32_t parity) {
  const uint64_t t0 = global_ns();
  for (;;) {
    uint32_t done;
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; "
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

// Bits of the device status word the partitioned passes report through
// (sbbf_device_status turns any of them into SBBF_ETIMEOUT).
constexpr unsigned kStatusWaitTimedOut = 1u;  // a bulk-copy wait ran out; plain loads took over
constexpr unsigned kStatusCopyPending = 2u;   // a copy had not landed when the CTA gave up on it

// Thread 0's record of the bulk copies it issued into a CTA's two key
// buffers: which buffer has a copy whose completion no wait has observed
// yet, and the mbarrier phase parity that completion will show.  After a
// timed-out wait the CTA stops using the buffers (plain loads instead), so a
// late copy can only land in a buffer nothing reads; before the CTA exits,
// drain() waits -- again with the time limit -- for every copy still
// outstanding, so that its shared memory is not handed to another CTA while
// a copy may still write it.
struct CopyTrack {
  uint32_t pending = 0, parity = 0;
  __device__ void issued(int buf, uint32_t expected_parity) {
    pending |= 1u << buf;
    parity = (parity & ~(1u << buf)) | (expected_parity << buf);
  }
  __device__ void observed(int buf) { pending &= ~(1u << buf); }
  __device__ void drain(uint32_t bar0, uint32_t bar1, unsigned* status) {
    for (int b = 0; b < 2; ++b)
      if (((pending >> b) & 1) && !wait_phase(b ? bar1 : bar0, (parity >> b) & 1))
        atomicOr(status, kStatusCopyPending);
    pending = 0;
  }
};

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

// ---- 1. scatter -----------------------------------------------------------------

// Shared memory of the scatter: two input tiles, the per-slice bucket
// cursors (i32) and counts / run starts (u32), and the sorted tile as the
// input positions of its keys (u16).
__host__ __device__ constexpr size_t scatter_smem_bytes(uint32_t tile, uint32_t n_slices) {
  return 2ull * 8 * tile + 8ull * n_slices + 2ull * tile;
}

// Keys into slice order.  CTA c streams its range in tiles: each key, read
// once from the input buffer, claims its rank among the tile's keys of its
// slice with one shared atomic (so the counters end as the slice counts),
// the counts are scanned in place into run starts, and the tile's sort is
// recorded as the input position of the key at each sorted slot (16 bits).
// The write pass then walks the sorted slots in order, gathers each key from
// the input buffer and stores it at its bucket's cursor (kept during the tile
// as cursor minus run start, so that a key's slot is one add), consecutive
// threads writing consecutive addresses within each run.  A key past its
// bucket's capacity is dropped and the CTA marked spilled.  Tile t+1 is
// bulk-copied into the other buffer while tile t is processed; the copies
// need a 16-byte aligned key array, and with any other alignment, or if a
// copy ever failed to complete in time, the CTA reads the keys straight from
// global memory instead.  At the end the CTA records each bucket's fill and
// its spill flag.  Lookups (kIndex) also write each key's original position,
// as its 16-bit offset within its sub-range, and the bucket cursors at every
// sub-range start (and after the last tile) to marks[c][u][q], `rows` rows
// per CTA.  CTA 0 also resets the slice pass's tile counter.
template <bool kFew, bool kIndex, uint32_t kT>
__global__ void __launch_bounds__(kPartThreads, 1)
    scatter_kernel(const uint64_t* __restrict__ hashes, uint64_t n, uint32_t nb, int shift,
                   Buckets bk, uint64_t range, uint64_t* __restrict__ out,
                   uint16_t* __restrict__ out_idx, uint32_t* __restrict__ marks, uint32_t rows,
                   uint32_t* __restrict__ fill, uint32_t* __restrict__ spill,
                   unsigned long long* __restrict__ tiles, unsigned* __restrict__ status) {
  constexpr uint32_t kPer = TileShape<kT>::kPer, kSub = TileShape<kT>::kSub;
  extern __shared__ __align__(16) unsigned long long smem[];
  const uint32_t S = bk.n_slices;
  uint64_t* s_buf0 = reinterpret_cast<uint64_t*>(smem);
  uint64_t* s_buf1 = s_buf0 + kT;
  int* s_rel = reinterpret_cast<int*>(s_buf1 + kT);                 // [S] keys in bucket (q, c)
  unsigned* s_cnt = reinterpret_cast<unsigned*>(s_rel + S);         // [S]
  uint16_t* s_perm = reinterpret_cast<uint16_t*>(s_cnt + S);        // [kT]
  __shared__ unsigned warp_sums[32];
  __shared__ __align__(8) unsigned long long s_bar[2];
  __shared__ unsigned s_spill;

  const uint32_t c = blockIdx.x;
  const int cap = static_cast<int>(bk.cap);
  if (c == 0 && threadIdx.x == 0) *tiles = 0;
  const uint64_t a = static_cast<uint64_t>(c) * range;
  const uint64_t b = a < n ? (a + range < n ? a + range : n) : a;
  const uint64_t n_tiles = (b - a + kT - 1) / kT;  // 0 past the keys
  for (uint32_t i = threadIdx.x; i < S; i += blockDim.x) {
    s_rel[i] = 0;
    s_cnt[i] = 0;
  }
  if (threadIdx.x == 0) s_spill = 0;
  bool bulk = (reinterpret_cast<uintptr_t>(hashes) & 15) == 0 && n_tiles > 0;  // CTA-uniform
  const uint32_t bar0 = smem_u32(&s_bar[0]), bar1 = smem_u32(&s_bar[1]);
  if (threadIdx.x == 0 && bulk) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar0) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar1) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  uint32_t parity = 0;  // bit i: phase parity expected next on buffer i
  CopyTrack track;      // thread 0's outstanding copies
  // thread 0 starts the copy of tile t (its even-length head; an odd last
  // key is loaded after the wait)
  auto issue = [&](uint64_t t) {
    const uint64_t t0 = a + t * kT;
    const uint64_t m = b - t0 < kT ? b - t0 : kT;
    const int buf = static_cast<int>(t & 1);
    track.issued(buf, (parity >> buf) & 1);
    bulk_load(buf ? s_buf1 : s_buf0, hashes + t0, static_cast<uint32_t>((m & ~1ull) * 8),
              buf ? bar1 : bar0);
  };
  if (threadIdx.x == 0 && bulk) issue(0);
  const uint64_t pol = policy_evict_first();

  uint32_t* my_marks = kIndex ? marks + static_cast<uint64_t>(c) * rows * S : nullptr;
  for (uint64_t t = 0; t < n_tiles; ++t) {
    const uint64_t t0 = a + t * kT;
    const uint32_t m = static_cast<uint32_t>(b - t0 < kT ? b - t0 : kT);
    const int cur = static_cast<int>(t & 1);
    uint64_t* s_in = cur ? s_buf1 : s_buf0;
    // offset of the tile's first key within its sub-range
    const uint32_t sub_off = static_cast<uint32_t>((t % (kSub / kT)) * kT);
    if (kIndex && sub_off == 0) {  // bucket cursors are true cursors between tiles
      uint32_t* row = my_marks + (t / (kSub / kT)) * S;
      for (uint32_t q = threadIdx.x; q < S; q += blockDim.x)
        row[q] = static_cast<uint32_t>(bk.base(q, c) + (s_rel[q] < cap ? s_rel[q] : cap));
    }
    if (bulk) {
      // the other buffer's last reader finished at the previous tile's end
      if (threadIdx.x == 0 && t + 1 < n_tiles) issue(t + 1);
      // an odd last key lies past the copied span: stored before the barrier
      if ((m & 1) && threadIdx.x == 0) s_in[m - 1] = load_key1(hashes + t0 + m - 1, pol);
      const bool ok = wait_phase(cur ? bar1 : bar0, (parity >> cur) & 1);
      if (ok && threadIdx.x == 0) track.observed(cur);
      parity ^= 1u << cur;
      bulk = __syncthreads_and(ok);  // all threads agree; on failure never use the buffers again
      if (!bulk && threadIdx.x == 0) atomicOr(status, kStatusWaitTimedOut);
    }
    const bool from_smem = bulk;
    // each key claims its rank among the tile's keys of its slice (the
    // counters end as the slice counts); slice and rank stay in registers
    uint32_t qr[kPer];  // slice << 14 | rank (ranks < 12288; slices < 4096)
#pragma unroll
    for (uint32_t i = 0; i < kPer; ++i) {
      const uint32_t j = i * kPartThreads + threadIdx.x;
      const bool v = j < m;
      const uint64_t key = !v ? 0 : from_smem ? s_in[j] : load_key1(hashes + t0 + j, pol);
      const uint32_t q = v ? slice_of(key, nb, shift) : 0u;
      qr[i] = (q << 14) | rank_warp<kFew>(s_cnt, v, q);
    }
    __syncthreads();
    cta_exclusive_scan(s_cnt, S, warp_sums);  // counts -> run starts (ends with a barrier)
    for (uint32_t q = threadIdx.x; q < S; q += blockDim.x) s_rel[q] -= static_cast<int>(s_cnt[q]);
#pragma unroll
    for (uint32_t i = 0; i < kPer; ++i) {
      const uint32_t j = i * kPartThreads + threadIdx.x;
      if (j < m) s_perm[s_cnt[qr[i] >> 14] + (qr[i] & 0x3FFFu)] = static_cast<uint16_t>(j);
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < m; i += blockDim.x) {
      const uint32_t src = s_perm[i];
      const uint64_t key = from_smem ? s_in[src] : load_key1(hashes + t0 + src, pol);
      const uint32_t q = slice_of(key, nb, shift);
      const int rel = s_rel[q] + static_cast<int>(i);  // this key's slot in bucket (q, c)
      if (rel < cap) {
        const uint64_t pos = bk.base(q, c) + static_cast<uint64_t>(rel);
        out[pos] = key;
        if (kIndex) out_idx[pos] = static_cast<uint16_t>(sub_off + src);
      } else {
        s_spill = 1;
      }
    }
    __syncthreads();
    // the cursor advances by the run's length: cursor - start + end
    for (uint32_t q = threadIdx.x; q < S; q += blockDim.x)
      s_rel[q] += static_cast<int>(q + 1 < S ? s_cnt[q + 1] : m);
    __syncthreads();  // every run end is read before the counters are cleared
    for (uint32_t q = threadIdx.x; q < S; q += blockDim.x) s_cnt[q] = 0;
    __syncthreads();
  }
  if (kIndex) {
    uint32_t* row = my_marks + static_cast<uint64_t>(sub_ranges(b - a, kSub)) * S;
    for (uint32_t q = threadIdx.x; q < S; q += blockDim.x)
      row[q] = static_cast<uint32_t>(bk.base(q, c) + (s_rel[q] < cap ? s_rel[q] : cap));
  }
  for (uint32_t q = threadIdx.x; q < S; q += blockDim.x)
    fill[static_cast<uint64_t>(c) * S + q] = static_cast<uint32_t>(s_rel[q] < cap ? s_rel[q] : cap);
  if (threadIdx.x == 0) {
    spill[c] = s_spill;
    track.drain(bar0, bar1, status);
  }
}

// ---- 2. the slice-ordered passes ---------------------------------------------------

// One past the last key of the 64-position group g: a group lies within one
// bucket (cap is a multiple of 64), whose first fill[c][q] positions hold
// keys.  Group indexes stay below 2^32 (positions below 2^38), so the
// divisions are 32-bit.
__device__ __forceinline__ uint64_t group_end(const Buckets& bk, const uint32_t* __restrict__ fill,
                                              uint64_t g) {
  const uint32_t g32 = static_cast<uint32_t>(g);
  const uint32_t per = static_cast<uint32_t>(bk.cap >> 6);  // groups per bucket
  const uint32_t bucket = g32 / per;                        // q * ctas + c
  const uint32_t o = (g32 - bucket * per) << 6;             // the group's offset in its bucket
  const uint32_t q = bucket / bk.ctas;
  const uint32_t c = bucket - q * bk.ctas;
  const uint32_t f = __ldg(fill + static_cast<uint64_t>(c) * bk.n_slices + q);
  const uint32_t valid = f > o ? (f - o < 64 ? f - o : 64) : 0;
  return (g << 6) + valid;
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

// Streaming prefetch by position.  Slice q holds positions [q P, (q + 1) P)
// (P = bk.slice_positions()) and filter blocks [q << shift, ...); position p
// of slice q is mapped to byte
//   slice_lo + floor((p - q P) * slice_blocks / P) * 32
// so consecutive position ranges map to consecutive, disjoint byte ranges and
// every byte of every slice is covered exactly once.  A warp prefetches the
// bytes of positions [p0, p1) (any number of slices).
__device__ __forceinline__ uint64_t position_byte(uint32_t nb, int shift, uint32_t q, uint64_t P,
                                                  uint64_t p) {
  const uint64_t b0 = static_cast<uint64_t>(q) << shift;
  const uint64_t b1 = b0 + (1ull << shift) < nb ? b0 + (1ull << shift) : nb;
  const uint64_t blocks = b1 - b0;
  // (p - qP) * blocks / P without overflow: split the quotient
  const uint64_t d = p - static_cast<uint64_t>(q) * P;
  const uint64_t blk = (d / P) * blocks + ((d % P) * blocks) / P;
  return 32 * (b0 + blk);
}

__device__ __forceinline__ void prefetch_positions(const uint32_t* words, uint32_t nb, int shift,
                                                   const Buckets& bk, uint64_t p0, uint64_t p1) {
  const uint64_t P = bk.slice_positions(), n = bk.positions();
  if (p0 >= n) return;
  if (p1 > n) p1 = n;
  for (uint64_t q = p0 / P; q < bk.n_slices && q * P < p1; ++q) {
    const uint64_t lo = q * P, hi = lo + P;
    const uint64_t a = p0 > lo ? p0 : lo, b = p1 < hi ? p1 : hi;
    if (a >= b) continue;
    prefetch_bytes(words, position_byte(nb, shift, static_cast<uint32_t>(q), P, a),
                   position_byte(nb, shift, static_cast<uint32_t>(q), P, b));
  }
}

// Distance, in positions, that the streaming prefetch runs ahead of the
// newest claimed tile: one whole slice, so a slice's blocks are all in L2
// before its first key is processed, plus half the window of positions in
// flight, for the prefetches to land.  The L2 footprint is then about one
// slice plus 1.5 windows of filter bytes.
__device__ __forceinline__ uint64_t prefetch_ahead(const Buckets& bk, uint64_t window) {
  return bk.slice_positions() + window / 2;
}

// Rounds of 64-position groups per warp per tile (a launch argument, 1..8;
// even for lookups).  The host picks it from the filter bytes per key: the
// window of keys in flight (CTAs x tile) times that is held near 24 MiB, so
// window and prefetch fit in L2 with a slice; dense batches get long tiles
// (fewer claims of the shared tile counter), sparse ones short tiles.
constexpr int kMaxSlicedRounds = 8;

// Slice-ordered insert with the in-order dynamic tile schedule.  Every tile
// at position a0 prefetches the filter bytes of positions [a0 + ahead,
// a0 + ahead + tile) (see prefetch_ahead), so each block is read from DRAM
// once, sequentially, before its keys arrive.  At launch the CTAs split the
// prefetch of positions [0, ahead).
__global__ void __launch_bounds__(256)
    sliced_insert_kernel(uint32_t* __restrict__ words, uint32_t nb, int shift,
                         const uint64_t* __restrict__ keys, Buckets bk,
                         const uint32_t* __restrict__ fill, unsigned long long* __restrict__ tiles,
                         int rounds) {
  __shared__ unsigned long long s_tile;
  const unsigned wpc = blockDim.x >> 5, wic = threadIdx.x >> 5;
  const uint64_t n_pos = bk.positions(), n_groups = n_pos >> 6;
  const uint64_t groups_per_tile = static_cast<uint64_t>(wpc) * rounds;
  const uint64_t keys_per_tile = groups_per_tile * 64;
  const uint64_t pol = policy_evict_first();
  OneFilter res{nb};
  uint64_t ahead = 0;
  if (wic == 0) {
    ahead = prefetch_ahead(bk, keys_per_tile * gridDim.x);
    const uint64_t share = (ahead + gridDim.x - 1) / gridDim.x;
    prefetch_positions(words, nb, shift, bk, blockIdx.x * share, (blockIdx.x + 1) * share);
  }
  for (;;) {
    if (threadIdx.x == 0) s_tile = atomicAdd(tiles, 1ull);
    __syncthreads();
    const uint64_t g0 = s_tile * groups_per_tile;
    __syncthreads();
    if (g0 >= n_groups) break;
    if (wic == 0)
      prefetch_positions(words, nb, shift, bk, g0 * 64 + ahead, g0 * 64 + ahead + keys_per_tile);
    for (int r = 0; r < rounds; ++r) {
      const uint64_t g = g0 + static_cast<uint64_t>(r) * wpc + wic;
      // the group's keys are loaded whole while its fill is looked up
      if (g < n_groups)
        insert_group8(words, res, HashInput(keys), n_pos, pol, g, group_end(bk, fill, g));
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

// Slice-ordered lookups of the keys at positions [0, bk.positions()), with
// the same schedule and streaming prefetch as the sliced insert; positions
// past a bucket's fill answer 0.  The answers are written in sorted order,
// packed like the unpartitioned lookup's (bit k of the pair of words 2g,
// 2g+1 answers position 64g + k); unscatter_kernel moves them to the keys'
// original positions.
// Groups a lane has in flight per step of the slice pass (two block loads
// each): 2 at four CTAs per SM (4 at two CTAs per SM measured 18% slower).
constexpr int kFindGroups = 2;
constexpr int kFindMinCtas = kFindGroups == 2 ? 4 : 2;

__global__ void __launch_bounds__(256, kFindMinCtas)
    sliced_find_kernel(const uint32_t* __restrict__ words, uint32_t nb, int shift,
                       const uint64_t* __restrict__ keys, Buckets bk,
                       const uint32_t* __restrict__ fill, unsigned long long* __restrict__ tiles,
                       uint32_t* __restrict__ sorted_bits, int rounds) {
  __shared__ unsigned long long s_tile;
  const unsigned wpc = blockDim.x >> 5, wic = threadIdx.x >> 5, lane = lane_id();
  const uint64_t n_pos = bk.positions(), n_groups = n_pos >> 6;
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
    ahead = prefetch_ahead(bk, keys_per_tile * gridDim.x);
    const uint64_t share = (ahead + gridDim.x - 1) / gridDim.x;
    prefetch_positions(words, nb, shift, bk, blockIdx.x * share, (blockIdx.x + 1) * share);
  }
  for (;;) {
    if (threadIdx.x == 0) s_tile = atomicAdd(tiles, 1ull);
    __syncthreads();
    const uint64_t g0 = s_tile * groups_per_tile;
    __syncthreads();
    if (g0 >= n_groups) break;
    if (wic == 0)
      prefetch_positions(words, nb, shift, bk, g0 * 64 + ahead, g0 * 64 + ahead + keys_per_tile);
    // kFindGroups rounds per step: 2 kFindGroups block loads per lane in
    // flight before any test
    for (int r = 0; r < rounds; r += kFindGroups) {
      uint64_t k[kFindGroups], lim[kFindGroups], h[kFindGroups][2];
      uint32_t w[kFindGroups][2][8];
#pragma unroll
      for (int u = 0; u < kFindGroups; ++u) {
        const uint64_t g = g0 + static_cast<uint64_t>(r + u) * wpc + wic;
        k[u] = g * 64 + 2 * lane;
        // the group's keys are loaded whole (every position is readable)
        // while its fill is looked up; keys [64 g, lim) are valid
        HashInput(keys).pair(k[u], n_pos, pk, h[u][0], h[u][1]);
        lim[u] = g < n_groups ? group_end(bk, fill, g) : 0;
      }
#pragma unroll
      for (int u = 0; u < kFindGroups; ++u) {
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          if (k[u] + e < lim[u]) {
            load_block_na(words + 8ull * block_of(h[u][e], nb), pf, w[u][e]);
          } else {
#pragma unroll
            for (int i = 0; i < 8; ++i) w[u][e][i] = 0;
          }
        }
      }
#pragma unroll
      for (int u = 0; u < kFindGroups; ++u) {
        // bit l of b0 / b1: key 2l / 2l + 1 of the group
        const uint32_t b0 = __ballot_sync(
            0xFFFFFFFFu, k[u] < lim[u] && block_has(w[u][0], static_cast<uint32_t>(h[u][0])));
        const uint32_t b1 = __ballot_sync(
            0xFFFFFFFFu,
            k[u] + 1 < lim[u] && block_has(w[u][1], static_cast<uint32_t>(h[u][1])));
        const uint64_t g = g0 + static_cast<uint64_t>(r + u) * wpc + wic;
        if (lane == 0 && g < n_groups)
          *reinterpret_cast<uint2*>(sorted_bits + 2 * g) =
              make_uint2(interleave16(b0 & 0xFFFFu, b1 & 0xFFFFu), interleave16(b0 >> 16, b1 >> 16));
      }
    }
  }
}

// ---- 3. answers back to key order ---------------------------------------------------

// CTA (c, u) owns the original positions [lo, hi): sub-range u of scatter
// CTA c's key range.  The scatter put the keys of that sub-range that fall in
// slice q at sorted positions [marks[c][u][q], marks[c][u + 1][q]).  The CTA
// lists the answer words that overlap these runs (shared memory holds each
// run's bounds and the list offset of its first word); a lane takes one
// word, masks it to its run, and for each found key -- each set bit -- loads
// the key's offset within the sub-range and sets its bit in a shared-memory
// copy of the sub-range's result words, four bits per round so that their
// loads overlap.  The words are then stored whole: every result word belongs
// to exactly one CTA, so there are no global atomics and no zeroing pass.
// Positions and runs are clamped to their buffers (n_pos positions), so keys
// that changed between the passes give wrong answers, never an access out of
// bounds.
constexpr int kUnscatterThreads = 512;

__host__ __device__ constexpr size_t unscatter_smem_bytes(uint32_t n_slices) {
  return 4ull * (kMaxSubKeys / 32) + 4ull * 3 * n_slices;
}

__global__ void __launch_bounds__(kUnscatterThreads)
    unscatter_kernel(const uint32_t* __restrict__ sorted_bits, const uint16_t* __restrict__ idx,
                     const uint32_t* __restrict__ marks, uint64_t n, uint64_t n_pos,
                     uint64_t range, uint32_t sub_keys, uint32_t rows, uint32_t n_slices,
                     uint32_t* __restrict__ out) {
  extern __shared__ __align__(16) uint32_t s_mem[];
  uint32_t* s_out = s_mem;                           // result words of the sub-range
  uint32_t* s_lo = s_out + kMaxSubKeys / 32;         // run q: sorted positions [s_lo, s_hi)
  uint32_t* s_hi = s_lo + n_slices;
  uint32_t* s_item = s_hi + n_slices;                // list offset of run q's first word
  __shared__ unsigned warp_sums[32];
  __shared__ uint32_t s_last;
  const uint32_t subs = rows - 1;
  const uint32_t c = blockIdx.x / subs, u = blockIdx.x % subs;
  const uint64_t a = static_cast<uint64_t>(c) * range;
  const uint64_t end = a + range < n ? a + range : n;
  const uint64_t lo = a + static_cast<uint64_t>(u) * sub_keys;
  if (lo >= end) return;  // the whole CTA
  const uint64_t hi = lo + sub_keys < end ? lo + sub_keys : end;
  const uint32_t span = static_cast<uint32_t>(hi - lo);
  const uint32_t n_words = (span + 31) / 32;
  const uint32_t* m0 = marks + (static_cast<uint64_t>(c) * rows + u) * n_slices;
  const uint32_t* m1 = m0 + n_slices;
  for (uint32_t i = threadIdx.x; i < n_words; i += blockDim.x) s_out[i] = 0;
  for (uint32_t q = threadIdx.x; q < n_slices; q += blockDim.x) {
    const uint32_t p1 = static_cast<uint32_t>(m1[q] < n_pos ? m1[q] : n_pos);
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

// ---- 4. spilled CTAs by the random-access path ----------------------------------

constexpr int kFixupThreads = 256;

// CTA c of the scatter spilled: insert its whole key range [c R, (c+1) R)
// again, one warp per 64 keys (a repeated insert changes nothing).
__global__ void __launch_bounds__(kFixupThreads)
    fixup_insert_kernel(uint32_t* __restrict__ words, uint32_t nb,
                        const uint64_t* __restrict__ hashes, uint64_t n, uint64_t range,
                        const uint32_t* __restrict__ spill) {
  const uint32_t c = blockIdx.x;
  if (spill[c] == 0) return;
  const uint64_t a = static_cast<uint64_t>(c) * range;
  if (a >= n) return;
  const uint64_t m = a + range < n ? range : n - a;
  const uint64_t pol = policy_evict_first();
  OneFilter res{nb};
  const unsigned wpc = blockDim.x >> 5, wic = threadIdx.x >> 5;
  for (uint64_t g = wic; g < (m + 63) / 64; g += wpc)
    insert_group8(words, res, HashInput(hashes + a), m, pol, g);
}

// CTA c of the scatter spilled: answer its whole key range again and rewrite
// the range's result words (a range is a whole number of words).
__global__ void __launch_bounds__(kFixupThreads)
    fixup_find_kernel(const uint32_t* __restrict__ words, uint32_t nb,
                      const uint64_t* __restrict__ hashes, uint64_t n, uint64_t range,
                      const uint32_t* __restrict__ spill, uint32_t* __restrict__ out) {
  const uint32_t c = blockIdx.x;
  if (spill[c] == 0) return;
  const uint64_t a = static_cast<uint64_t>(c) * range;
  if (a >= n) return;
  const uint64_t b = a + range < n ? a + range : n;
  const uint64_t pk = policy_evict_first(), pf = policy_evict_normal();
  const unsigned lane = lane_id(), wpc = blockDim.x >> 5, wic = threadIdx.x >> 5;
  for (uint64_t k0 = a + 32ull * wic; k0 < b; k0 += 32ull * wpc) {
    const uint64_t k = k0 + lane;
    bool hit = false;
    if (k < b) {
      const uint64_t h = load_key1(hashes + k, pk);
      uint32_t w[8];
      load_block_na(words + 8ull * block_of(h, nb), pf, w);
      hit = block_has(w, static_cast<uint32_t>(h));
    }
    const uint32_t bits = __ballot_sync(0xFFFFFFFFu, hit);
    if (lane == 0) out[k0 / 32] = bits;
  }
}

// ---- host side ------------------------------------------------------------------------

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
static_assert(scatter_smem_bytes(8192, kMaxSlices) <= kSmemBudget, "scatter tables fit");

// Scatter tile for n_slices slices: 12288 keys when that fits.
uint32_t scatter_tile(uint32_t n_slices) {
  return scatter_smem_bytes(12288, n_slices) <= kSmemBudget ? 12288u : 8192u;
}

// CTAs of the scatter (one per SM).
uint32_t partition_ctas() { return static_cast<uint32_t>(sm_count()); }

uint32_t slices_at(uint32_t num_blocks, int shift) {
  return static_cast<uint32_t>((static_cast<uint64_t>(num_blocks) + (1ull << shift) - 1) >> shift);
}

// Smallest slice shift lookups may take: 4 MiB, or larger until at most 1024
// slices (the answer pass's per-sub-range runs).
int lookup_min_shift(uint32_t num_blocks) {
  int shift = kMinSliceShift;
  while (shift < kMaxSliceShift && slices_at(num_blocks, shift) > 1024) ++shift;
  return shift;
}

int find_occupancy() {
  static const int occ = occupancy(sliced_find_kernel, 256);
  return occ;
}

// Live-set budget of the slice pass: a slice plus 1.5 windows of filter
// bytes.  Measured: on a 2 GiB filter a 62 MB live set re-read the filter
// (5.85 GB of DRAM reads for 3.5 GB of keys and filter; 46 MB: 4.31 GB),
// which the plans below never approach at that density; on the 32 GiB
// filter with ~1 key per block, 32 MiB slices leave the window room to
// grow only under a larger budget, and 64 MiB (the grid no longer shrunk
// to half) ran lookups at 46.5 against 41.8 G/s with 48, 80 no better.
constexpr double kLiveBytes = 64.0 * 1024 * 1024;

// Batches with fewer keys than blocks (the slice pass streams mostly
// untouched filter bytes) may take 64 MiB slices under a 96 MiB budget:
// measured on 1e9 lookups into the 32 GiB filter (0.93 keys per block) 53.4
// against 51.1 G/s, while denser batches lose with them (2 GiB: 114 against
// 118; 4.1 GB: 109 against 115).
constexpr int kMaxSparseLookupShift = 21;
constexpr double kLiveBytesSparse = 96.0 * 1024 * 1024;

// Slice shift, grid and tile rounds of a partitioned lookup of n keys.  A
// slice's blocks stay in L2 from its prefetch until its last key is
// processed, so a slice plus the keys in flight (and those prefetched ahead)
// must fit there, while the scatter pays for every extra slice (shorter
// runs): lookups take the largest slice (at most 32 MiB, 64 MiB for sparse
// batches; no smaller than lookup_min_shift) within the live-set budget.  When even that slice leaves
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
  const int rounds = sliced_rounds(grid, n, 32ull * num_blocks, kFindGroups);
  const double keys_per_cta = 8.0 * rounds * 64;
  const double window = grid * keys_per_cta * per_key;
  const int floor_shift = lookup_min_shift(num_blocks);
  const bool sparse = n < num_blocks;
  const double live = sparse ? kLiveBytesSparse : kLiveBytes;
  int shift = sparse ? kMaxSparseLookupShift : kMaxSliceShift;
  while (shift > floor_shift && 32.0 * static_cast<double>(1ull << shift) + 1.5 * window > live)
    --shift;
  const double room = (live - 32.0 * static_cast<double>(1ull << shift)) / 1.5;
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
int insert_shift(uint32_t num_blocks) {
  int shift = kMinSliceShift;
  while (shift < kMaxSliceShift && slices_at(num_blocks, shift) > kTargetSlices) ++shift;
  return shift;
}

// Capacity of one bucket: the keys a (slice, CTA) pair expects -- its range
// times the slice's share of the blocks -- plus six standard deviations of
// that binomial count and 64, rounded up to a multiple of 64.  Uniform hashes
// overflow a bucket with probability ~1e-9, and an overflow only sends that
// CTA's range down the random-access path.
uint64_t bucket_cap(uint64_t range, uint32_t num_blocks, int shift) {
  const double share =
      std::fmin(1.0, static_cast<double>(1ull << shift) / static_cast<double>(num_blocks));
  const double e = static_cast<double>(range) * share;
  const uint64_t cap = static_cast<uint64_t>(std::ceil(e + 6.0 * std::sqrt(e) + 64.0));
  return (cap + 63) & ~63ull;
}

// Largest batch a partitioned lookup handles in one piece (32-bit sorted
// positions in the scatter's marks; the padded positions of a piece stay
// below 2^32), and a partitioned insert (32-bit bucket cursors: ranges below
// 2^31 keys).
constexpr uint64_t kMaxIndexedKeys = 1ull << 31;
constexpr uint64_t kMaxInsertKeys = 1ull << 34;

// The geometry of one piece of n keys.
struct Piece {
  int shift;
  uint32_t n_slices;
  uint64_t range;
  Buckets bk;
  uint32_t tile;      // scatter tile, 8192 or 12288 keys
  uint32_t sub_keys;  // lookups: keys per sub-range (a whole number of tiles)
  uint32_t rows;      // lookups: mark rows per CTA (sub-ranges + 1)
  FindPlan plan;      // lookups
};

Piece piece_of(uint32_t num_blocks, uint64_t n, bool lookup) {
  Piece p{};
  const uint32_t ctas = partition_ctas();
  if (lookup) {
    p.plan = find_plan(num_blocks, n);
    p.shift = p.plan.shift;
  } else {
    p.shift = insert_shift(num_blocks);
  }
  p.n_slices = slices_at(num_blocks, p.shift);
  p.range = range_keys(n, ctas);
  p.bk = Buckets{ctas, p.n_slices, bucket_cap(p.range, num_blocks, p.shift)};
  p.tile = scatter_tile(p.n_slices);
  p.sub_keys = p.tile == 12288 ? TileShape<12288>::kSub : TileShape<8192>::kSub;
  p.rows = sub_ranges(p.range, p.sub_keys) + 1;
  return p;
}

uint64_t piece_scratch_bytes(const Piece& p, bool with_index) {
  const uint64_t cells = static_cast<uint64_t>(p.bk.ctas) * p.n_slices;
  const uint64_t pos = p.bk.positions();
  uint64_t bytes = 256 + align256(4 * cells) + align256(4ull * p.bk.ctas) + align256(8 * pos);
  if (with_index)
    bytes += align256(2 * pos) + align256(pos / 8) + align256(4 * cells * p.rows);
  return bytes;
}

struct PartScratch {
  unsigned long long* tiles;  // dynamic-schedule counter of the slice pass
  uint32_t* fill;             // [ctas][n_slices] keys in bucket (q, c)
  uint32_t* spill;            // [ctas] 1: the CTA's range overflowed a bucket
  uint64_t* sorted;           // [positions] slice-ordered keys
  uint16_t* idx;              // [positions] offset of the original position in its sub-range
  uint32_t* sorted_bits;      // [positions / 32] answers in sorted order (lookups)
  uint32_t* marks;            // [ctas][rows][n_slices] sub-range cursors (lookups)
};

PartScratch carve(void* scratch, const Piece& p) {
  PartScratch r;
  char* c = static_cast<char*>(scratch);
  const uint64_t cells = static_cast<uint64_t>(p.bk.ctas) * p.n_slices;
  const uint64_t pos = p.bk.positions();
  r.tiles = reinterpret_cast<unsigned long long*>(c);
  c += 256;
  r.fill = reinterpret_cast<uint32_t*>(c);
  c += align256(4 * cells);
  r.spill = reinterpret_cast<uint32_t*>(c);
  c += align256(4ull * p.bk.ctas);
  r.sorted = reinterpret_cast<uint64_t*>(c);
  c += align256(8 * pos);
  r.idx = reinterpret_cast<uint16_t*>(c);
  c += align256(2 * pos);
  r.sorted_bits = reinterpret_cast<uint32_t*>(c);
  c += align256(pos / 8);
  r.marks = reinterpret_cast<uint32_t*>(c);
  return r;
}

template <bool kFew, bool kIndex, uint32_t kT>
sbbf_status launch_scatter(const uint64_t* hashes, uint64_t n, uint32_t nb, const Piece& p,
                           const PartScratch& ps, unsigned* status, cudaStream_t s) {
  const size_t smem = scatter_smem_bytes(kT, p.n_slices);
  static const cudaError_t attr = [] {
    cudaError_t e = cudaFuncSetAttribute(scatter_kernel<kFew, kIndex, kT>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(kSmemBudget));
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(scatter_kernel<kFew, kIndex, kT>,
                               cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    return e;
  }();
  if (attr != cudaSuccess) return record_cuda(attr);
  scatter_kernel<kFew, kIndex, kT><<<p.bk.ctas, kPartThreads, smem, s>>>(
      hashes, n, nb, p.shift, p.bk, p.range, ps.sorted, kIndex ? ps.idx : nullptr,
      kIndex ? ps.marks : nullptr, p.rows, ps.fill, ps.spill, ps.tiles, status);
  return launch_status();
}

// Step 1: the slice-ordered keys (and positions), bucket fills and spills.
sbbf_status scatter(const uint64_t* hashes, uint64_t n, uint32_t num_blocks, const Piece& p,
                    const PartScratch& ps, bool with_index, unsigned* status, cudaStream_t s) {
  const bool few = p.n_slices <= kFewSlices, big = p.tile == 12288;
  const auto go = [&](auto launch) { return launch(hashes, n, num_blocks, p, ps, status, s); };
  if (with_index) {
    if (few) return big ? go(launch_scatter<true, true, 12288>) : go(launch_scatter<true, true, 8192>);
    return big ? go(launch_scatter<false, true, 12288>) : go(launch_scatter<false, true, 8192>);
  }
  if (few) return big ? go(launch_scatter<true, false, 12288>) : go(launch_scatter<true, false, 8192>);
  return big ? go(launch_scatter<false, false, 12288>) : go(launch_scatter<false, false, 8192>);
}

bool piece_fits(const Piece& p, bool lookup) {
  if (p.n_slices == 0 || p.n_slices > kMaxSlices || p.bk.cap >= (1ull << 31)) return false;
  if ((p.bk.positions() >> 6) >= (1ull << 32)) return false;  // 32-bit group indexes
  return !lookup || p.bk.positions() < (1ull << 32);
}

}  // namespace

// Scratch bytes for a partitioned insert (or, with_index, lookup) of n keys
// into num_blocks blocks, processed in pieces: enough for the largest piece
// (a full piece and the last one can have different geometries).
uint64_t partition_scratch_bytes(uint32_t num_blocks, uint64_t n, bool with_index) {
  const uint64_t max_piece = with_index ? kMaxIndexedKeys : kMaxInsertKeys;
  if (n == 0) return 256;
  const uint64_t full = n < max_piece ? n : max_piece;
  uint64_t bytes = piece_scratch_bytes(piece_of(num_blocks, full, with_index), with_index);
  const uint64_t last = n % max_piece;
  if (n > max_piece && last > 0) {
    const uint64_t b = piece_scratch_bytes(piece_of(num_blocks, last, with_index), with_index);
    if (b > bytes) bytes = b;
  }
  return bytes;
}

// Partitioned insert (see the file comment): scatter, slice-ordered insert
// and the spilled ranges, per piece of at most kMaxInsertKeys keys.
// `scratch` holds at least partition_scratch_bytes(num_blocks, n, false)
// bytes of device memory.
sbbf_status launch_insert_partitioned(uint32_t* words, uint32_t num_blocks, const uint64_t* hashes,
                                      uint64_t n, void* scratch, unsigned* status,
                                      cudaStream_t s) {
  SBBF_TRACE_NAMED("sbbf_partitioned_insert");
  static const int occ_ins = occupancy(sliced_insert_kernel, 256);
  for (uint64_t off = 0; off < n; off += kMaxInsertKeys) {
    const uint64_t m = n - off < kMaxInsertKeys ? n - off : kMaxInsertKeys;
    const Piece p = piece_of(num_blocks, m, false);
    if (!piece_fits(p, false)) return SBBF_EINVAL;
    const PartScratch ps = carve(scratch, p);
    sbbf_status st = scatter(hashes + off, m, num_blocks, p, ps, false, status, s);
    if (st != SBBF_OK) return st;
    const unsigned grid = grid_for(p.bk.positions() / 64, 8, occ_ins);
    const int rounds = sliced_rounds(grid, m, 32ull * num_blocks, 1);
    sliced_insert_kernel<<<grid, 256, 0, s>>>(words, num_blocks, p.shift, ps.sorted, p.bk, ps.fill,
                                              ps.tiles, rounds);
    if ((st = launch_status()) != SBBF_OK) return st;
    fixup_insert_kernel<<<p.bk.ctas, kFixupThreads, 0, s>>>(words, num_blocks, hashes + off, m,
                                                            p.range, ps.spill);
    if ((st = launch_status()) != SBBF_OK) return st;
  }
  return SBBF_OK;
}

// Partitioned lookup of d_hashes[0..n) into the packed bitmask d_out (the
// same bits as the unpartitioned lookup; every word of the answer is
// written): scatter, slice-ordered lookup, answers back to key order and the
// spilled ranges, per piece of at most 2^31 keys (a multiple of 32).
// `scratch` holds at least partition_scratch_bytes(num_blocks, n, true) bytes.
sbbf_status launch_find_partitioned(const uint32_t* words, uint32_t num_blocks,
                                    const uint64_t* hashes, uint64_t n, uint32_t* d_out,
                                    void* scratch, unsigned* status, cudaStream_t s) {
  SBBF_TRACE_NAMED("sbbf_partitioned_find");
  static const cudaError_t attr = cudaFuncSetAttribute(
      unscatter_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(kSmemBudget));
  if (attr != cudaSuccess) return record_cuda(attr);
  for (uint64_t off = 0; off < n; off += kMaxIndexedKeys) {
    const uint64_t m = n - off < kMaxIndexedKeys ? n - off : kMaxIndexedKeys;
    const Piece p = piece_of(num_blocks, m, true);
    if (!piece_fits(p, true)) return SBBF_EINVAL;
    const PartScratch ps = carve(scratch, p);
    sbbf_status st = scatter(hashes + off, m, num_blocks, p, ps, true, status, s);
    if (st != SBBF_OK) return st;
    sliced_find_kernel<<<p.plan.grid, 256, 0, s>>>(words, num_blocks, p.shift, ps.sorted, p.bk,
                                                   ps.fill, ps.tiles, ps.sorted_bits,
                                                   p.plan.rounds);
    if ((st = launch_status()) != SBBF_OK) return st;
    unscatter_kernel<<<p.bk.ctas * (p.rows - 1), kUnscatterThreads,
                       unscatter_smem_bytes(p.n_slices), s>>>(
        ps.sorted_bits, ps.idx, ps.marks, m, p.bk.positions(), p.range, p.sub_keys, p.rows,
        p.n_slices, d_out + off / 32);
    if ((st = launch_status()) != SBBF_OK) return st;
    fixup_find_kernel<<<p.bk.ctas, kFixupThreads, 0, s>>>(words, num_blocks, hashes + off, m,
                                                          p.range, ps.spill, d_out + off / 32);
    if ((st = launch_status()) != SBBF_OK) return st;
  }
  return SBBF_OK;
}

}  // namespace sbbf

sbbf_status sbbf_partition_applies(const sbbf_t* f, size_t n, int lookup, int* applies) {
  if (!f || !applies) return SBBF_EINVAL;
  *applies = sbbf::want_partition(f, n, lookup != 0) ? 1 : 0;
  return SBBF_OK;
}
