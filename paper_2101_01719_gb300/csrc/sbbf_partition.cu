// Block-range partitioned inserts for filters larger than L2.
//
// A random 32-byte block of a filter far larger than L2 costs a DRAM access
// of at least 64 bytes, and DRAM serves only ~40 G random accesses per
// second, whereas the same block in L2 costs one L1/L2 request.  So for a
// large batch the keys are first grouped by filter slice -- 2^20 consecutive
// blocks (32 MiB) -- and then inserted slice by slice, in order:
//   1. count the keys of every slice (per-CTA shared-memory histogram,
//      warp-aggregated with __match_any_sync, then one global add per slice);
//   2. exclusive scan of the counts (one CTA);
//   3. scatter the keys into slice order (per 16384-key tile: count, reserve
//      each slice's run with one global add, place with shared-memory ranks);
//   4. insert the slice-ordered keys with the in-order dynamic tile schedule;
//      the CTA that starts a slice prefetches the next slice into L2 with
//      bulk prefetches, so its blocks are read from DRAM sequentially and hit
//      in L2 when their keys arrive.
// Inserts commute (OR), so the order within a slice does not matter and the
// filter equals the unpartitioned insert bit for bit.
#include <cuda_runtime.h>

#include <cstdint>

#include "sbbf.h"
#include "sbbf_device.cuh"
#include "sbbf_host.cuh"
#include "sbbf_kernels.cuh"

namespace sbbf {
sbbf_status launch_clear(uint32_t* dst, uint64_t n_words, cudaStream_t s);

namespace {

constexpr int kSliceShift = 20;          // 2^20 blocks (32 MiB) per slice
constexpr uint32_t kMaxSlices = 4096;    // num_blocks < 2^32
constexpr uint32_t kFewSlices = 32;      // ballot counting up to this many slices
constexpr int kPartThreads = 512;

__device__ __forceinline__ uint32_t slice_of(uint64_t h, uint32_t nb) {
  return block_of(h, nb) >> kSliceShift;
}

__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// Keys per thread per pass and keys per tile of the scatter (kept in
// registers between the passes).
constexpr int kKeysPerThread = 16;
constexpr uint32_t kTileKeys = kPartThreads * kKeysPerThread;  // 8192

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

// Loads the kKeysPerThread keys of this thread in tile [t0, t1): key i of
// thread x is t0 + 2 * (i / 2) * blockDim + 2 * x + (i % 2), so each load
// instruction reads 16 consecutive bytes per lane.
__device__ __forceinline__ void load_tile_keys(const uint64_t* __restrict__ hashes, uint64_t t0,
                                               uint64_t t1, bool vec, uint64_t pol,
                                               uint64_t h[kKeysPerThread], bool ok[kKeysPerThread]) {
#pragma unroll
  for (int i = 0; i < kKeysPerThread; i += 2) {
    const uint64_t k = t0 + static_cast<uint64_t>(i / 2) * 2 * blockDim.x + 2 * threadIdx.x;
    ok[i] = k < t1;
    ok[i + 1] = k + 1 < t1;
    if (vec && ok[i + 1]) {
      load_keys2(hashes + k, pol, h[i], h[i + 1]);
    } else {
      h[i] = ok[i] ? load_key1(hashes + k, pol) : 0;
      h[i + 1] = ok[i + 1] ? load_key1(hashes + k + 1, pol) : 0;
    }
  }
}

// counts[p] += number of keys in slice p.
template <bool kFew>
__global__ void __launch_bounds__(kPartThreads)
    count_kernel(const uint64_t* __restrict__ hashes, uint64_t n, uint32_t nb, uint32_t n_slices,
                 unsigned long long* __restrict__ counts) {
  extern __shared__ unsigned s_cnt[];
  for (uint32_t i = threadIdx.x; i < n_slices; i += blockDim.x) s_cnt[i] = 0;
  __syncthreads();
  const uint64_t pol = policy_evict_first();
  const bool vec = (reinterpret_cast<uintptr_t>(hashes) & 15) == 0;
  const uint64_t n_tiles = (n + kTileKeys - 1) / kTileKeys;
  for (uint64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
    const uint64_t t0 = tile * kTileKeys, t1 = t0 + kTileKeys < n ? t0 + kTileKeys : n;
    uint64_t h[kKeysPerThread];
    bool ok[kKeysPerThread];
    load_tile_keys(hashes, t0, t1, vec, pol, h, ok);
#pragma unroll
    for (int i = 0; i < kKeysPerThread; ++i)
      count_warp<kFew>(s_cnt, n_slices, ok[i], ok[i] ? slice_of(h[i], nb) : 0u);
  }
  __syncthreads();
  for (uint32_t i = threadIdx.x; i < n_slices; i += blockDim.x)
    if (s_cnt[i]) atomicAdd(&counts[i], static_cast<unsigned long long>(s_cnt[i]));
}

// offsets[0..n_slices] = exclusive scan of counts; cursors = offsets.
__global__ void __launch_bounds__(1024)
    scan_kernel(const unsigned long long* __restrict__ counts, uint32_t n_slices,
                unsigned long long* __restrict__ offsets, unsigned long long* __restrict__ cursors) {
  __shared__ unsigned long long warp_total[32];
  __shared__ unsigned long long carry;
  const unsigned lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (uint32_t start = 0; start < n_slices; start += blockDim.x) {
    const uint32_t t = start + threadIdx.x;
    const unsigned long long v = t < n_slices ? counts[t] : 0ull;
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
      cursors[t] = before;
    }
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) carry += warp_total[31];
    __syncthreads();
  }
  if (threadIdx.x == 0) offsets[n_slices] = carry;
}

// Exclusive scan of vals[0..n) in place over the CTA (n <= 8 * blockDim);
// each thread scans up to 8 consecutive entries, then the per-thread sums
// are scanned with warp shuffles.
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

// Keys into slice order, one tile of kTileKeys at a time: the tile is
// counted per slice, counting-sorted into shared memory, each slice's run is
// reserved in the output with one global add, and the sorted tile is written
// out in order, so consecutive threads write consecutive output positions.
template <bool kFew, bool kIndex>
__global__ void __launch_bounds__(kPartThreads)
    scatter_kernel(const uint64_t* __restrict__ hashes, uint64_t n, uint32_t nb, uint32_t n_slices,
                   unsigned long long* __restrict__ cursors, uint64_t* __restrict__ out,
                   uint32_t* __restrict__ out_idx) {
  extern __shared__ unsigned long long smem[];
  uint64_t* s_keys = reinterpret_cast<uint64_t*>(smem);                      // kTileKeys
  unsigned long long* s_gbase = smem + kTileKeys;                             // n_slices
  unsigned* s_cnt = reinterpret_cast<unsigned*>(s_gbase + n_slices);          // n_slices
  unsigned* s_off = s_cnt + n_slices;                                         // n_slices
  unsigned* s_idx = s_off + n_slices;  // kTileKeys original positions (kIndex)
  __shared__ unsigned warp_sums[32];
  const uint64_t pol = policy_evict_first();
  const bool vec = (reinterpret_cast<uintptr_t>(hashes) & 15) == 0;
  const uint64_t n_tiles = (n + kTileKeys - 1) / kTileKeys;
  for (uint64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
    const uint64_t t0 = tile * kTileKeys, t1 = t0 + kTileKeys < n ? t0 + kTileKeys : n;
    const uint32_t m = static_cast<uint32_t>(t1 - t0);
    for (uint32_t i = threadIdx.x; i < n_slices; i += blockDim.x) s_cnt[i] = 0;
    __syncthreads();
    uint64_t h[kKeysPerThread];
    bool ok[kKeysPerThread];
    uint32_t p[kKeysPerThread];
    load_tile_keys(hashes, t0, t1, vec, pol, h, ok);
#pragma unroll
    for (int i = 0; i < kKeysPerThread; ++i) {
      p[i] = ok[i] ? slice_of(h[i], nb) : 0u;
      count_warp<kFew>(s_cnt, n_slices, ok[i], p[i]);
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < n_slices; i += blockDim.x) {
      const unsigned c = s_cnt[i];
      s_off[i] = c;
      if (c) s_gbase[i] = atomicAdd(&cursors[i], static_cast<unsigned long long>(c));
    }
    __syncthreads();
    cta_exclusive_scan(s_off, n_slices, warp_sums);  // local run starts (ends with a barrier)
    for (uint32_t i = threadIdx.x; i < n_slices; i += blockDim.x) s_cnt[i] = 0;
    __syncthreads();
#pragma unroll
    for (int i = 0; i < kKeysPerThread; ++i) {
      const unsigned r = rank_warp<kFew>(s_cnt, n_slices, ok[i], p[i]);
      if (ok[i]) {
        s_keys[s_off[p[i]] + r] = h[i];
        if (kIndex)  // tile position of key i of this thread (see load_tile_keys)
          s_idx[s_off[p[i]] + r] = (i / 2) * 2 * blockDim.x + 2 * threadIdx.x + (i % 2);
      }
    }
    __syncthreads();
    for (uint32_t j = threadIdx.x; j < m; j += blockDim.x) {
      const uint64_t key = s_keys[j];
      const uint32_t q = slice_of(key, nb);
      const unsigned long long pos = s_gbase[q] + (j - s_off[q]);
      if (pos < n) {  // in range unless the input changed between the passes
        out[pos] = key;
        if (kIndex) out_idx[pos] = static_cast<uint32_t>(t0 + s_idx[j]);
      }
    }
    __syncthreads();
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

// Byte range [lo, hi) of slice s, or an empty range past the filter.
__device__ __forceinline__ void slice_bytes(uint32_t nb, uint32_t s, uint64_t& lo, uint64_t& hi) {
  const uint64_t first = static_cast<uint64_t>(s) << kSliceShift;
  const uint64_t end = first + (1ull << kSliceShift) < nb ? first + (1ull << kSliceShift) : nb;
  lo = first < nb ? first * 32 : 0;
  hi = first < nb ? end * 32 : 0;
}

// Part `part` of `parts` equal parts (32-byte aligned) of [lo, hi).
__device__ __forceinline__ void share(uint64_t lo, uint64_t hi, uint64_t part, uint64_t parts,
                                      uint64_t& a, uint64_t& b) {
  const uint64_t blocks = (hi - lo) / 32;
  const uint64_t per = (blocks + parts - 1) / parts;
  a = lo + 32 * (part * per < blocks ? part * per : blocks);
  b = lo + 32 * ((part + 1) * per < blocks ? (part + 1) * per : blocks);
}

// Slice-ordered insert with the in-order dynamic tile schedule (tiles of
// kTileRounds x warps-per-CTA 64-key groups).  The L2 prefetch of the next
// slice is spread over the current slice's tiles: tile i of the T tiles
// covering slice q prefetches part i of T of slice q + 1, so every SM's bulk
// prefetch unit takes a share and the next slice is in L2 when its keys
// start.  At launch every CTA prefetches its share of slice 0.
__global__ void __launch_bounds__(256)
    sliced_insert_kernel(uint32_t* __restrict__ words, uint32_t nb,
                         const uint64_t* __restrict__ keys, uint64_t n,
                         const unsigned long long* __restrict__ offsets, uint32_t n_slices,
                         unsigned long long* __restrict__ tiles) {
  __shared__ unsigned long long s_tile;
  const unsigned wpc = blockDim.x >> 5, wic = threadIdx.x >> 5;
  const uint64_t n_groups = (n + 63) >> 6;
  const uint64_t groups_per_tile = static_cast<uint64_t>(wpc) * kTileRounds;
  const uint64_t keys_per_tile = groups_per_tile * 64;
  const uint64_t pol = policy_evict_first();
  OneFilter res{nb};
  if (wic == 0) {
    uint64_t lo, hi, a, b;
    slice_bytes(nb, 0, lo, hi);
    share(lo, hi, blockIdx.x, gridDim.x, a, b);
    prefetch_bytes(words, a, b);
  }
  for (;;) {
    if (threadIdx.x == 0) s_tile = atomicAdd(tiles, 1ull);
    __syncthreads();
    const uint64_t g0 = s_tile * groups_per_tile;
    __syncthreads();
    if (g0 >= n_groups) break;
    if (wic == 0) {
      const uint64_t a0 = g0 * 64;
      uint32_t lo = 0, hi = n_slices;  // last q with offsets[q] <= a0
      while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (offsets[mid] <= a0) lo = mid; else hi = mid;
      }
      const uint64_t q_first = offsets[lo], q_end = offsets[lo + 1];
      const uint64_t n_tiles_q = (q_end - q_first + keys_per_tile - 1) / keys_per_tile;
      if (n_tiles_q > 0 && lo + 1 < n_slices) {
        uint64_t s_lo, s_hi, a, b;
        slice_bytes(nb, lo + 1, s_lo, s_hi);
        const uint64_t i = (a0 - q_first) / keys_per_tile;
        share(s_lo, s_hi, i < n_tiles_q ? i : n_tiles_q - 1, n_tiles_q, a, b);
        prefetch_bytes(words, a, b);
      }
    }
    for (int r = 0; r < kTileRounds; ++r) {
      const uint64_t g = g0 + static_cast<uint64_t>(r) * wpc + wic;
      if (g < n_groups) insert_group8(words, res, HashInput(keys), n, pol, g);
    }
  }
}

// Slice-ordered lookups of keys[0..n) (original positions idx[]), with the
// same tile schedule and distributed prefetch as the sliced insert.  A key
// found in the filter sets bit idx of `out` (zeroed beforehand) with one
// atomicOr; misses write nothing.
__global__ void __launch_bounds__(256)
    sliced_find_kernel(const uint32_t* __restrict__ words, uint32_t nb,
                       const uint64_t* __restrict__ keys, const uint32_t* __restrict__ idx,
                       uint64_t n, const unsigned long long* __restrict__ offsets,
                       uint32_t n_slices, unsigned long long* __restrict__ tiles,
                       uint32_t* __restrict__ out) {
  __shared__ unsigned long long s_tile;
  const unsigned wpc = blockDim.x >> 5, wic = threadIdx.x >> 5, lane = lane_id();
  const uint64_t n_groups = (n + 63) >> 6;
  const uint64_t groups_per_tile = static_cast<uint64_t>(wpc) * kTileRounds;
  const uint64_t keys_per_tile = groups_per_tile * 64;
  const uint64_t pk = policy_evict_first();
  const uint64_t pf = policy_evict_last();
  if (wic == 0) {
    uint64_t lo, hi, a, b;
    slice_bytes(nb, 0, lo, hi);
    share(lo, hi, blockIdx.x, gridDim.x, a, b);
    prefetch_bytes(words, a, b);
  }
  for (;;) {
    if (threadIdx.x == 0) s_tile = atomicAdd(tiles, 1ull);
    __syncthreads();
    const uint64_t g0 = s_tile * groups_per_tile;
    __syncthreads();
    if (g0 >= n_groups) break;
    if (wic == 0) {
      const uint64_t a0 = g0 * 64;
      uint32_t lo = 0, hi = n_slices;  // last q with offsets[q] <= a0
      while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (offsets[mid] <= a0) lo = mid; else hi = mid;
      }
      const uint64_t q_first = offsets[lo], q_end = offsets[lo + 1];
      const uint64_t n_tiles_q = (q_end - q_first + keys_per_tile - 1) / keys_per_tile;
      if (n_tiles_q > 0 && lo + 1 < n_slices) {
        uint64_t s_lo, s_hi, a, b;
        slice_bytes(nb, lo + 1, s_lo, s_hi);
        const uint64_t i = (a0 - q_first) / keys_per_tile;
        share(s_lo, s_hi, i < n_tiles_q ? i : n_tiles_q - 1, n_tiles_q, a, b);
        prefetch_bytes(words, a, b);
      }
    }
    for (int r = 0; r < kTileRounds; ++r) {
      const uint64_t g = g0 + static_cast<uint64_t>(r) * wpc + wic;
      if (g >= n_groups) continue;
      const uint64_t k = g * 64 + 2 * lane;
      uint64_t h0, h1;
      HashInput(keys).pair(k, n, pk, h0, h1);
      uint32_t w0[8], w1[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) w0[i] = w1[i] = 0;
      if (k < n) load_block_na(words + 8ull * block_of(h0, nb), pf, w0);
      if (k + 1 < n) load_block_na(words + 8ull * block_of(h1, nb), pf, w1);
      if (k < n && block_has(w0, static_cast<uint32_t>(h0))) {
        const uint32_t j = idx[k];
        atomicOr(out + (j >> 5), 1u << (j & 31));
      }
      if (k + 1 < n && block_has(w1, static_cast<uint32_t>(h1))) {
        const uint32_t j = idx[k + 1];
        atomicOr(out + (j >> 5), 1u << (j & 31));
      }
    }
  }
}

inline uint64_t align256(uint64_t x) { return (x + 255) & ~255ull; }

}  // namespace

// Scratch bytes for a partitioned insert (or, with_index, lookup) of n keys
// into num_blocks blocks.
uint64_t partition_scratch_bytes(uint32_t num_blocks, uint64_t n, bool with_index) {
  const uint64_t s = (static_cast<uint64_t>(num_blocks) + (1ull << kSliceShift) - 1) >> kSliceShift;
  return 3 * align256(8 * (s + 1)) + 256 + align256(8 * n) + (with_index ? align256(4 * n) : 0);
}

// Largest batch a partitioned lookup handles in one pass (32-bit positions).
constexpr uint64_t kMaxIndexedKeys = 1ull << 31;

namespace {

struct PartScratch {
  unsigned long long *counts, *offsets, *cursors, *tiles;
  uint64_t* sorted;
  uint32_t* idx;
};

PartScratch carve(void* scratch, uint32_t n_slices, uint64_t n) {
  PartScratch r;
  char* p = static_cast<char*>(scratch);
  r.counts = reinterpret_cast<unsigned long long*>(p);
  p += align256(8 * (n_slices + 1));
  r.offsets = reinterpret_cast<unsigned long long*>(p);
  p += align256(8 * (n_slices + 1));
  r.cursors = reinterpret_cast<unsigned long long*>(p);
  p += align256(8 * (n_slices + 1));
  r.tiles = reinterpret_cast<unsigned long long*>(p);
  p += 256;
  r.sorted = reinterpret_cast<uint64_t*>(p);
  p += align256(8 * n);
  r.idx = reinterpret_cast<uint32_t*>(p);
  return r;
}

// Steps 1-3: counts, offsets and the slice-ordered keys (and positions).
sbbf_status partition(const uint64_t* hashes, uint64_t n, uint32_t num_blocks, uint32_t n_slices,
                      const PartScratch& ps, bool with_index, cudaStream_t s) {
  SBBF_CUDA(cudaMemsetAsync(ps.counts, 0, 8ull * n_slices, s));
  const bool few = n_slices <= kFewSlices;
  const uint64_t tiles_n = (n + kTileKeys - 1) / kTileKeys;
  const size_t count_smem = 4ull * n_slices;
  const size_t scatter_smem = 8ull * kTileKeys + 16ull * n_slices + (with_index ? 4ull * kTileKeys : 0);
  const size_t max_smem = 12ull * kTileKeys + 16ull * kMaxSlices;
  static const bool smem_set = [max_smem] {
    cudaFuncSetAttribute(scatter_kernel<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         static_cast<int>(max_smem));
    cudaFuncSetAttribute(scatter_kernel<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         static_cast<int>(max_smem));
    cudaFuncSetAttribute(scatter_kernel<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         static_cast<int>(max_smem));
    cudaFuncSetAttribute(scatter_kernel<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         static_cast<int>(max_smem));
    return true;
  }();
  (void)smem_set;
  static int occ_count_few = occupancy(count_kernel<true>, kPartThreads, 4 * kFewSlices);
  static int occ_count_many = occupancy(count_kernel<false>, kPartThreads, 4 * kMaxSlices);
  static int occ_scatter = occupancy(scatter_kernel<false, true>, kPartThreads, max_smem);
  if (few)
    count_kernel<true><<<grid_for(tiles_n, 1, occ_count_few), kPartThreads, count_smem, s>>>(
        hashes, n, num_blocks, n_slices, ps.counts);
  else
    count_kernel<false><<<grid_for(tiles_n, 1, occ_count_many), kPartThreads, count_smem, s>>>(
        hashes, n, num_blocks, n_slices, ps.counts);
  sbbf_status st = launch_status();
  if (st != SBBF_OK) return st;
  scan_kernel<<<1, 1024, 0, s>>>(ps.counts, n_slices, ps.offsets, ps.cursors);
  if ((st = launch_status()) != SBBF_OK) return st;
  const unsigned grid = grid_for(tiles_n, 1, occ_scatter);
  if (few && with_index)
    scatter_kernel<true, true><<<grid, kPartThreads, scatter_smem, s>>>(
        hashes, n, num_blocks, n_slices, ps.cursors, ps.sorted, ps.idx);
  else if (few)
    scatter_kernel<true, false><<<grid, kPartThreads, scatter_smem, s>>>(
        hashes, n, num_blocks, n_slices, ps.cursors, ps.sorted, nullptr);
  else if (with_index)
    scatter_kernel<false, true><<<grid, kPartThreads, scatter_smem, s>>>(
        hashes, n, num_blocks, n_slices, ps.cursors, ps.sorted, ps.idx);
  else
    scatter_kernel<false, false><<<grid, kPartThreads, scatter_smem, s>>>(
        hashes, n, num_blocks, n_slices, ps.cursors, ps.sorted, nullptr);
  return launch_status();
}

uint32_t slices_of(uint32_t num_blocks) {
  return static_cast<uint32_t>((static_cast<uint64_t>(num_blocks) + (1ull << kSliceShift) - 1) >>
                               kSliceShift);
}

}  // namespace

// Partitioned insert (see the file comment).  `scratch` holds at least
// partition_scratch_bytes(num_blocks, n, false) bytes of device memory.
sbbf_status launch_insert_partitioned(uint32_t* words, uint32_t num_blocks, const uint64_t* hashes,
                                      uint64_t n, void* scratch, cudaStream_t s) {
  if (n == 0) return SBBF_OK;
  const uint32_t n_slices = slices_of(num_blocks);
  if (n_slices == 0 || n_slices > kMaxSlices) return SBBF_EINVAL;
  const PartScratch ps = carve(scratch, n_slices, n);
  sbbf_status st = partition(hashes, n, num_blocks, n_slices, ps, false, s);
  if (st != SBBF_OK) return st;
  SBBF_CUDA(cudaMemsetAsync(ps.tiles, 0, 8, s));
  static int occ_ins = occupancy(sliced_insert_kernel, 256);
  sliced_insert_kernel<<<grid_for((n + 63) / 64, 8, occ_ins), 256, 0, s>>>(
      words, num_blocks, ps.sorted, n, ps.offsets, n_slices, ps.tiles);
  return launch_status();
}

// Partitioned lookup of d_hashes[0..n) into the packed bitmask d_out (the
// same bits as the unpartitioned lookup).  `scratch` holds at least
// partition_scratch_bytes(num_blocks, min(n, 2^31), true) bytes; batches
// larger than 2^31 keys run in pieces of 2^31 (a multiple of 32).
sbbf_status launch_find_partitioned(const uint32_t* words, uint32_t num_blocks,
                                    const uint64_t* hashes, uint64_t n, uint32_t* d_out,
                                    void* scratch, cudaStream_t s) {
  if (n == 0) return SBBF_OK;
  const uint32_t n_slices = slices_of(num_blocks);
  if (n_slices == 0 || n_slices > kMaxSlices) return SBBF_EINVAL;
  for (uint64_t off = 0; off < n; off += kMaxIndexedKeys) {
    const uint64_t m = n - off < kMaxIndexedKeys ? n - off : kMaxIndexedKeys;
    const PartScratch ps = carve(scratch, n_slices, m);
    sbbf_status st = partition(hashes + off, m, num_blocks, n_slices, ps, true, s);
    if (st != SBBF_OK) return st;
    uint32_t* out = d_out + off / 32;
    SBBF_CUDA(cudaMemsetAsync(out, 0, 4 * ((m + 31) / 32), s));
    SBBF_CUDA(cudaMemsetAsync(ps.tiles, 0, 8, s));
    static int occ_find = occupancy(sliced_find_kernel, 256);
    sliced_find_kernel<<<grid_for((m + 63) / 64, 8, occ_find), 256, 0, s>>>(
        words, num_blocks, ps.sorted, ps.idx, m, ps.offsets, n_slices, ps.tiles, out);
    st = launch_status();
    if (st != SBBF_OK) return st;
  }
  return SBBF_OK;
}

}  // namespace sbbf
