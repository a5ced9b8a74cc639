// Insert and lookup kernels, generic over how a key finds its block.
//
// A "resolver" maps key k with hash h to a global block index in the word
// arena (or kNoBlock64 to skip the key):
//   OneFilter    one filter of num_blocks blocks at block 0 (appendix
//                block_index);
//   Segments     several filters in one arena; keys grouped by filter,
//                filter t owning keys [offsets[t], offsets[t+1]);
//   Tagged       several filters; key k names its filter in ids[k];
//   RegionFilter one filter restricted to the blocks [lo, hi): keys whose
//                block lies outside are skipped (one pass of a region-pass
//                insert).
// For several filters, filter t is the plain filter of dir[t].num_blocks
// blocks whose block 0 is arena block dir[t].base, so every filter keeps the
// paper's block selection and mask.
//
// A key source S (sbbf_keys.cuh) yields each key's 64-bit hash: the caller's
// hashes (the paper's input) or raw keys hashed in the same pass.
//
// Warp work unit: 64 consecutive keys, two per lane (one 16-byte load when
// the hash array is 16-byte aligned).
//
// Insert, 8 lanes per key (kLanes8): in 16 rounds each group of eight lanes
// takes one key; lane j ORs lane j's mask bit into word j of the block with
// red.or.b32, so one warp instruction covers four whole 32-byte sectors.
// Insert, 1 lane per key: each lane issues four red.or.b64 for its own key.
//
// Lookup, 1 lane per key: one 256-bit load per key, all eight lanes tested
// in registers, 64 answers packed by two OR reductions; U 64-key groups in
// flight per warp.  Lookup, 8 lanes per key: lane j loads word j of the
// block; a ballot gathers the eight tests.
#pragma once

#include <cstdint>

#include "sbbf_device.cuh"
#include "sbbf_keys.cuh"

namespace sbbf {

constexpr uint64_t kNoBlock64 = ~0ull;
constexpr int kMaxThreads = 512;

// Directory entry of one filter in an arena (16 bytes).
struct FilterRef {
  uint64_t base;        // first block of the filter in the arena
  uint32_t num_blocks;  // blocks of the filter (>= 1)
  uint32_t reserved;
};

__device__ __forceinline__ FilterRef load_ref(const FilterRef* dir, uint32_t t) {
  const uint4 v = __ldg(reinterpret_cast<const uint4*>(dir) + t);
  FilterRef r;
  r.base = (static_cast<uint64_t>(v.y) << 32) | v.x;
  r.num_blocks = v.z;
  r.reserved = v.w;
  return r;
}

struct OneFilter {
  static constexpr int kMinBlocks = 3;
  uint32_t num_blocks;
  __device__ __forceinline__ void begin_chunk(uint64_t) {}
  __device__ __forceinline__ uint64_t block(uint64_t, uint64_t h) const {
    return block_of(h, num_blocks);
  }
  __device__ __forceinline__ void finish() const {}
};

struct RegionFilter {
  static constexpr int kMinBlocks = 3;
  uint32_t num_blocks;
  uint32_t lo, hi;
  __device__ __forceinline__ void begin_chunk(uint64_t) {}
  __device__ __forceinline__ uint64_t block(uint64_t, uint64_t h) const {
    const uint32_t b = block_of(h, num_blocks);
    return b - lo < hi - lo ? static_cast<uint64_t>(b) : kNoBlock64;
  }
  __device__ __forceinline__ void finish() const {}
};

struct Segments {
  static constexpr int kMinBlocks = 2;
  const uint64_t* offsets;  // n_filters + 1 non-decreasing key offsets
  const FilterRef* dir;
  uint32_t n_filters;
  // Cached per warp (all lanes hold the same values): the filter of the
  // current chunk's first key, its key range and its directory entry.
  uint32_t t0;
  uint64_t seg_lo, seg_hi;
  FilterRef ref0;

  // Makes t0 the last t with offsets[t] <= k (k < offsets[n_filters]).
  // Chunks mostly stay in the same segment or move forward, so the cached
  // range usually answers without any memory access.  The cache is valid
  // when seg_lo < seg_hi (a found segment always contains its key).
  __device__ __forceinline__ void begin_chunk(uint64_t k) {
    if (k >= seg_lo && k < seg_hi) return;
    uint32_t lo = 0, hi = n_filters;  // invariant: offsets[lo] <= k < offsets[hi]
    bool found = false;
    if (seg_lo < seg_hi && k >= seg_hi) {
      lo = t0 + 1;  // offsets[t0 + 1] = seg_hi <= k
      found = lo + 1 >= n_filters || __ldg(offsets + lo + 1) > k;  // the next segment
    }
    if (!found) {
      while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (__ldg(offsets + mid) <= k) lo = mid; else hi = mid;
      }
    }
    t0 = lo;
    seg_lo = __ldg(offsets + t0);
    seg_hi = __ldg(offsets + t0 + 1);
    ref0 = load_ref(dir, t0);
  }
  __device__ __forceinline__ uint64_t block(uint64_t k, uint64_t h) const {
    if (k < seg_hi) return ref0.base + block_of(h, ref0.num_blocks);
    uint32_t t = t0;  // a later segment within this chunk
    while (t + 1 < n_filters && __ldg(offsets + t + 1) <= k) ++t;
    const FilterRef r = load_ref(dir, t);
    return r.base + block_of(h, r.num_blocks);
  }
  __device__ __forceinline__ void finish() const {}
};

struct Tagged {
  static constexpr int kMinBlocks = 3;
  const uint32_t* ids;
  const FilterRef* dir;
  uint32_t n_filters;
  unsigned long long* invalid;  // device count of keys whose id >= n_filters
  uint32_t bad;

  __device__ __forceinline__ void begin_chunk(uint64_t) {}
  __device__ __forceinline__ uint64_t block(uint64_t k, uint64_t h) {
    const uint32_t t = __ldg(ids + k);
    if (t >= n_filters) {
      ++bad;
      return kNoBlock64;
    }
    const FilterRef r = load_ref(dir, t);
    return r.base + block_of(h, r.num_blocks);
  }
  __device__ __forceinline__ void finish() const {
    unsigned long long c = bad;
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xFFFFFFFFu, c, o);
    if (lane_id() == 0 && c) atomicAdd(invalid, c);
  }
};

__device__ __forceinline__ void warp_span(uint64_t& warp, uint64_t& n_warps) {
  warp = (static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  n_warps = (static_cast<uint64_t>(gridDim.x) * blockDim.x) >> 5;
}

// ---- work scheduling -----------------------------------------------------------
//
// A warp processes one "unit" of 64-key groups at a time.  Static schedule
// (tiles == nullptr): warp w takes units w, w + W, w + 2W, ... (W warps in the
// grid).  Dynamic schedule (tiles != nullptr, zeroed before the launch): each
// CTA takes the next tile of kTileRounds x (warps per CTA) consecutive units
// from a global counter, so every CTA works on neighbouring keys in key order.
// Keys grouped by filter then keep only a few filters in flight at any time,
// which keeps them resident in L2 even when the whole arena is not.

constexpr int kTileRounds = 8;

// Every thread of the CTA calls next() until it returns false; in the
// dynamic schedule all threads fetch the same tiles, so the two barriers per
// tile are reached the same number of times by every thread.
struct UnitIter {
  uint64_t n_units;
  unsigned long long* tiles;
  uint64_t pos, step;  // static: next unit and stride; dynamic: tile start
  int round;
  unsigned wpc, wic;

  __device__ __forceinline__ UnitIter(uint64_t n, unsigned long long* t) : n_units(n), tiles(t) {
    wpc = blockDim.x >> 5;
    wic = threadIdx.x >> 5;
    if (tiles == nullptr) {
      warp_span(pos, step);
    } else {
      pos = 0;
      step = static_cast<uint64_t>(wpc) * kTileRounds;
      round = kTileRounds;  // fetch a tile on the first call
    }
  }

  __device__ __forceinline__ bool next(uint64_t& unit) {
    if (tiles == nullptr) {
      if (pos >= n_units) return false;
      unit = pos;
      pos += step;
      return true;
    }
    __shared__ unsigned long long s_tile;
    for (;;) {
      if (round == kTileRounds) {
        if (threadIdx.x == 0) s_tile = atomicAdd(tiles, 1ull);
        __syncthreads();
        pos = s_tile * step;
        __syncthreads();  // all have read s_tile before the next fetch
        if (pos >= n_units) return false;
        round = 0;
      }
      const uint64_t u = pos + static_cast<uint64_t>(round) * wpc + wic;
      ++round;
      if (u < n_units) {
        unit = u;
        return true;
      }
    }
  }
};

// ---- insert ----------------------------------------------------------------

// Inserts the 64-hash group g with eight lanes per key: in 16 rounds each
// group of eight lanes takes one key and lane j ORs lane j's mask bit into
// word j of the key's block.
template <class R, class S>
__device__ __forceinline__ void insert_group8(uint32_t* __restrict__ words, R& res, const S& src,
                                              uint64_t n, uint64_t pol, uint64_t g,
                                              uint64_t lim = ~0ull) {
  const unsigned lane = lane_id();
  const uint32_t seed = lane_seed(lane & 7);
  uint32_t* const word_j = words + (lane & 7);
  const int group_base = static_cast<int>(lane & ~7u);
  const uint64_t k = g * 64 + 2 * lane;
  uint64_t h0, h1;
  src.pair(k, n, pol, h0, h1);  // keys [0, n) are readable; [0, min(n, lim)) are inserted
  res.begin_chunk(g * 64);
  const uint64_t end = n < lim ? n : lim;
  const uint64_t b0 = k < end ? res.block(k, h0) : kNoBlock64;
  const uint64_t b1 = k + 1 < end ? res.block(k + 1, h1) : kNoBlock64;
  const uint32_t x0 = static_cast<uint32_t>(h0), x1 = static_cast<uint32_t>(h1);
#pragma unroll
  for (int r = 0; r < 16; ++r) {
    const int src = group_base + (r >> 1);
    const uint32_t x = __shfl_sync(0xFFFFFFFFu, (r & 1) ? x1 : x0, src);
    const uint64_t b = __shfl_sync(0xFFFFFFFFu, (r & 1) ? b1 : b0, src);
    if (b != kNoBlock64) red_or(word_j + 8ull * b, 1u << bit_index(x, seed));
  }
}

// The same group with one lane per key: four red.or.b64 per key.
template <class R, class S>
__device__ __forceinline__ void insert_group1(uint32_t* __restrict__ words, R& res, const S& src,
                                              uint64_t n, uint64_t pol, uint64_t g) {
  const unsigned lane = lane_id();
  const uint64_t k = g * 64 + 2 * lane;
  uint64_t h0, h1;
  src.pair(k, n, pol, h0, h1);
  res.begin_chunk(g * 64);
  const uint64_t b0 = k < n ? res.block(k, h0) : kNoBlock64;
  const uint64_t b1 = k + 1 < n ? res.block(k + 1, h1) : kNoBlock64;
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    const uint64_t b = s ? b1 : b0;
    const uint32_t x = static_cast<uint32_t>(s ? h1 : h0);
    if (b == kNoBlock64) continue;
    unsigned long long* p = reinterpret_cast<unsigned long long*>(words + 8ull * b);
    red_or64(p + 0, mask_pair(x, SBBF_SEED0, SBBF_SEED1));
    red_or64(p + 1, mask_pair(x, SBBF_SEED2, SBBF_SEED3));
    red_or64(p + 2, mask_pair(x, SBBF_SEED4, SBBF_SEED5));
    red_or64(p + 3, mask_pair(x, SBBF_SEED6, SBBF_SEED7));
  }
}

template <class R, bool kLanes8, class S = HashInput>
__global__ void __launch_bounds__(kMaxThreads)
    insert_kernel(uint32_t* __restrict__ words, R res, S src, uint64_t n,
                  unsigned long long* __restrict__ tiles) {
  const uint64_t n_groups = (n + 63) >> 6;
  const uint64_t pol = policy_evict_first();
  UnitIter it(n_groups, tiles);
  for (uint64_t g; it.next(g);) {
    if (kLanes8) insert_group8(words, res, src, n, pol, g);
    else insert_group1(words, res, src, n, pol, g);
  }
  res.finish();
}

// ---- lookup ----------------------------------------------------------------

// Register budget per shape: one-lane shapes with up to two groups in flight
// are held to R::kMinBlocks 512-thread CTAs per SM (<= 42 registers at 3,
// <= 64 at 2), which keeps occupancy high without spilling; the others may
// use up to 128 registers so that their loads in flight do not spill.
template <class R, class S>
constexpr int find_min_blocks(bool lanes8, int unroll) {
  return (lanes8 || unroll >= 4 || S::kHeavy) ? 1 : R::kMinBlocks;
}

template <class R, bool kLanes8, int U, bool kL1Bypass, class S = HashInput>
__global__ void __launch_bounds__(kMaxThreads, find_min_blocks<R, S>(kLanes8, U))
    find_kernel(const uint32_t* __restrict__ words, R res, S src, uint64_t n,
                uint32_t* __restrict__ out, unsigned long long* __restrict__ tiles) {
  constexpr bool l1_bypass = kL1Bypass;  // block loads skip L1 allocation
  const unsigned lane = lane_id();
  const uint64_t n_groups = (n + 63) >> 6;
  const uint64_t n_out = (n + 31) >> 5;
  const uint64_t pk = policy_evict_first();
  const uint64_t pf = policy_evict_last();
  const bool out16 = (reinterpret_cast<uintptr_t>(out) & 15) == 0;
  const bool out8 = (reinterpret_cast<uintptr_t>(out) & 7) == 0;

  if (!kLanes8) {
    // a unit is U consecutive groups, all loads issued before any test
    const uint64_t n_units = (n_groups + U - 1) / U;
    UnitIter it(n_units, tiles);
    for (uint64_t unit; it.next(unit);) {
      const uint64_t g0 = unit * U;
      uint64_t h[U][2], b[U][2];
#pragma unroll
      for (int u = 0; u < U; ++u)
        src.pair((g0 + u) * 64 + 2 * lane, n, pk, h[u][0], h[u][1]);
#pragma unroll
      for (int u = 0; u < U; ++u) {
        res.begin_chunk((g0 + u) * 64 < n ? (g0 + u) * 64 : 0);
#pragma unroll
        for (int s = 0; s < 2; ++s) {
          const uint64_t k = (g0 + u) * 64 + 2 * lane + s;
          b[u][s] = k < n ? res.block(k, h[u][s]) : kNoBlock64;
        }
      }
      uint32_t w[U][2][8];
#pragma unroll
      for (int u = 0; u < U; ++u) {
#pragma unroll
        for (int s = 0; s < 2; ++s) {
          if (b[u][s] != kNoBlock64) {
            if (l1_bypass) load_block_na(words + 8ull * b[u][s], pf, w[u][s]);
            else load_block(words + 8ull * b[u][s], pf, w[u][s]);
          } else {
#pragma unroll
            for (int i = 0; i < 8; ++i) w[u][s][i] = 0;
          }
        }
      }
      uint32_t lo[U], hi[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const uint32_t r0 = block_has(w[u][0], static_cast<uint32_t>(h[u][0]));
        const uint32_t r1 = block_has(w[u][1], static_cast<uint32_t>(h[u][1]));
        const uint32_t v = (r0 | (r1 << 1)) << (2 * (lane & 15));
        lo[u] = __reduce_or_sync(0xFFFFFFFFu, lane < 16 ? v : 0u);
        hi[u] = __reduce_or_sync(0xFFFFFFFFu, lane >= 16 ? v : 0u);
      }
      store_answers<U>(out, n_out, 2 * g0, lo, hi, lane, out16, out8);
    }
  } else {
    const uint32_t seed = lane_seed(lane & 7);
    const unsigned j = lane & 7;
    const unsigned grp = lane >> 3;
    UnitIter it(n_groups, tiles);
    for (uint64_t g; it.next(g);) {
      const uint64_t k = g * 64 + 2 * lane;
      uint64_t h0, h1;
      src.pair(k, n, pk, h0, h1);
      res.begin_chunk(g * 64);
      const uint64_t b0 = k < n ? res.block(k, h0) : kNoBlock64;
      const uint64_t b1 = k + 1 < n ? res.block(k + 1, h1) : kNoBlock64;
      uint32_t lo = 0, hi = 0;
#pragma unroll 4
      for (int rb = 0; rb < 16; rb += U) {
        uint32_t wv[U], xv[U];
        bool ok[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {  // U rounds of loads in flight
          const int r = rb + u;
          const int src = static_cast<int>(grp * 8) + (r >> 1);
          xv[u] = __shfl_sync(0xFFFFFFFFu, static_cast<uint32_t>((r & 1) ? h1 : h0), src);
          const uint64_t bb = __shfl_sync(0xFFFFFFFFu, (r & 1) ? b1 : b0, src);
          ok[u] = bb != kNoBlock64;
          wv[u] = !ok[u] ? 0u
                  : l1_bypass ? load_word_na(words + 8ull * bb + j, pf)
                              : load_word(words + 8ull * bb + j, pf);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int r = rb + u;
          const bool bit = ok[u] && ((wv[u] >> bit_index(xv[u], seed)) & 1u);
          const uint32_t vote = __ballot_sync(0xFFFFFFFFu, bit);
          // key 16*grp + r: group 0/1 -> word 0 bits r / 16+r, group 2/3 -> word 1
          const uint32_t h_g0 = (vote & 0x000000FFu) == 0x000000FFu;
          const uint32_t h_g1 = (vote & 0x0000FF00u) == 0x0000FF00u;
          const uint32_t h_g2 = (vote & 0x00FF0000u) == 0x00FF0000u;
          const uint32_t h_g3 = (vote & 0xFF000000u) == 0xFF000000u;
          lo |= (h_g0 << r) | (h_g1 << (16 + r));
          hi |= (h_g2 << r) | (h_g3 << (16 + r));
        }
      }
      const uint32_t lo1[1] = {lo}, hi1[1] = {hi};
      store_answers<1>(out, n_out, 2 * g, lo1, hi1, lane, out16, out8);
    }
  }
  res.finish();
}

// ---- region-pass lookup ----------------------------------------------------

// One pass of a region-pass lookup into a one-filter of num_blocks blocks,
// of which `words` holds the blocks from `base` on (kBased: a block-range
// shard; otherwise the whole filter and base is 0 -- a separate instance,
// since the subtraction measured 5% slower for whole filters): the keys whose
// block (the appendix block_index) lies in [lo, hi) are looked up; the others answer 0 in the first pass (kMerge false: every answer word
// is written) and keep their bit in the later passes (kMerge true: the new
// bits are ORed in with fire-and-forget reductions, one per answer word that
// gains a bit).  With the filter split into regions small enough to stay in
// L2, each pass finds its blocks in L2 at the price of reading all the keys.
// Each warp takes units of U 64-key groups by grid stride and loads the next
// unit's hashes (or keys, hashed as they arrive) before it waits on this
// unit's blocks, so the DRAM latency of the key stream and the L2 latency of
// the block loads overlap.
template <int U, bool kMerge, class S = HashInput, bool kBased = false>
__global__ void __launch_bounds__(kMaxThreads)
    region_find_kernel(const uint32_t* __restrict__ words, uint32_t num_blocks, uint32_t base,
                       uint32_t lo, uint32_t hi, S src, uint64_t n,
                       uint32_t* __restrict__ out) {
  const unsigned lane = lane_id();
  const uint64_t n_groups = (n + 63) >> 6;
  const uint64_t n_units = (n_groups + U - 1) / U;
  const uint64_t n_out = (n + 31) >> 5;
  const uint64_t n_warps = (static_cast<uint64_t>(gridDim.x) * blockDim.x) >> 5;
  const uint64_t pk = policy_evict_first();
  const uint64_t pf = policy_evict_last();
  const bool out16 = (reinterpret_cast<uintptr_t>(out) & 15) == 0;
  const bool out8 = (reinterpret_cast<uintptr_t>(out) & 7) == 0;
  const uint32_t span = hi - lo;

  uint64_t unit = (static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  uint64_t h[U][2];
#pragma unroll
  for (int u = 0; u < U; ++u)
    src.pair((unit * U + u) * 64 + 2 * lane, unit < n_units ? n : 0, pk, h[u][0], h[u][1]);
  for (; unit < n_units; unit += n_warps) {
    const uint64_t g0 = unit * U;
    uint32_t b[U][2];
    bool act[U][2];
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
      for (int s = 0; s < 2; ++s) {
        const uint64_t k = (g0 + u) * 64 + 2 * lane + s;
        b[u][s] = block_of(h[u][s], num_blocks);
        act[u][s] = k < n && b[u][s] - lo < span;
      }
    // the blocks of the keys in range (the others' words are never read:
    // their test below is not evaluated)
    uint32_t w[U][2][8];
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
      for (int s = 0; s < 2; ++s)
        if (act[u][s]) load_block_na(words + 8ull * (kBased ? b[u][s] - base : b[u][s]), pf, w[u][s]);
    // the next unit's hashes, in flight while this unit's blocks arrive
    const uint64_t next = unit + n_warps;
    uint64_t hn[U][2];
#pragma unroll
    for (int u = 0; u < U; ++u)
      src.pair((next * U + u) * 64 + 2 * lane, next < n_units ? n : 0, pk, hn[u][0], hn[u][1]);
    uint32_t lo_w[U], hi_w[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const uint32_t r0 = act[u][0] && block_has(w[u][0], static_cast<uint32_t>(h[u][0]));
      const uint32_t r1 = act[u][1] && block_has(w[u][1], static_cast<uint32_t>(h[u][1]));
      const uint32_t v = (r0 | (r1 << 1)) << (2 * (lane & 15));
      lo_w[u] = __reduce_or_sync(0xFFFFFFFFu, lane < 16 ? v : 0u);
      hi_w[u] = __reduce_or_sync(0xFFFFFFFFu, lane >= 16 ? v : 0u);
    }
    if (kMerge) {
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const unsigned l = lane - 2u * u;  // 0: lo_w[u], 1: hi_w[u]
        if (l < 2u) {
          const uint32_t v = l ? hi_w[u] : lo_w[u];
          const uint64_t wd = 2 * (g0 + u) + l;
          if (v && wd < n_out) atomicOr(out + wd, v);
        }
      }
    } else {
      store_answers<U>(out, n_out, 2 * g0, lo_w, hi_w, lane, out16, out8);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      h[u][0] = hn[u][0];
      h[u][1] = hn[u][1];
    }
  }
}

}  // namespace sbbf
