// Four- and sixteen-lane split block filters.  The paper uses eight hash
// functions so that a block's lanes fill one 256-bit SIMD register, and notes
// that four or sixteen would work too.  A K-lane block is K consecutive
// 32-bit words (16 bytes for K = 4, 64 bytes -- two sectors -- for K = 16);
// block selection is the appendix block_index over the filter's K-lane blocks
// and lane i sets bit (s_i * x mod 2^32) >> 27, x the hash's low 32 bits.
// Seeds: K = 4 takes appendix lanes 0..3; K = 16 takes the eight appendix
// seeds and, for lanes 8..15 (the paper names no more), the odd constants
// (splitmix64 output j of seed 0 >> 32) | 1, j = 0..7.
//
// Kernels (one filter, hashes from any key source):
//   insert: K lanes per key, lane j ORs word j of the key's block with one
//     red.or.b32, so one warp instruction covers 32 / K whole blocks;
//   lookup: one lane per key, the block read with one 16-byte load (K = 4) or
//     two 32-byte loads (K = 16), 64 answers per warp packed by OR reductions.
#pragma once

#include <cstdint>

#include "sbbf_device.cuh"
#include "sbbf_host.cuh"
#include "sbbf_kernels.cuh"
#include "sbbf_keys.cuh"

namespace sbbf {

__device__ __forceinline__ uint32_t lane_seed16(int j) {
  switch (j & 15) {
    case 8: return 0xe220a839u;
    case 9: return 0x6e789e6bu;
    case 10: return 0x06c45d19u;
    case 11: return 0xf88bb8a9u;
    case 12: return 0x1b39896bu;
    case 13: return 0x53cb9f0du;
    case 14: return 0x2c829abfu;
    case 15: return 0xc584133bu;
    default: return lane_seed(j);
  }
}

template <int K>
__device__ __forceinline__ bool block_has_k(const uint32_t* w, uint32_t x) {
  uint32_t t = 1;
#pragma unroll
  for (int i = 0; i < K; ++i) t &= w[i] >> bit_index(x, lane_seed16(i));
  return t & 1u;
}

__device__ __forceinline__ void load_block16(const uint32_t* p, uint64_t pol, uint32_t w[4]) {
  asm("ld.global.nc.L2::cache_hint.v4.u32 {%0,%1,%2,%3}, [%4], %5;"
      : "=r"(w[0]), "=r"(w[1]), "=r"(w[2]), "=r"(w[3])
      : "l"(p), "l"(pol));
}

template <int K, class S>
__global__ void __launch_bounds__(256)
    insert_lanes_kernel(uint32_t* __restrict__ words, uint32_t num_blocks, S src, uint64_t n) {
  static_assert(K == 4 || K == 16, "lanes");
  const unsigned lane = lane_id();
  const unsigned j = lane % K;
  const uint32_t seed = lane_seed16(static_cast<int>(j));
  const int group_base = static_cast<int>(lane - j);
  const uint64_t pol = policy_evict_first();
  const uint64_t n_groups = (n + 63) >> 6;
  uint64_t warp, n_warps;
  warp_span(warp, n_warps);
  for (uint64_t g = warp; g < n_groups; g += n_warps) {
    const uint64_t k = g * 64 + 2 * lane;
    uint64_t h0, h1;
    src.pair(k, n, pol, h0, h1);
    const uint32_t b0 = k < n ? block_of(h0, num_blocks) : kNoBlock;
    const uint32_t b1 = k + 1 < n ? block_of(h1, num_blocks) : kNoBlock;
    const uint32_t x0 = static_cast<uint32_t>(h0), x1 = static_cast<uint32_t>(h1);
    // group of K lanes: in 2K rounds it takes both keys of each of its lanes
#pragma unroll 4
    for (int r = 0; r < 2 * K; ++r) {
      const int from = group_base + (r >> 1);
      const uint32_t x = __shfl_sync(0xFFFFFFFFu, (r & 1) ? x1 : x0, from);
      const uint32_t b = __shfl_sync(0xFFFFFFFFu, (r & 1) ? b1 : b0, from);
      if (b != kNoBlock) red_or(words + static_cast<uint64_t>(K) * b + j, 1u << bit_index(x, seed));
    }
  }
}

template <int K, class S>
__global__ void __launch_bounds__(256)
    find_lanes_kernel(const uint32_t* __restrict__ words, uint32_t num_blocks, S src, uint64_t n,
                      uint32_t* __restrict__ out) {
  static_assert(K == 4 || K == 16, "lanes");
  const unsigned lane = lane_id();
  const uint64_t pk = policy_evict_first();
  const uint64_t pf = policy_evict_last();
  const uint64_t n_groups = (n + 63) >> 6;
  const uint64_t n_out = (n + 31) >> 5;
  const bool out8 = (reinterpret_cast<uintptr_t>(out) & 7) == 0;
  uint64_t warp, n_warps;
  warp_span(warp, n_warps);
  for (uint64_t g = warp; g < n_groups; g += n_warps) {
    const uint64_t k = g * 64 + 2 * lane;
    uint64_t h[2];
    src.pair(k, n, pk, h[0], h[1]);
    uint32_t w[2][K];
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      if (k + s < n) {
        const uint32_t* p = words + static_cast<uint64_t>(K) * block_of(h[s], num_blocks);
        if (K == 4) {
          load_block16(p, pf, w[s]);
        } else {
          load_block(p, pf, w[s]);
          load_block(p + 8, pf, w[s] + 8);
        }
      } else {
#pragma unroll
        for (int i = 0; i < K; ++i) w[s][i] = 0;
      }
    }
    const uint32_t r0 = k < n && block_has_k<K>(w[0], static_cast<uint32_t>(h[0]));
    const uint32_t r1 = k + 1 < n && block_has_k<K>(w[1], static_cast<uint32_t>(h[1]));
    const uint32_t v = (r0 | (r1 << 1)) << (2 * (lane & 15));
    const uint32_t lo = __reduce_or_sync(0xFFFFFFFFu, lane < 16 ? v : 0u);
    const uint32_t hi = __reduce_or_sync(0xFFFFFFFFu, lane >= 16 ? v : 0u);
    const uint32_t lo1[1] = {lo}, hi1[1] = {hi};
    store_answers<1>(out, n_out, 2 * g, lo1, hi1, lane, false, out8);
  }
}

// Host launches of the K-lane kernels (K = 4 or 16).
template <class S>
sbbf_status launch_insert_lanes(int lanes, uint32_t* words, uint32_t num_blocks, S src,
                                uint64_t n, cudaStream_t s) {
  if (n == 0) return SBBF_OK;
  auto k = lanes == 4 ? insert_lanes_kernel<4, S> : insert_lanes_kernel<16, S>;
  static int occ4 = occupancy(insert_lanes_kernel<4, S>, 256);
  static int occ16 = occupancy(insert_lanes_kernel<16, S>, 256);
  k<<<grid_for((n + 63) / 64, 8, lanes == 4 ? occ4 : occ16), 256, 0, s>>>(words, num_blocks, src,
                                                                           n);
  return launch_status();
}

template <class S>
sbbf_status launch_find_lanes(int lanes, const uint32_t* words, uint32_t num_blocks, S src,
                              uint64_t n, uint32_t* out, cudaStream_t s) {
  if (n == 0) return SBBF_OK;
  auto k = lanes == 4 ? find_lanes_kernel<4, S> : find_lanes_kernel<16, S>;
  static int occ4 = occupancy(find_lanes_kernel<4, S>, 256);
  static int occ16 = occupancy(find_lanes_kernel<16, S>, 256);
  k<<<grid_for((n + 63) / 64, 8, lanes == 4 ? occ4 : occ16), 256, 0, s>>>(words, num_blocks, src,
                                                                           n, out);
  return launch_status();
}

}  // namespace sbbf
