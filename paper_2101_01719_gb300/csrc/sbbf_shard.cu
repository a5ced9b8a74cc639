// One filter sharded by block range over several devices.
//
// The method maps every key to exactly one block (intro: one block per key,
// appendix block_index), so a filter split into contiguous block ranges is
// the same filter: shard s of G owns global blocks [s P, min(B, (s + 1) P)),
// P = ceil(B / G), and a key belongs to the shard owning its block.  A batch
// is processed as: route (group the hashes by owner, remembering each one's
// position), exchange (an all-to-all of the grouped hashes, done by the
// caller's collective library), the local insert or lookup on the owned
// range (global block index minus the range start), for lookups the reverse
// exchange of the answer words and finally the answers back to query order.
// This file holds the device steps; the exchanges are the caller's.
#include <cuda_runtime.h>

#include <cstdint>

#include "sbbf.h"
#include "sbbf_device.cuh"
#include "sbbf_host.cuh"
#include "sbbf_kernels.cuh"
#include "sbbf_launch.cuh"

namespace sbbf {
namespace {

constexpr uint32_t kMaxShards = 1024;
constexpr int kRouteThreads = 512;
constexpr uint32_t kPadPerm = 0xFFFFFFFFu;  // d_perm value of a padding entry

inline uint32_t shard_blocks(uint32_t num_blocks, uint32_t n_shards) {
  return static_cast<uint32_t>((static_cast<uint64_t>(num_blocks) + n_shards - 1) / n_shards);
}

// A shard's part of a filter: global blocks [lo, hi) stored from block 0 of
// its own words; keys of other shards are skipped (lookups answer 0).
struct ShardFilter {
  static constexpr int kMinBlocks = 3;
  uint32_t num_blocks;  // of the whole filter
  uint32_t lo, hi;
  __device__ __forceinline__ void begin_chunk(uint64_t) {}
  __device__ __forceinline__ uint64_t block(uint64_t, uint64_t h) const {
    const uint32_t b = block_of(h, num_blocks);
    return b >= lo && b < hi ? static_cast<uint64_t>(b - lo) : kNoBlock64;
  }
  __device__ __forceinline__ void finish() const {}
};

__device__ __forceinline__ uint32_t owner_of(uint64_t h, uint32_t num_blocks, uint32_t per_shard) {
  return block_of(h, num_blocks) / per_shard;
}

// Keys [c R, min(n, (c + 1) R)) belong to CTA c of the route passes.
__host__ __device__ __forceinline__ uint64_t route_range(uint64_t n, uint32_t ctas) {
  return (n + ctas - 1) / ctas;
}

// hist[c][g] = keys of CTA c's range owned by shard g.
__global__ void __launch_bounds__(kRouteThreads)
    route_count_kernel(const uint64_t* __restrict__ hashes, uint64_t n, uint32_t nb,
                       uint32_t per_shard, uint32_t G, uint64_t range, unsigned* __restrict__ hist) {
  __shared__ unsigned s_cnt[kMaxShards];
  for (uint32_t g = threadIdx.x; g < G; g += blockDim.x) s_cnt[g] = 0;
  __syncthreads();
  const uint64_t a = static_cast<uint64_t>(blockIdx.x) * range;
  const uint64_t b = a + range < n ? a + range : n;
  const uint64_t pol = policy_evict_first();
  // warp-uniform trip count: every lane takes part in the match, lanes past
  // the range with an owner no shard has
  for (uint64_t k0 = a; k0 < b; k0 += blockDim.x) {
    const uint64_t k = k0 + threadIdx.x;
    const bool v = k < b;
    const uint32_t g = v ? owner_of(load_key1(hashes + k, pol), nb, per_shard) : kMaxShards;
    const unsigned peers = __match_any_sync(0xFFFFFFFFu, g);
    if (v && lane_id() == static_cast<unsigned>(__ffs(peers) - 1))
      atomicAdd(&s_cnt[g], __popc(peers));
  }
  __syncthreads();
  for (uint32_t g = threadIdx.x; g < G; g += blockDim.x)
    hist[static_cast<uint64_t>(blockIdx.x) * G + g] = s_cnt[g];
}

// One CTA, thread g per shard: shard g's total, padded to a multiple of 32
// when `pad`, the exclusive scan of the padded totals into group starts,
// base[c][g] = start of CTA c's keys of shard g, counts[g] = the padded total;
// and the padding entries themselves: a hash of the shard's first block
// (its high word is the smallest x with (x * B) >> 32 = lo) and position
// kPadPerm.
__global__ void __launch_bounds__(kMaxShards)
    route_scan_kernel(const unsigned* __restrict__ hist, uint32_t ctas, uint32_t G, uint32_t nb,
                      uint32_t per_shard, int pad, unsigned long long* __restrict__ base,
                      unsigned long long* __restrict__ counts, uint64_t* __restrict__ routed,
                      uint32_t* __restrict__ perm) {
  __shared__ unsigned long long s_tot[kMaxShards];
  const uint32_t g = threadIdx.x;
  unsigned long long total = 0;
  if (g < G)
    for (uint32_t c = 0; c < ctas; ++c) total += hist[static_cast<uint64_t>(c) * G + g];
  const unsigned long long padded = pad ? (total + 31) & ~31ull : total;
  if (g < kMaxShards) s_tot[g] = g < G ? padded : 0;
  __syncthreads();
  if (g >= G) return;
  unsigned long long start = 0;  // G <= 1024: a plain loop is cheap here
  for (uint32_t i = 0; i < g; ++i) start += s_tot[i];
  unsigned long long run = start;
  for (uint32_t c = 0; c < ctas; ++c) {
    base[static_cast<uint64_t>(c) * G + g] = run;
    run += hist[static_cast<uint64_t>(c) * G + g];
  }
  counts[g] = padded;
  if (padded > total) {
    const uint64_t lo = static_cast<uint64_t>(g) * per_shard;  // < nb: the shard owns keys
    const uint64_t x = ((lo << 32) + nb - 1) / nb;
    for (unsigned long long p = start + total; p < start + padded; ++p) {
      routed[p] = x << 32;
      perm[p] = kPadPerm;
    }
  }
}

// Keys of CTA c's range to their owners' groups: within a warp the lanes
// with the same owner claim consecutive slots with one shared atomic.
__global__ void __launch_bounds__(kRouteThreads)
    route_scatter_kernel(const uint64_t* __restrict__ hashes, uint64_t n, uint32_t nb,
                         uint32_t per_shard, uint32_t G, uint64_t range,
                         const unsigned long long* __restrict__ base,
                         uint64_t* __restrict__ routed, uint32_t* __restrict__ perm) {
  __shared__ unsigned long long s_cur[kMaxShards];
  for (uint32_t g = threadIdx.x; g < G; g += blockDim.x)
    s_cur[g] = base[static_cast<uint64_t>(blockIdx.x) * G + g];
  __syncthreads();
  const uint64_t a = static_cast<uint64_t>(blockIdx.x) * range;
  const uint64_t b = a + range < n ? a + range : n;
  const uint64_t pol = policy_evict_first();
  unsigned lt;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(lt));
  for (uint64_t k0 = a; k0 < b; k0 += blockDim.x) {  // warp-uniform, as in the count
    const uint64_t k = k0 + threadIdx.x;
    const bool v = k < b;
    const uint64_t h = v ? load_key1(hashes + k, pol) : 0;
    const uint32_t g = v ? owner_of(h, nb, per_shard) : kMaxShards;
    const unsigned peers = __match_any_sync(0xFFFFFFFFu, g);
    const int leader = __ffs(peers) - 1;
    unsigned long long first = 0;
    if (v && lane_id() == static_cast<unsigned>(leader)) first = atomicAdd(&s_cur[g], __popc(peers));
    first = __shfl_sync(0xFFFFFFFFu, first, leader);
    if (!v) continue;
    const unsigned long long slot = first + __popc(peers & lt);
    routed[slot] = h;
    perm[slot] = static_cast<uint32_t>(k);
  }
}

// Sets bit perm[i] of out for every set bit i of routed_bits that is not
// padding; out was zeroed on the stream first.
__global__ void unpermute_kernel(const uint32_t* __restrict__ routed_bits,
                                 const uint32_t* __restrict__ perm, uint64_t n_routed, uint64_t n,
                                 uint32_t* __restrict__ out) {
  const uint64_t n_words = (n_routed + 31) / 32;
  for (uint64_t w = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; w < n_words;
       w += static_cast<uint64_t>(gridDim.x) * blockDim.x) {
    uint32_t bits = routed_bits[w];
    if (32 * w + 32 > n_routed) bits &= (1u << (n_routed - 32 * w)) - 1;  // the last word's tail
    while (bits) {
      const uint32_t i = __ffs(bits) - 1;
      bits &= bits - 1;
      const uint32_t p = perm[32 * w + i];
      if (p != kPadPerm && p < n) atomicOr(out + p / 32, 1u << (p % 32));
    }
  }
}

}  // namespace
}  // namespace sbbf

using namespace sbbf;

sbbf_status sbbf_shard_range(uint32_t num_blocks, uint32_t n_shards, uint32_t shard, uint32_t* lo,
                             uint32_t* hi) {
  if (num_blocks == 0 || n_shards == 0 || n_shards > kMaxShards || shard >= n_shards || !lo || !hi)
    return SBBF_EINVAL;
  const uint64_t per = shard_blocks(num_blocks, n_shards);
  const uint64_t a = per * shard, b = a + per;
  *lo = static_cast<uint32_t>(a < num_blocks ? a : num_blocks);
  *hi = static_cast<uint32_t>(b < num_blocks ? b : num_blocks);
  return SBBF_OK;
}

size_t sbbf_shard_routed_capacity(size_t n, uint32_t n_shards, int pad) {
  return n + (pad ? 31ull * n_shards : 0);
}

size_t sbbf_shard_route_scratch_bytes(size_t n, uint32_t n_shards) {
  (void)n;
  const uint64_t cells = static_cast<uint64_t>(sm_count()) * n_shards;
  return static_cast<size_t>(((4 * cells + 255) & ~255ull) + 8 * cells + 256);
}

sbbf_status sbbf_shard_route(const uint64_t* d_hashes, size_t n, uint32_t num_blocks,
                             uint32_t n_shards, int pad, uint64_t* d_routed, uint32_t* d_perm,
                             uint64_t* d_counts, void* d_scratch, size_t scratch_bytes,
                             sbbf_stream_t stream) {
  SBBF_TRACE();
  if (num_blocks == 0 || n_shards == 0 || n_shards > kMaxShards || !d_counts ||
      (n > 0 && (!d_hashes || !d_routed || !d_perm)) || n >= (1ull << 32) ||
      (reinterpret_cast<uintptr_t>(d_hashes) & 7) || (reinterpret_cast<uintptr_t>(d_counts) & 7) ||
      (reinterpret_cast<uintptr_t>(d_scratch) & 7) ||
      scratch_bytes < sbbf_shard_route_scratch_bytes(n, n_shards))
    return SBBF_EINVAL;
  const uint32_t ctas = static_cast<uint32_t>(sm_count());
  const uint64_t range = route_range(n, ctas);
  const uint32_t per = shard_blocks(num_blocks, n_shards);
  const uint64_t cells = static_cast<uint64_t>(ctas) * n_shards;
  auto* hist = static_cast<unsigned*>(d_scratch);
  auto* base = reinterpret_cast<unsigned long long*>(static_cast<char*>(d_scratch) +
                                                    ((4 * cells + 255) & ~255ull));
  route_count_kernel<<<ctas, kRouteThreads, 0, stream>>>(d_hashes, n, num_blocks, per, n_shards,
                                                         range, hist);
  sbbf_status st = launch_status();
  if (st != SBBF_OK) return st;
  route_scan_kernel<<<1, kMaxShards, 0, stream>>>(hist, ctas, n_shards, num_blocks, per, pad, base,
                                                  reinterpret_cast<unsigned long long*>(d_counts),
                                                  d_routed, d_perm);
  if ((st = launch_status()) != SBBF_OK) return st;
  if (n == 0) return SBBF_OK;
  route_scatter_kernel<<<ctas, kRouteThreads, 0, stream>>>(d_hashes, n, num_blocks, per, n_shards,
                                                           range, base, d_routed, d_perm);
  return launch_status();
}

sbbf_status sbbf_shard_insert(sbbf_t* f, uint32_t num_blocks, uint32_t lo, const uint64_t* d_hashes,
                              size_t n, sbbf_stream_t stream) {
  SBBF_TRACE();
  if (!f || f->lanes != 8 || f->device != current_device() || num_blocks == 0 ||
      static_cast<uint64_t>(lo) + f->num_blocks > num_blocks)
    return SBBF_EINVAL;
  if (n == 0) return SBBF_OK;
  if (!d_hashes || (reinterpret_cast<uintptr_t>(d_hashes) & 7)) return SBBF_EINVAL;
  return launch_insert_t(kDefaultInsert, f->words, ShardFilter{num_blocks, lo, lo + f->num_blocks},
                         d_hashes, n, stream);
}

sbbf_status sbbf_shard_find(const sbbf_t* f, uint32_t num_blocks, uint32_t lo,
                            const uint64_t* d_hashes, size_t n, uint32_t* d_out_bits,
                            sbbf_stream_t stream) {
  SBBF_TRACE();
  if (!f || f->lanes != 8 || f->device != current_device() || num_blocks == 0 ||
      static_cast<uint64_t>(lo) + f->num_blocks > num_blocks)
    return SBBF_EINVAL;
  if (n == 0) return SBBF_OK;
  if (!d_hashes || !d_out_bits || (reinterpret_cast<uintptr_t>(d_hashes) & 7) ||
      (reinterpret_cast<uintptr_t>(d_out_bits) & 3))
    return SBBF_EINVAL;
  // a shard somewhat larger than what L2 keeps under random access is looked
  // up in region passes over its block range, as a whole filter would be
  const uint32_t passes = region_passes(f, n, true);
  if (passes > 1)
    return launch_find_regions(f->words, num_blocks, lo, lo, lo + f->num_blocks,
                               HashInput(d_hashes), n, d_out_bits, passes, stream);
  Tuning t = kDefaultFind;
  t.l1_bypass = static_cast<uint64_t>(f->num_blocks) * 32 > kL1BypassBytes;
  return launch_find_t(t, f->words, ShardFilter{num_blocks, lo, lo + f->num_blocks}, d_hashes, n,
                       d_out_bits, stream);
}

sbbf_status sbbf_shard_unpermute(const uint32_t* d_routed_bits, const uint32_t* d_perm,
                                 size_t n_routed, size_t n, uint32_t* d_out_bits,
                                 sbbf_stream_t stream) {
  SBBF_TRACE();
  if ((n_routed > 0 && (!d_routed_bits || !d_perm)) || (n > 0 && !d_out_bits) ||
      (reinterpret_cast<uintptr_t>(d_out_bits) & 3))
    return SBBF_EINVAL;
  if (n > 0) SBBF_CUDA(cudaMemsetAsync(d_out_bits, 0, 4 * ((n + 31) / 32), stream));
  if (n_routed == 0) return SBBF_OK;
  static const int occ = occupancy(unpermute_kernel, 256);
  unpermute_kernel<<<grid_for((n_routed + 31) / 32, 256, occ), 256, 0, stream>>>(
      d_routed_bits, d_perm, n_routed, n, d_out_bits);
  return launch_status();
}
