// Host-side launch of the generic insert / lookup kernels with a tunable
// shape: CTA size, lanes per key (1 or 8) and 64-key groups in flight per
// warp (lookups, 1 lane per key) or rounds in flight (8 lanes per key).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>
#include <mutex>
#include <unordered_map>

#include "sbbf_host.cuh"
#include "sbbf_kernels.cuh"

namespace sbbf {

struct Tuning {
  int threads;    // CTA size: 128, 256 or 512
  int lanes;      // lanes per key: 1 or 8
  int unroll;     // lookups: groups (lanes 1) or rounds (lanes 8) in flight: 1, 2, 4
  int l1_bypass;  // lookups: 1 = block loads do not allocate in L1
};

constexpr Tuning kDefaultFind = {256, 1, 2, 0};
constexpr Tuning kDefaultInsert = {256, 8, 1, 0};

// Filters larger than this get L1-bypassing block loads by default: their
// random blocks almost never hit in L1, and skipping the allocation measured
// 8% more random blocks per second from L2.
constexpr uint64_t kL1BypassBytes = 512 * 1024;

inline bool tuning_valid(const Tuning& t) {
  return (t.threads == 128 || t.threads == 256 || t.threads == 512) &&
         (t.lanes == 1 || t.lanes == 8) && (t.unroll == 1 || t.unroll == 2 || t.unroll == 4) &&
         (t.l1_bypass == 0 || t.l1_bypass == 1);
}

// Resident CTAs per SM for (kernel, CTA size), cached.
inline int cached_occupancy(const void* func, int threads) {
  static std::mutex mu;
  static std::unordered_map<uint64_t, int> cache;
  const uint64_t key = reinterpret_cast<uintptr_t>(func) ^ (static_cast<uint64_t>(threads) << 52);
  std::lock_guard<std::mutex> lock(mu);
  auto it = cache.find(key);
  if (it != cache.end()) return it->second;
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, func, threads, 0) != cudaSuccess || n < 1)
    n = 1;
  try {
    cache[key] = n;
  } catch (...) {  // out of host memory: answer without caching
  }
  return n;
}

// With `tiles` (a device counter), the launch uses the dynamic in-order
// schedule: the counter is zeroed on the stream first.
template <class R, class S>
sbbf_status launch_insert_src(const Tuning& t, uint32_t* words, R res, S src, uint64_t n,
                              cudaStream_t s, unsigned long long* tiles = nullptr) {
  if (n == 0) return SBBF_OK;
  void (*k)(uint32_t*, R, S, uint64_t, unsigned long long*) =
      t.lanes == 8 ? insert_kernel<R, true, S> : insert_kernel<R, false, S>;
  const uint64_t groups = (n + 63) / 64;
  const unsigned grid =
      grid_for(groups, t.threads / 32, cached_occupancy(reinterpret_cast<const void*>(k), t.threads));
  if (tiles) SBBF_CUDA(cudaMemsetAsync(tiles, 0, sizeof(unsigned long long), s));
  k<<<grid, t.threads, 0, s>>>(words, res, src, n, tiles);
  return launch_status();
}

template <class R>
sbbf_status launch_insert_t(const Tuning& t, uint32_t* words, R res, const uint64_t* hashes,
                            uint64_t n, cudaStream_t s, unsigned long long* tiles = nullptr) {
  return launch_insert_src(t, words, res, HashInput(hashes), n, s, tiles);
}

template <class R, bool kB, class S>
auto find_kernel_pick(const Tuning& t) {
  void (*k)(const uint32_t*, R, S, uint64_t, uint32_t*, unsigned long long*) = nullptr;
  if (t.lanes == 8) {
    k = t.unroll == 1 ? find_kernel<R, true, 1, kB, S>
        : t.unroll == 2 ? find_kernel<R, true, 2, kB, S> : find_kernel<R, true, 4, kB, S>;
  } else {
    k = t.unroll == 1 ? find_kernel<R, false, 1, kB, S>
        : t.unroll == 2 ? find_kernel<R, false, 2, kB, S> : find_kernel<R, false, 4, kB, S>;
  }
  return k;
}

template <class R, class S = HashInput>
auto find_kernel_for(const Tuning& t) {
  return t.l1_bypass ? find_kernel_pick<R, true, S>(t) : find_kernel_pick<R, false, S>(t);
}

// The one shape a fused key-hashing lookup is built in (one lane per key, two
// groups in flight), with or without L1 allocation of block loads.
template <class R, class S>
auto find_kernel_fused(bool l1_bypass) {
  return l1_bypass ? find_kernel<R, false, 2, true, S> : find_kernel<R, false, 2, false, S>;
}

// CTAs for a lookup launch of n keys with shape t.
inline unsigned find_grid(const Tuning& t, uint64_t n, const void* k) {
  const uint64_t groups = (n + 63) / 64;
  const uint64_t per_warp = t.lanes == 8 ? 1 : static_cast<uint64_t>(t.unroll);
  return grid_for(groups, (t.threads / 32) * per_warp, cached_occupancy(k, t.threads));
}

template <class R>
sbbf_status launch_find_t(const Tuning& t, const uint32_t* words, R res, const uint64_t* hashes,
                          uint64_t n, uint32_t* out, cudaStream_t s,
                          unsigned long long* tiles = nullptr) {
  if (n == 0) return SBBF_OK;
  auto k = find_kernel_for<R>(t);
  const unsigned grid = find_grid(t, n, reinterpret_cast<const void*>(k));
  if (tiles) SBBF_CUDA(cudaMemsetAsync(tiles, 0, sizeof(unsigned long long), s));
  k<<<grid, t.threads, 0, s>>>(words, res, HashInput(hashes), n, out, tiles);
  return launch_status();
}

// Lookup with a key source other than plain hashes, in the fused shape.
template <class R, class S>
sbbf_status launch_find_src(bool l1_bypass, const uint32_t* words, R res, S src, uint64_t n,
                            uint32_t* out, cudaStream_t s) {
  if (n == 0) return SBBF_OK;
  const Tuning t = {256, 1, 2, l1_bypass ? 1 : 0};
  auto k = find_kernel_fused<R, S>(l1_bypass);
  const unsigned grid = find_grid(t, n, reinterpret_cast<const void*>(k));
  k<<<grid, t.threads, 0, s>>>(words, res, src, n, out, nullptr);
  return launch_status();
}

// Region passes of a one-filter lookup (region_find_kernel): `passes`
// launches over all n keys, pass p answering the keys whose block lies in
// the p-th of `passes` equal parts of the block range [lo, hi) (the whole
// filter, or a shard whose words, held from block `base` on, cover it); the
// first writes every answer word, the later ones OR their bits in.
// Hashes: two 64-key groups per warp in flight; raw keys (hashed in the
// kernel, more registers) one.
constexpr int kRegionThreads = 512;
template <class S>
constexpr int region_unroll() {
  return std::is_same<S, HashInput>::value ? 2 : 1;
}

template <bool kMerge, class S>
sbbf_status launch_region_pass(const uint32_t* words, uint32_t num_blocks, uint32_t base,
                               S src, uint64_t n, uint32_t* out, uint32_t lo, uint32_t hi,
                               cudaStream_t s) {
  constexpr int kU = region_unroll<S>();
  auto k = base ? region_find_kernel<kU, kMerge, S, true> : region_find_kernel<kU, kMerge, S, false>;
  const uint64_t units = ((n + 63) / 64 + kU - 1) / kU;
  const unsigned grid = grid_for(units, kRegionThreads / 32,
                                 cached_occupancy(reinterpret_cast<const void*>(k), kRegionThreads));
  k<<<grid, kRegionThreads, 0, s>>>(words, num_blocks, base, lo, hi, src, n, out);
  return launch_status();
}

template <class S>
sbbf_status launch_find_regions(const uint32_t* words, uint32_t num_blocks, uint32_t base,
                                uint32_t lo, uint32_t hi, S src, uint64_t n, uint32_t* out,
                                uint32_t passes, cudaStream_t s) {
  const uint64_t span = hi - lo;
  for (uint32_t p = 0; p < passes; ++p) {
    const uint32_t a = lo + static_cast<uint32_t>(span * p / passes);
    const uint32_t b = lo + static_cast<uint32_t>(span * (p + 1) / passes);
    const sbbf_status st =
        p == 0 ? launch_region_pass<false>(words, num_blocks, base, src, n, out, a, b, s)
               : launch_region_pass<true>(words, num_blocks, base, src, n, out, a, b, s);
    if (st != SBBF_OK) return st;
  }
  return SBBF_OK;
}

}  // namespace sbbf
