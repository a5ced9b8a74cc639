// Single-filter kernels and entry points: insert (appendix add_hash), lookup
// (appendix find_hash), union, clear.
//
// Insert: warp-cooperative, eight lanes per key.  A warp loads 64 hashes with
// 16-byte loads (two per lane), then in 16 rounds each group of eight lanes
// takes one key: lane j of the group builds lane j's mask bit and issues one
// 32-bit red.or on word j of the key's block.  One warp instruction therefore
// covers four whole 32-byte sectors, one L2 atomic request per key, and the
// final filter is independent of the order in which the ORs land.
//
// Lookup: one thread per key.  Each lane takes two consecutive hashes (one
// 16-byte load), fetches each block with one 256-bit load, tests all eight
// lanes, and the warp packs 64 answers into two output words with two OR
// reductions.  Several 64-key groups are in flight per warp to cover DRAM
// latency.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdlib>

#include "sbbf.h"
#include "sbbf_device.cuh"
#include "sbbf_host.cuh"

namespace sbbf {

constexpr int kThreads = 256;
constexpr int kFindUnroll = 2;  // 64-key groups in flight per warp

template <bool kVec>
__device__ __forceinline__ void load_pair(const uint64_t* __restrict__ hashes,
                                          uint64_t k, uint64_t n, uint64_t pol,
                                          uint64_t& h0, uint64_t& h1) {
  if (kVec && k + 1 < n) {
    load_keys2(hashes + k, pol, h0, h1);
  } else {
    h0 = k < n ? load_key1(hashes + k, pol) : 0;
    h1 = k + 1 < n ? load_key1(hashes + k + 1, pol) : 0;
  }
}

template <bool kVec>
__global__ void __launch_bounds__(kThreads)
    insert_kernel(uint32_t* __restrict__ words, uint32_t num_blocks,
                  const uint64_t* __restrict__ hashes, uint64_t n) {
  const unsigned lane = lane_id();
  const uint64_t warp = (static_cast<uint64_t>(blockIdx.x) * kThreads + threadIdx.x) >> 5;
  const uint64_t n_warps = (static_cast<uint64_t>(gridDim.x) * kThreads) >> 5;
  const uint64_t n_groups = (n + 63) >> 6;
  const uint64_t pol = policy_evict_first();
  const uint32_t seed = lane_seed(lane & 7);
  uint32_t* const word_j = words + (lane & 7);
  const int group_base = static_cast<int>(lane & ~7u);

  for (uint64_t g = warp; g < n_groups; g += n_warps) {
    const uint64_t k = g * 64 + 2 * lane;
    uint64_t h0, h1;
    load_pair<kVec>(hashes, k, n, pol, h0, h1);
    const uint32_t x0 = static_cast<uint32_t>(h0), x1 = static_cast<uint32_t>(h1);
    const uint32_t b0 = k < n ? block_of(h0, num_blocks) : kNoBlock;
    const uint32_t b1 = k + 1 < n ? block_of(h1, num_blocks) : kNoBlock;
#pragma unroll
    for (int r = 0; r < 16; ++r) {
      const int src = group_base + (r >> 1);
      const uint32_t x = __shfl_sync(0xFFFFFFFFu, (r & 1) ? x1 : x0, src);
      const uint32_t b = __shfl_sync(0xFFFFFFFFu, (r & 1) ? b1 : b0, src);
      if (b != kNoBlock) red_or(word_j + 8ull * b, 1u << bit_index(x, seed));
    }
  }
}

template <bool kVec>
__global__ void __launch_bounds__(kThreads)
    find_kernel(const uint32_t* __restrict__ words, uint32_t num_blocks,
                const uint64_t* __restrict__ hashes, uint64_t n,
                uint32_t* __restrict__ out) {
  const unsigned lane = lane_id();
  const uint64_t warp = (static_cast<uint64_t>(blockIdx.x) * kThreads + threadIdx.x) >> 5;
  const uint64_t n_warps = (static_cast<uint64_t>(gridDim.x) * kThreads) >> 5;
  const uint64_t n_groups = (n + 63) >> 6;
  const uint64_t n_out = (n + 31) >> 5;
  const uint64_t pk = policy_evict_first();
  const uint64_t pf = policy_evict_last();

  for (uint64_t g0 = warp * kFindUnroll; g0 < n_groups; g0 += n_warps * kFindUnroll) {
    uint64_t h[kFindUnroll][2];
#pragma unroll
    for (int u = 0; u < kFindUnroll; ++u)
      load_pair<kVec>(hashes, (g0 + u) * 64 + 2 * lane, n, pk, h[u][0], h[u][1]);
    uint32_t w[kFindUnroll][2][8];
#pragma unroll
    for (int u = 0; u < kFindUnroll; ++u) {
#pragma unroll
      for (int s = 0; s < 2; ++s) {
        const uint64_t k = (g0 + u) * 64 + 2 * lane + s;
        if (k < n) {
          load_block(words + 8ull * block_of(h[u][s], num_blocks), pf, w[u][s]);
        } else {
#pragma unroll
          for (int i = 0; i < 8; ++i) w[u][s][i] = 0;
        }
      }
    }
#pragma unroll
    for (int u = 0; u < kFindUnroll; ++u) {
      const uint32_t r0 = block_has(w[u][0], static_cast<uint32_t>(h[u][0]));
      const uint32_t r1 = block_has(w[u][1], static_cast<uint32_t>(h[u][1]));
      const uint32_t v = (r0 | (r1 << 1)) << (2 * (lane & 15));
      const uint32_t lo = __reduce_or_sync(0xFFFFFFFFu, lane < 16 ? v : 0u);
      const uint32_t hi = __reduce_or_sync(0xFFFFFFFFu, lane >= 16 ? v : 0u);
      const uint64_t word = 2 * (g0 + u);
      if (lane == 0 && word < n_out) store_stream(out + word, lo);
      if (lane == 1 && word + 1 < n_out) store_stream(out + word + 1, hi);
    }
  }
}

__global__ void union_kernel(uint4* __restrict__ dst, const uint4* __restrict__ src,
                             uint64_t n16) {
  const uint64_t stride = static_cast<uint64_t>(gridDim.x) * blockDim.x;
  for (uint64_t i = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n16;
       i += stride) {
    uint4 d = dst[i];
    const uint4 s = __ldg(src + i);
    d.x |= s.x;
    d.y |= s.y;
    d.z |= s.z;
    d.w |= s.w;
    dst[i] = d;
  }
}

__global__ void clear_kernel(uint4* __restrict__ dst, uint64_t n16) {
  const uint64_t stride = static_cast<uint64_t>(gridDim.x) * blockDim.x;
  for (uint64_t i = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n16;
       i += stride)
    dst[i] = make_uint4(0, 0, 0, 0);
}

// ---- launchers (shared with the host-buffer pipeline) ----------------------

sbbf_status launch_insert(uint32_t* words, uint32_t num_blocks, const uint64_t* d_hashes,
                          uint64_t n, cudaStream_t s) {
  if (n == 0) return SBBF_OK;
  const uint64_t groups = (n + 63) / 64;
  const bool vec = (reinterpret_cast<uintptr_t>(d_hashes) & 15) == 0;
  if (vec) {
    static int occ = occupancy(insert_kernel<true>, kThreads);
    insert_kernel<true><<<grid_for(groups, kThreads / 32, occ), kThreads, 0, s>>>(
        words, num_blocks, d_hashes, n);
  } else {
    static int occ = occupancy(insert_kernel<false>, kThreads);
    insert_kernel<false><<<grid_for(groups, kThreads / 32, occ), kThreads, 0, s>>>(
        words, num_blocks, d_hashes, n);
  }
  return launch_status();
}

sbbf_status launch_find(const uint32_t* words, uint32_t num_blocks, const uint64_t* d_hashes,
                        uint64_t n, uint32_t* d_out, cudaStream_t s) {
  if (n == 0) return SBBF_OK;
  const uint64_t groups = (n + 63) / 64;
  const uint64_t per_cta = (kThreads / 32) * kFindUnroll;
  const bool vec = (reinterpret_cast<uintptr_t>(d_hashes) & 15) == 0;
  if (vec) {
    static int occ = occupancy(find_kernel<true>, kThreads);
    find_kernel<true><<<grid_for(groups, per_cta, occ), kThreads, 0, s>>>(
        words, num_blocks, d_hashes, n, d_out);
  } else {
    static int occ = occupancy(find_kernel<false>, kThreads);
    find_kernel<false><<<grid_for(groups, per_cta, occ), kThreads, 0, s>>>(
        words, num_blocks, d_hashes, n, d_out);
  }
  return launch_status();
}

sbbf_status launch_union(uint32_t* dst, const uint32_t* src, uint64_t n_words, cudaStream_t s) {
  const uint64_t n16 = n_words / 4;  // n_words is a multiple of 8
  static int occ = occupancy(union_kernel, kThreads);
  union_kernel<<<grid_for(n16, kThreads, occ), kThreads, 0, s>>>(
      reinterpret_cast<uint4*>(dst), reinterpret_cast<const uint4*>(src), n16);
  return launch_status();
}

sbbf_status launch_clear(uint32_t* dst, uint64_t n_words, cudaStream_t s) {
  const uint64_t n16 = n_words / 4;
  static int occ = occupancy(clear_kernel, kThreads);
  clear_kernel<<<grid_for(n16, kThreads, occ), kThreads, 0, s>>>(reinterpret_cast<uint4*>(dst),
                                                                 n16);
  return launch_status();
}

static bool on_device(const sbbf_t* f) { return f->device == current_device(); }

}  // namespace sbbf

using namespace sbbf;

extern "C" {

sbbf_status sbbf_create(uint32_t num_blocks, sbbf_t** out) {
  if (!out || num_blocks == 0) return SBBF_EINVAL;
  *out = nullptr;
  sbbf_t* f = static_cast<sbbf_t*>(std::calloc(1, sizeof(sbbf_t)));
  if (!f) return SBBF_ENOMEM;
  const size_t bytes = static_cast<size_t>(num_blocks) * 32;
  cudaError_t e = cudaMalloc(&f->words, bytes);
  if (e != cudaSuccess) {
    std::free(f);
    return record_cuda(e);
  }
  f->num_blocks = num_blocks;
  f->device = current_device();
  f->owns = 1;
  sbbf_status st = launch_clear(f->words, static_cast<uint64_t>(num_blocks) * 8, nullptr);
  if (st == SBBF_OK) {
    e = cudaStreamSynchronize(nullptr);
    if (e != cudaSuccess) st = record_cuda(e);
  }
  if (st != SBBF_OK) {
    cudaFree(f->words);
    std::free(f);
    return st;
  }
  *out = f;
  return SBBF_OK;
}

sbbf_status sbbf_wrap(uint32_t* d_words, uint32_t num_blocks, sbbf_t** out) {
  if (!out || !d_words || num_blocks == 0) return SBBF_EINVAL;
  if (reinterpret_cast<uintptr_t>(d_words) & 31) return SBBF_EINVAL;
  *out = nullptr;
  sbbf_t* f = static_cast<sbbf_t*>(std::calloc(1, sizeof(sbbf_t)));
  if (!f) return SBBF_ENOMEM;
  f->words = d_words;
  f->num_blocks = num_blocks;
  f->device = current_device();
  f->owns = 0;
  *out = f;
  return SBBF_OK;
}

sbbf_status sbbf_create_from_host(const uint32_t* h_words, uint32_t num_blocks, sbbf_t** out) {
  if (!h_words) return SBBF_EINVAL;
  sbbf_status st = sbbf_create(num_blocks, out);
  if (st != SBBF_OK) return st;
  cudaError_t e = cudaMemcpy((*out)->words, h_words, static_cast<size_t>(num_blocks) * 32,
                             cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    sbbf_destroy(*out);
    *out = nullptr;
    return record_cuda(e);
  }
  return SBBF_OK;
}

sbbf_status sbbf_destroy(sbbf_t* f) {
  if (!f) return SBBF_OK;
  sbbf_status st = SBBF_OK;
  if (f->owns) {
    cudaError_t e = cudaFree(f->words);  // cudaFree synchronises the device
    if (e != cudaSuccess) st = record_cuda(e);
  }
  std::free(f);
  return st;
}

uint32_t sbbf_num_blocks(const sbbf_t* f) { return f ? f->num_blocks : 0; }

sbbf_status sbbf_device_words(const sbbf_t* f, uint32_t** d_words, size_t* bytes) {
  if (!f) return SBBF_EINVAL;
  if (d_words) *d_words = f->words;
  if (bytes) *bytes = static_cast<size_t>(f->num_blocks) * 32;
  return SBBF_OK;
}

sbbf_status sbbf_clear(sbbf_t* f, sbbf_stream_t stream) {
  if (!f || !on_device(f)) return SBBF_EINVAL;
  return launch_clear(f->words, static_cast<uint64_t>(f->num_blocks) * 8, stream);
}

sbbf_status sbbf_insert_hashes(sbbf_t* f, const uint64_t* d_hashes, size_t n,
                               sbbf_stream_t stream) {
  if (!f || !on_device(f)) return SBBF_EINVAL;
  if (n == 0) return SBBF_OK;
  if (!d_hashes || (reinterpret_cast<uintptr_t>(d_hashes) & 7)) return SBBF_EINVAL;
  return launch_insert(f->words, f->num_blocks, d_hashes, n, stream);
}

sbbf_status sbbf_find_hashes(const sbbf_t* f, const uint64_t* d_hashes, size_t n,
                             uint32_t* d_out_bits, sbbf_stream_t stream) {
  if (!f || !on_device(f)) return SBBF_EINVAL;
  if (n == 0) return SBBF_OK;
  if (!d_hashes || !d_out_bits || (reinterpret_cast<uintptr_t>(d_hashes) & 7) ||
      (reinterpret_cast<uintptr_t>(d_out_bits) & 3))
    return SBBF_EINVAL;
  return launch_find(f->words, f->num_blocks, d_hashes, n, d_out_bits, stream);
}

sbbf_status sbbf_union(sbbf_t* dst, const sbbf_t* src, sbbf_stream_t stream) {
  if (!dst || !src || dst->num_blocks != src->num_blocks) return SBBF_EINVAL;
  if (!on_device(dst) || !on_device(src)) return SBBF_EINVAL;
  if (dst->words == src->words) return SBBF_OK;  // x | x == x
  return launch_union(dst->words, src->words, static_cast<uint64_t>(dst->num_blocks) * 8,
                      stream);
}

sbbf_status sbbf_copy_to_host(const sbbf_t* f, uint32_t* h_words, size_t bytes,
                              sbbf_stream_t stream) {
  if (!f || !h_words) return SBBF_EINVAL;
  const size_t need = static_cast<size_t>(f->num_blocks) * 32;
  if (bytes < need) return SBBF_EINVAL;
  SBBF_CUDA(cudaMemcpyAsync(h_words, f->words, need, cudaMemcpyDeviceToHost, stream));
  SBBF_CUDA(cudaStreamSynchronize(stream));
  return SBBF_OK;
}

}  // extern "C"
