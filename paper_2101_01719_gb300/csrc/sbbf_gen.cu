// Synthetic inputs on the device (not part of the method): splitmix64 in
// counter form (Steele, Lea, Flood, OOPSLA 2014), the member/fresh query
// mix, and a popcount of packed lookup results.
#include <cuda_runtime.h>

#include <cstdint>

#include "sbbf.h"
#include "sbbf_host.cuh"

namespace sbbf {

// Output i of the splitmix64 stream seeded with `seed`: the generator's state
// after i+1 increments of the golden-ratio gamma, passed through its mixer.
__device__ __forceinline__ uint64_t splitmix64_at(uint64_t seed, uint64_t i) {
  uint64_t z = seed + (i + 1) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__global__ void fill_splitmix_kernel(uint64_t* __restrict__ out, uint64_t n, uint64_t seed,
                                     uint64_t start) {
  const uint64_t stride = static_cast<uint64_t>(gridDim.x) * blockDim.x;
  for (uint64_t k = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x; k < n;
       k += stride)
    out[k] = splitmix64_at(seed, start + k);
}

__global__ void fill_queries_kernel(uint64_t* __restrict__ out, uint64_t n, uint64_t start,
                                    uint64_t ins_seed, uint64_t ins_start, uint64_t n_ins,
                                    uint64_t fresh_seed, uint64_t member_seed,
                                    uint64_t threshold) {
  const uint64_t stride = static_cast<uint64_t>(gridDim.x) * blockDim.x;
  for (uint64_t k = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x; k < n;
       k += stride) {
    const uint64_t j = start + k;
    const uint64_t r = splitmix64_at(member_seed, j);
    uint64_t q;
    if ((r >> 32) < threshold) {
      const uint64_t idx = ((r & 0xFFFFFFFFull) * n_ins) >> 32;
      q = splitmix64_at(ins_seed, ins_start + idx);
    } else {
      q = splitmix64_at(fresh_seed, j);
    }
    out[k] = q;
  }
}

// Last t with offsets[t] <= k (offsets[0] = 0 <= k < offsets[n_filters]).
__device__ __forceinline__ uint32_t segment_of(const uint64_t* offsets, uint32_t n_filters,
                                               uint64_t k) {
  uint32_t lo = 0, hi = n_filters;
  while (hi - lo > 1) {
    const uint32_t mid = (lo + hi) >> 1;
    if (offsets[mid] <= k) lo = mid; else hi = mid;
  }
  return lo;
}

__global__ void fill_segment_queries_kernel(uint64_t* __restrict__ out, uint64_t n,
                                            const uint64_t* __restrict__ q_off,
                                            const uint64_t* __restrict__ ins_off,
                                            uint32_t n_filters, uint64_t ins_seed,
                                            uint64_t fresh_seed, uint64_t member_seed,
                                            uint64_t threshold) {
  const uint64_t stride = static_cast<uint64_t>(gridDim.x) * blockDim.x;
  for (uint64_t k = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x; k < n;
       k += stride) {
    const uint32_t t = segment_of(q_off, n_filters, k);
    const uint64_t r = splitmix64_at(member_seed, k);
    const uint64_t s0 = ins_off[t], n_t = ins_off[t + 1] - s0;
    uint64_t q;
    if ((r >> 32) < threshold && n_t > 0)
      q = splitmix64_at(ins_seed, s0 + (((r & 0xFFFFFFFFull) * n_t) >> 32));
    else
      q = splitmix64_at(fresh_seed, k);
    out[k] = q;
  }
}

__global__ void fill_segment_ids_kernel(uint32_t* __restrict__ ids, uint64_t n,
                                        const uint64_t* __restrict__ off, uint32_t n_filters) {
  const uint64_t stride = static_cast<uint64_t>(gridDim.x) * blockDim.x;
  for (uint64_t k = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x; k < n;
       k += stride)
    ids[k] = segment_of(off, n_filters, k);
}

__global__ void count_bits_kernel(const uint32_t* __restrict__ bits, uint64_t n,
                                  unsigned long long* __restrict__ count) {
  const uint64_t n_words = (n + 31) / 32;
  const uint64_t stride = static_cast<uint64_t>(gridDim.x) * blockDim.x;
  unsigned long long c = 0;
  for (uint64_t w = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x; w < n_words;
       w += stride) {
    uint32_t v = bits[w];
    if (w == n_words - 1 && (n & 31)) v &= (1u << (n & 31)) - 1;
    c += __popc(v);
  }
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xFFFFFFFFu, c, o);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(count, c);
}

}  // namespace sbbf

using namespace sbbf;

extern "C" {

sbbf_status sbbf_fill_splitmix64(uint64_t* d_out, size_t n, uint64_t seed, uint64_t start,
                                 sbbf_stream_t stream) {
  if (n == 0) return SBBF_OK;
  if (!d_out) return SBBF_EINVAL;
  static int occ = occupancy(fill_splitmix_kernel, 256);
  fill_splitmix_kernel<<<grid_for(n, 256, occ), 256, 0, stream>>>(d_out, n, seed, start);
  return launch_status();
}

sbbf_status sbbf_fill_queries(uint64_t* d_out, size_t n, uint64_t start, uint64_t ins_seed,
                              uint64_t ins_start, uint64_t n_inserted, uint64_t fresh_seed,
                              uint64_t member_seed, uint64_t member_threshold,
                              sbbf_stream_t stream) {
  if (n == 0) return SBBF_OK;
  if (!d_out) return SBBF_EINVAL;
  if (member_threshold > 0 && (n_inserted == 0 || n_inserted > 0xFFFFFFFFull))
    return SBBF_EINVAL;
  static int occ = occupancy(fill_queries_kernel, 256);
  fill_queries_kernel<<<grid_for(n, 256, occ), 256, 0, stream>>>(
      d_out, n, start, ins_seed, ins_start, n_inserted, fresh_seed, member_seed,
      member_threshold);
  return launch_status();
}

sbbf_status sbbf_fill_segment_queries(uint64_t* d_out, size_t n, const uint64_t* d_q_offsets,
                                      const uint64_t* d_ins_offsets, uint32_t n_filters,
                                      uint64_t ins_seed, uint64_t fresh_seed,
                                      uint64_t member_seed, uint64_t member_threshold,
                                      sbbf_stream_t stream) {
  if (n == 0) return SBBF_OK;
  if (!d_out || !d_q_offsets || !d_ins_offsets || n_filters == 0) return SBBF_EINVAL;
  static int occ = occupancy(fill_segment_queries_kernel, 256);
  fill_segment_queries_kernel<<<grid_for(n, 256, occ), 256, 0, stream>>>(
      d_out, n, d_q_offsets, d_ins_offsets, n_filters, ins_seed, fresh_seed, member_seed,
      member_threshold);
  return launch_status();
}

sbbf_status sbbf_fill_segment_ids(uint32_t* d_ids, size_t n, const uint64_t* d_offsets,
                                  uint32_t n_filters, sbbf_stream_t stream) {
  if (n == 0) return SBBF_OK;
  if (!d_ids || !d_offsets || n_filters == 0) return SBBF_EINVAL;
  static int occ = occupancy(fill_segment_ids_kernel, 256);
  fill_segment_ids_kernel<<<grid_for(n, 256, occ), 256, 0, stream>>>(d_ids, n, d_offsets,
                                                                     n_filters);
  return launch_status();
}

sbbf_status sbbf_count_bits(const uint32_t* d_bits, size_t n, unsigned long long* d_count,
                            sbbf_stream_t stream) {
  if (!d_count || (n > 0 && !d_bits)) return SBBF_EINVAL;
  SBBF_CUDA(cudaMemsetAsync(d_count, 0, sizeof(unsigned long long), stream));
  if (n == 0) return SBBF_OK;
  static int occ = occupancy(count_bits_kernel, 256);
  count_bits_kernel<<<grid_for((n + 31) / 32, 256, occ), 256, 0, stream>>>(d_bits, n, d_count);
  return launch_status();
}

}  // extern "C"
