// Synthetic inputs on the device (not part of the method): splitmix64 in
// counter form (Steele, Lea, Flood, OOPSLA 2014), the member/fresh query
// mix, a popcount of packed lookup results, and the block-range verification
// digest of a filter's words.
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

// ---- verification digest ------------------------------------------------
// Over block ranges of a filter's words, read as 64-bit units (unit u = word
// 2u | word 2u+1 << 32): the sum mod 2^64 of splitmix64 output u seeded with
// the unit's value, the set bits, and the blocks holding both an all-zero
// and a non-zero lane (never produced by inserts, which set one bit in every
// lane of their block).  The sums are order-free, so the per-CTA partial sums
// meet in 64-bit atomics and the result is the same whatever the schedule.
//
// Each CTA streams one contiguous chunk of blocks; a thread reads 16-byte
// vectors (two units) with fully coalesced loads, four per thread, and issues
// the next four before mixing the current ones; the lanes of one block (1, 2
// or 4 vectors, adjacent threads of a warp) add their zero-lane counts by
// shuffles.  Per (chunk, range) segment the CTA reduces once and adds to
// the range's three counters.
constexpr int kDigestThreads = 256;
constexpr int kDigestUnroll = 4;

// Vectors v0 + k * kDigestThreads + threadIdx.x, k < kUnroll, below v_end
// (zero past it), read once with streaming loads.
template <int kUnroll>
__device__ __forceinline__ void load_digest_batch(const uint4* __restrict__ vecs, uint64_t v0,
                                                  uint64_t v_end, uint4 (&x)[kUnroll]) {
#pragma unroll
  for (int k = 0; k < kUnroll; ++k) {
    const uint64_t v = v0 + k * kDigestThreads + threadIdx.x;
    x[k] = v < v_end ? __ldcs(vecs + v) : make_uint4(0, 0, 0, 0);
  }
}

template <int kLanes>
__global__ void __launch_bounds__(kDigestThreads)
    range_digest_kernel(const uint4* __restrict__ vecs, uint64_t num_blocks,
                        uint64_t range_blocks, uint64_t chunk,
                        unsigned long long* __restrict__ digest,
                        unsigned long long* __restrict__ bits,
                        unsigned long long* __restrict__ partial) {
  constexpr int kVec = kLanes / 4;  // 16-byte vectors per block
  __shared__ unsigned long long red[3][kDigestThreads / 32];
  const uint64_t lo = static_cast<uint64_t>(blockIdx.x) * chunk;
  const uint64_t hi = min(num_blocks, lo + chunk);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (uint64_t seg = lo; seg < hi;) {
    const uint64_t r = seg / range_blocks;
    const uint64_t end = min(hi, (r + 1) * range_blocks);
    const uint64_t v_end = end * kVec;
    constexpr uint64_t kBatch = static_cast<uint64_t>(kDigestThreads) * kDigestUnroll;
    unsigned long long d = 0, b = 0, p = 0;
    uint4 x[kDigestUnroll];
    load_digest_batch<kDigestUnroll>(vecs, seg * kVec, v_end, x);
    for (uint64_t v0 = seg * kVec; v0 < v_end; v0 += kBatch) {
      uint4 y[kDigestUnroll];  // the next batch is in flight while this one is mixed
      load_digest_batch<kDigestUnroll>(vecs, v0 + kBatch, v_end, y);
      unsigned bb = 0, pp = 0;
#pragma unroll
      for (int k = 0; k < kDigestUnroll; ++k) {
        const uint64_t v = v0 + k * kDigestThreads + threadIdx.x;
        const bool live = v < v_end;  // the lanes of one block are live together
        int zero = (x[k].x == 0) + (x[k].y == 0) + (x[k].z == 0) + (x[k].w == 0);
#pragma unroll
        for (int o = 1; o < kVec; o <<= 1) zero += __shfl_xor_sync(0xFFFFFFFFu, zero, o);
        if (live) {
          const uint64_t u = 2 * v;
          d += splitmix64_at((static_cast<uint64_t>(x[k].y) << 32) | x[k].x, u);
          d += splitmix64_at((static_cast<uint64_t>(x[k].w) << 32) | x[k].z, u + 1);
          bb += __popc(x[k].x) + __popc(x[k].y) + __popc(x[k].z) + __popc(x[k].w);
          if ((lane & (kVec - 1)) == 0 && zero > 0 && zero < kLanes) ++pp;
        }
      }
      b += bb;
      p += pp;
#pragma unroll
      for (int k = 0; k < kDigestUnroll; ++k) x[k] = y[k];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      d += __shfl_xor_sync(0xFFFFFFFFu, d, o);
      b += __shfl_xor_sync(0xFFFFFFFFu, b, o);
      p += __shfl_xor_sync(0xFFFFFFFFu, p, o);
    }
    if (lane == 0) {
      red[0][warp] = d;
      red[1][warp] = b;
      red[2][warp] = p;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      unsigned long long sd = 0, sb = 0, sp = 0;
#pragma unroll
      for (int w = 0; w < kDigestThreads / 32; ++w) {
        sd += red[0][w];
        sb += red[1][w];
        sp += red[2][w];
      }
      atomicAdd(digest + r, sd);
      if (sb) atomicAdd(bits + r, sb);
      if (sp) atomicAdd(partial + r, sp);
    }
    __syncthreads();  // red is rewritten by the next segment
    seg = end;
  }
}

template <int kLanes>
sbbf_status launch_range_digest(const uint32_t* words, uint64_t num_blocks, uint64_t range_blocks,
                                unsigned long long* digest, unsigned long long* bits,
                                unsigned long long* partial, cudaStream_t stream) {
  static int occ = occupancy(range_digest_kernel<kLanes>, kDigestThreads);
  const uint64_t per_cta = static_cast<uint64_t>(kDigestThreads) * kDigestUnroll / (kLanes / 4);
  const unsigned grid = grid_for(num_blocks, per_cta, occ);
  const uint64_t chunk = (num_blocks + grid - 1) / grid;
  range_digest_kernel<kLanes><<<grid, kDigestThreads, 0, stream>>>(
      reinterpret_cast<const uint4*>(words), num_blocks, range_blocks, chunk, digest, bits,
      partial);
  return launch_status();
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

sbbf_status sbbf_range_digest(const uint32_t* d_words, uint64_t num_blocks, uint32_t lanes,
                              uint64_t range_blocks, unsigned long long* d_digest,
                              unsigned long long* d_bits, unsigned long long* d_partial,
                              sbbf_stream_t stream) {
  if ((lanes != 4 && lanes != 8 && lanes != 16) || range_blocks == 0 || !d_digest || !d_bits ||
      !d_partial || num_blocks > (1ull << 40))
    return SBBF_EINVAL;
  if (num_blocks == 0) return SBBF_OK;
  if (!d_words || (reinterpret_cast<uintptr_t>(d_words) & 15)) return SBBF_EINVAL;
  const size_t bytes = ((num_blocks - 1) / range_blocks + 1) * sizeof(unsigned long long);
  SBBF_CUDA(cudaMemsetAsync(d_digest, 0, bytes, stream));
  SBBF_CUDA(cudaMemsetAsync(d_bits, 0, bytes, stream));
  SBBF_CUDA(cudaMemsetAsync(d_partial, 0, bytes, stream));
  if (lanes == 4)
    return launch_range_digest<4>(d_words, num_blocks, range_blocks, d_digest, d_bits, d_partial,
                                  stream);
  if (lanes == 8)
    return launch_range_digest<8>(d_words, num_blocks, range_blocks, d_digest, d_bits, d_partial,
                                  stream);
  return launch_range_digest<16>(d_words, num_blocks, range_blocks, d_digest, d_bits, d_partial,
                                 stream);
}

}  // extern "C"
