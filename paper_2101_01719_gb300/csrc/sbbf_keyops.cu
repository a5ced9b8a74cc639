// Keys hashed on the device: the step before the method.  The paper hashes a
// key once to 64 bits (intro) and fixes no hash function; these entry points
// hash with XXH64 (sbbf_keys.cuh), either into a hash array or fused into the
// insert and lookup kernels so that no hash array is written or read.
//
// The fused calls run the same kernels as the hash calls (one-filter
// resolver, default shapes) with a key source in place of the hash array.  A
// batch that the filter's policy sends down the partitioned path (large
// filter, dense batch) is hashed into the filter's scratch first and then
// takes that path, since its counting pass reads each hash twice.
#include <cuda_runtime.h>

#include <cstdint>

#include "sbbf.h"
#include "sbbf_host.cuh"
#include "sbbf_keys.cuh"
#include "sbbf_lanes.cuh"
#include "sbbf_launch.cuh"

namespace sbbf {

constexpr int kHashThreads = 256;

// out[k] = hash of key k; each thread takes the pairs (k, k + 1), k even.
template <class S>
__global__ void __launch_bounds__(kHashThreads)
    hash_kernel(S src, uint64_t n, uint64_t* __restrict__ out) {
  const uint64_t pol = policy_evict_first();
  const uint64_t pairs = (n + 1) / 2;
  const uint64_t stride = static_cast<uint64_t>(gridDim.x) * blockDim.x;
  for (uint64_t p = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x; p < pairs;
       p += stride) {
    const uint64_t k = 2 * p;
    uint64_t h0, h1;
    src.pair(k, n, pol, h0, h1);
    out[k] = h0;
    if (k + 1 < n) out[k + 1] = h1;
  }
}

template <class S>
sbbf_status launch_hash(S src, uint64_t n, uint64_t* out, cudaStream_t s) {
  if (n == 0) return SBBF_OK;
  static int occ = occupancy(hash_kernel<S>, kHashThreads);
  hash_kernel<S><<<grid_for((n + 1) / 2, kHashThreads, occ), kHashThreads, 0, s>>>(src, n, out);
  return launch_status();
}

static bool on_device(const sbbf_t* f) { return f->device == current_device(); }

static size_t round256(size_t b) { return (b + 255) & ~static_cast<size_t>(255); }

template <class S>
sbbf_status insert_src(sbbf_t* f, S src, uint64_t n, cudaStream_t s) {
  if (n == 0) return SBBF_OK;
  if (want_partition(f, n, false)) {
    const size_t hb = round256(n * 8);
    const sbbf_status st = ensure_scratch(f, hb + partition_scratch_bytes(f->num_blocks, n, false));
    if (st == SBBF_OK) {
      uint64_t* hashes = static_cast<uint64_t*>(f->scratch);
      const sbbf_status hs = launch_hash(src, n, hashes, s);
      if (hs != SBBF_OK) return hs;
      return launch_insert_partitioned(f->words, f->num_blocks, hashes, n,
                                       static_cast<char*>(f->scratch) + hb, f->status, s);
    }
    if (st != SBBF_ENOMEM || f->partition_mode == SBBF_PARTITION_ON) return st;
  }
  if (f->lanes != 8)
    return launch_insert_lanes(static_cast<int>(f->lanes), f->words, f->num_blocks, src, n, s);
  return launch_insert_src(kDefaultInsert, f->words, OneFilter{f->num_blocks}, src, n, s);
}

template <class S>
sbbf_status find_src(const sbbf_t* f, S src, uint64_t n, uint32_t* out, cudaStream_t s) {
  if (n == 0) return SBBF_OK;
  if (want_partition(f, n, true)) {
    const size_t hb = round256(n * 8);
    sbbf_t* fm = const_cast<sbbf_t*>(f);
    const sbbf_status st = ensure_scratch(fm, hb + partition_scratch_bytes(f->num_blocks, n, true));
    if (st == SBBF_OK) {
      uint64_t* hashes = static_cast<uint64_t*>(fm->scratch);
      const sbbf_status hs = launch_hash(src, n, hashes, s);
      if (hs != SBBF_OK) return hs;
      return launch_find_partitioned(f->words, f->num_blocks, hashes, n, out,
                                     static_cast<char*>(fm->scratch) + hb, fm->status, s);
    }
    if (st != SBBF_ENOMEM || f->partition_mode == SBBF_PARTITION_ON) return st;
  }
  if (f->lanes != 8)
    return launch_find_lanes(static_cast<int>(f->lanes), f->words, f->num_blocks, src, n, out, s);
  if (!S::kHeavy) {  // fixed-width keys, hashed in every pass
    const uint32_t passes = region_passes(f, n, true);
    if (passes > 1)
      return launch_find_regions(f->words, f->num_blocks, 0, 0, f->num_blocks, src, n, out,
                                 passes, s);
  }
  const bool bypass = static_cast<uint64_t>(f->num_blocks) * 32 > kL1BypassBytes;
  return launch_find_src(bypass, f->words, OneFilter{f->num_blocks}, src, n, out, s);
}

static bool fixed_keys_ok(const void* d_keys, uint32_t key_bytes, size_t n) {
  if (key_bytes != 4 && key_bytes != 8) return false;
  if (n == 0) return true;
  return d_keys && (reinterpret_cast<uintptr_t>(d_keys) % key_bytes) == 0;
}

static bool bytes_ok(const uint8_t* d_data, const uint64_t* d_offsets, size_t n) {
  if (n == 0) return true;
  return d_data && d_offsets && (reinterpret_cast<uintptr_t>(d_offsets) & 7) == 0;
}

}  // namespace sbbf

using namespace sbbf;

extern "C" {

sbbf_status sbbf_hash_keys(const void* d_keys, uint32_t key_bytes, size_t n, uint64_t seed,
                           uint64_t* d_hashes, sbbf_stream_t stream) {
  SBBF_TRACE();
  if (!fixed_keys_ok(d_keys, key_bytes, n)) return SBBF_EINVAL;
  if (n == 0) return SBBF_OK;
  if (!d_hashes || (reinterpret_cast<uintptr_t>(d_hashes) & 7)) return SBBF_EINVAL;
  if (key_bytes == 8)
    return launch_hash(Key64Input{static_cast<const uint64_t*>(d_keys), seed}, n, d_hashes, stream);
  return launch_hash(Key32Input{static_cast<const uint32_t*>(d_keys), seed}, n, d_hashes, stream);
}

sbbf_status sbbf_hash_bytes(const uint8_t* d_data, const uint64_t* d_offsets, size_t n,
                            uint64_t seed, uint64_t* d_hashes, sbbf_stream_t stream) {
  SBBF_TRACE();
  if (!bytes_ok(d_data, d_offsets, n)) return SBBF_EINVAL;
  if (n == 0) return SBBF_OK;
  if (!d_hashes || (reinterpret_cast<uintptr_t>(d_hashes) & 7)) return SBBF_EINVAL;
  return launch_hash(BytesInput{d_data, d_offsets, seed}, n, d_hashes, stream);
}

sbbf_status sbbf_insert_keys(sbbf_t* f, const void* d_keys, uint32_t key_bytes, size_t n,
                             uint64_t seed, sbbf_stream_t stream) {
  SBBF_TRACE();
  if (!f || !on_device(f) || !fixed_keys_ok(d_keys, key_bytes, n)) return SBBF_EINVAL;
  if (key_bytes == 8)
    return insert_src(f, Key64Input{static_cast<const uint64_t*>(d_keys), seed}, n, stream);
  return insert_src(f, Key32Input{static_cast<const uint32_t*>(d_keys), seed}, n, stream);
}

sbbf_status sbbf_find_keys(const sbbf_t* f, const void* d_keys, uint32_t key_bytes, size_t n,
                           uint64_t seed, uint32_t* d_out_bits, sbbf_stream_t stream) {
  SBBF_TRACE();
  if (!f || !on_device(f) || !fixed_keys_ok(d_keys, key_bytes, n)) return SBBF_EINVAL;
  if (n == 0) return SBBF_OK;
  if (!d_out_bits || (reinterpret_cast<uintptr_t>(d_out_bits) & 3)) return SBBF_EINVAL;
  if (key_bytes == 8)
    return find_src(f, Key64Input{static_cast<const uint64_t*>(d_keys), seed}, n, d_out_bits,
                    stream);
  return find_src(f, Key32Input{static_cast<const uint32_t*>(d_keys), seed}, n, d_out_bits,
                  stream);
}

sbbf_status sbbf_insert_bytes(sbbf_t* f, const uint8_t* d_data, const uint64_t* d_offsets,
                              size_t n, uint64_t seed, sbbf_stream_t stream) {
  SBBF_TRACE();
  if (!f || !on_device(f) || !bytes_ok(d_data, d_offsets, n)) return SBBF_EINVAL;
  return insert_src(f, BytesInput{d_data, d_offsets, seed}, n, stream);
}

sbbf_status sbbf_find_bytes(const sbbf_t* f, const uint8_t* d_data, const uint64_t* d_offsets,
                            size_t n, uint64_t seed, uint32_t* d_out_bits,
                            sbbf_stream_t stream) {
  SBBF_TRACE();
  if (!f || !on_device(f) || !bytes_ok(d_data, d_offsets, n)) return SBBF_EINVAL;
  if (n == 0) return SBBF_OK;
  if (!d_out_bits || (reinterpret_cast<uintptr_t>(d_out_bits) & 3)) return SBBF_EINVAL;
  return find_src(f, BytesInput{d_data, d_offsets, seed}, n, d_out_bits, stream);
}

}  // extern "C"
