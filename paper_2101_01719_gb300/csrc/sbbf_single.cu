// Single-filter entry points: insert (appendix add_hash), lookup (appendix
// find_hash), union, clear.  Insert and lookup run the generic kernels of
// sbbf_kernels.cuh with the one-filter block resolver:
//   insert: 8 lanes per key, one red.or.b32 per lane on word j of the key's
//     block, so a warp instruction covers four whole 32-byte sectors and the
//     final filter is independent of the order the ORs land in;
//   lookup: one lane per key, one 256-bit block load, 64 answers per warp
//     packed by two OR reductions, two 64-key groups in flight per warp.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdlib>

#include "sbbf.h"
#include "sbbf_device.cuh"
#include "sbbf_host.cuh"
#include "sbbf_lanes.cuh"
#include "sbbf_launch.cuh"

namespace sbbf {

constexpr int kThreads = 256;

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
  return launch_insert_t(kDefaultInsert, words, OneFilter{num_blocks}, d_hashes, n, s);
}

sbbf_status launch_find(const uint32_t* words, uint32_t num_blocks, const uint64_t* d_hashes,
                        uint64_t n, uint32_t* d_out, cudaStream_t s) {
  Tuning t = kDefaultFind;
  t.l1_bypass = static_cast<uint64_t>(num_blocks) * 32 > kL1BypassBytes;
  return launch_find_t(t, words, OneFilter{num_blocks}, d_hashes, n, d_out, s);
}

sbbf_status launch_union(uint32_t* dst, const uint32_t* src, uint64_t n_words, cudaStream_t s) {
  const uint64_t n16 = n_words / 4;  // n_words is a multiple of 4
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


// Region passes of a lookup: the filter's blocks split into `passes` equal
// ranges of at most kRegionBytes, one launch per range over all the keys,
// each looking up only the keys whose block lies in its range (the first
// writes every answer word, the later ones OR their bits in).  A filter
// somewhat larger than what L2 keeps under random access is then read from
// L2 range by range, at the price of reading the keys once per pass.
// Automatic mode takes them for filters of more than 84 MiB and at most
// 192 MiB (two or three 64 MiB regions) and batches of at least 8Mi hashes.
// Measured on GB300 (1e9 lookups, G/s, region passes against random and
// partitioned): 80 MiB 183 / 217 / 108, 88 MiB 183 / 171 / 112, 128 MiB 181
// / 108 / 114, 160 MiB 121 / 88 / 115, 192 MiB 121 / 78 / 116, and at 128
// MiB with 4Mi, 16Mi and 64Mi hashes 82 / 85 / 45, 137 / 104 / 85, 168 / 110
// / 106.  Every pass reads all the keys (about 2.8 ms per 1e9 hashes), so
// smaller regions do not pay: four 32 MiB passes ran 79 G/s at 128 MiB (in
// a form of the kernel without the hash prefetch, which ran 157 with two).
constexpr uint64_t kRegionBytes = 64ull << 20;
constexpr uint64_t kRegionMinBytes = 84ull << 20;
constexpr uint64_t kRegionMaxBytes = 192ull << 20;
constexpr uint64_t kRegionMinKeys = 8ull << 20;
// Inserts by region passes (the same ranges; one insert_kernel launch per
// pass, keys outside the pass's range skipped) are not taken in automatic
// mode: measured against the partitioned insert (100M hashes in 16M batches,
// G/s) 75 / 77 at 96 MiB, 71 / 77 at 128 MiB, 52 / 75 at 160 MiB; with 4M
// batches at 128 MiB 56 / 50 against 56 random.  SBBF_PARTITION_REGIONS
// still forces them.
constexpr uint64_t kRegionInsertMinBytes = 0;
constexpr uint64_t kRegionInsertMaxBytes = 0;
constexpr uint64_t kRegionInsertMinKeys = 8ull << 20;

uint32_t region_passes(const sbbf_t* f, uint64_t n, bool lookup) {
  if (f->lanes != 8 || n == 0) return 1;
  const uint64_t bytes = static_cast<uint64_t>(f->num_blocks) * 32;
  const uint64_t p = (bytes + kRegionBytes - 1) / kRegionBytes;
  if (f->partition_mode == SBBF_PARTITION_REGIONS) return p > 1 ? static_cast<uint32_t>(p) : 1;
  if (f->partition_mode != SBBF_PARTITION_AUTO) return 1;
  const uint64_t lo = lookup ? kRegionMinBytes : kRegionInsertMinBytes;
  const uint64_t hi = lookup ? kRegionMaxBytes : kRegionInsertMaxBytes;
  const uint64_t min_keys = lookup ? kRegionMinKeys : kRegionInsertMinKeys;
  return bytes > lo && bytes <= hi && n >= min_keys && p > 1 ? static_cast<uint32_t>(p) : 1;
}

// Block range of pass p of `passes` over num_blocks blocks.
void region_of(uint64_t num_blocks, uint32_t p, uint32_t passes, uint32_t& lo, uint32_t& hi) {
  lo = static_cast<uint32_t>(num_blocks * p / passes);
  hi = static_cast<uint32_t>(num_blocks * (p + 1) / passes);
}

sbbf_status launch_insert_filter(const sbbf_t* f, const uint64_t* d_hashes, uint64_t n,
                                 cudaStream_t s, bool regions) {
  if (f->lanes != 8)
    return launch_insert_lanes(static_cast<int>(f->lanes), f->words, f->num_blocks,
                               HashInput(d_hashes), n, s);
  const uint32_t passes = regions ? region_passes(f, n, false) : 1;
  for (uint32_t p = 0; passes > 1 && p < passes; ++p) {
    uint32_t lo, hi;
    region_of(f->num_blocks, p, passes, lo, hi);
    const sbbf_status st = launch_insert_t(kDefaultInsert, f->words,
                                           RegionFilter{f->num_blocks, lo, hi}, d_hashes, n, s);
    if (st != SBBF_OK || p + 1 == passes) return st;
  }
  return launch_insert(f->words, f->num_blocks, d_hashes, n, s);
}

sbbf_status launch_find_filter(const sbbf_t* f, const uint64_t* d_hashes, uint64_t n,
                               uint32_t* d_out, cudaStream_t s, bool regions) {
  if (f->lanes != 8)
    return launch_find_lanes(static_cast<int>(f->lanes), f->words, f->num_blocks,
                             HashInput(d_hashes), n, d_out, s);
  const uint32_t passes = regions ? region_passes(f, n, true) : 1;
  if (passes > 1)
    return launch_find_regions(f->words, f->num_blocks, 0, 0, f->num_blocks, HashInput(d_hashes),
                               n, d_out, passes, s);
  return launch_find(f->words, f->num_blocks, d_hashes, n, d_out, s);
}

// Batches at least this large (kPartitionMinKeys for inserts,
// kPartitionMinLookupKeys for lookups) go through the partitioned path when
// the filter is at least kPartitionMin{Insert,Lookup}Bytes (automatic mode;
// lookups into filters of at most 192 MiB take region passes instead).
// Measured on GB300 (100M inserts in 16M batches, 1e9 lookups, partitioned
// against random G keys/s): inserts 78 / 119 at 64 MiB (the filter stays in
// L2), 77 / 73 at 96 MiB, 77 / 55-65 at 128 MiB, 70 / 40 at 256 MiB;
// lookups 113 / 148 at 96 MiB, 111-113 / 108-114 at 128 MiB (the two within
// the spread between boxes: the random path, one kernel and no scratch, is
// kept there), 110 / 97 at 144 MiB, 118 / 66 at 256 MiB; at 32 GiB 49 / 21.5
// G inserts/s.  Partitioned lookups of 4Mi hashes ran 45 / 85 G/s at 128 MiB
// and 42 / 69 at 192 MiB, so lookups partition from 8Mi hashes.
constexpr uint64_t kPartitionMinKeys = 4ull << 20;
constexpr uint64_t kPartitionMinLookupKeys = 8ull << 20;
constexpr uint64_t kPartitionMinInsertBytes = 96ull << 20;
constexpr uint64_t kPartitionMinLookupBytes = (128ull << 20) + 1;

// Automatic mode also wants enough keys per block: a partitioned pass reads
// every block of the filter once (the slice prefetch), so it pays only when
// the batch touches enough of the blocks.  Measured on the 32 GiB filter
// (2^30 blocks), partitioned against random G keys/s: lookups 17.6 / 38.5 at
// 0.125 keys per block, 25.8 / 38.6 at 0.25, 38.4 / 38.7 at 0.5, 46.6 / 38.6
// at 0.75, 50.0 / 38.5 at 0.93; inserts 16.3 / 22.2 at 0.125, 24.6 / 22.3 at
// 0.25, 37.3 / 22.3 at 0.5, 56.5 / 22.3 at 1.  So lookups partition from 0.6
// keys per block and inserts from 0.25 (also measured: lookups 2.1x faster
// at 2 keys per block on 2^26 blocks, 2.4x at 7.8 on 128.9M blocks).
bool want_partition(const sbbf_t* f, uint64_t n, bool lookup) {
  if (f->lanes != 8 || f->partition_mode == SBBF_PARTITION_OFF) return false;
  if (f->partition_mode == SBBF_PARTITION_ON) return true;
  if (region_passes(f, n, lookup) > 1) return false;  // region passes take the batch
  const uint64_t nb = f->num_blocks;
  const bool dense = lookup ? 5 * n >= 3 * nb : 4 * n >= nb;
  const uint64_t min_bytes = lookup ? kPartitionMinLookupBytes : kPartitionMinInsertBytes;
  const uint64_t min_keys = lookup ? kPartitionMinLookupKeys : kPartitionMinKeys;
  return n >= min_keys && nb * 32 >= min_bytes && dense;
}

// Grows the filter's scratch (cudaMalloc, synchronous) to hold `bytes`.
sbbf_status ensure_scratch(sbbf_t* f, size_t bytes) {
  if (!f->status) {
    unsigned* w = nullptr;
    cudaError_t e = cudaMalloc(&w, 256);
    if (e == cudaSuccess) e = cudaMemset(w, 0, 256);
    if (e != cudaSuccess) {
      if (w) cudaFree(w);
      return record_cuda(e);
    }
    f->status = w;
  }
  if (f->scratch_bytes >= bytes) return SBBF_OK;
  if (f->scratch) {
    cudaError_t e = cudaFree(f->scratch);
    f->scratch = nullptr;
    f->scratch_bytes = 0;
    if (e != cudaSuccess) return record_cuda(e);
  }
  cudaError_t e = cudaMalloc(&f->scratch, bytes);
  if (e != cudaSuccess) {
    f->scratch = nullptr;
    return record_cuda(e);
  }
  f->scratch_bytes = bytes;
  return SBBF_OK;
}

}  // namespace sbbf

using namespace sbbf;

extern "C" {

sbbf_status sbbf_create_lanes(uint32_t num_blocks, uint32_t lanes, sbbf_t** out) {
  if (!out || num_blocks == 0 || (lanes != 4 && lanes != 8 && lanes != 16)) return SBBF_EINVAL;
  *out = nullptr;
  sbbf_t* f = static_cast<sbbf_t*>(std::calloc(1, sizeof(sbbf_t)));
  if (!f) return SBBF_ENOMEM;
  f->num_blocks = num_blocks;
  f->lanes = lanes;
  cudaError_t e = cudaMalloc(&f->words, filter_bytes(f));
  if (e != cudaSuccess) {
    std::free(f);
    return record_cuda(e);
  }
  f->device = current_device();
  f->owns = 1;
  sbbf_status st = launch_clear(f->words, filter_words(f), nullptr);
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

sbbf_status sbbf_create(uint32_t num_blocks, sbbf_t** out) {
  return sbbf_create_lanes(num_blocks, 8, out);
}

sbbf_status sbbf_wrap_lanes(uint32_t* d_words, uint32_t num_blocks, uint32_t lanes,
                            sbbf_t** out) {
  if (!out || !d_words || num_blocks == 0) return SBBF_EINVAL;
  if (lanes != 4 && lanes != 8 && lanes != 16) return SBBF_EINVAL;
  if (reinterpret_cast<uintptr_t>(d_words) & 31) return SBBF_EINVAL;
  *out = nullptr;
  sbbf_t* f = static_cast<sbbf_t*>(std::calloc(1, sizeof(sbbf_t)));
  if (!f) return SBBF_ENOMEM;
  f->words = d_words;
  f->num_blocks = num_blocks;
  f->lanes = lanes;
  f->device = current_device();
  f->owns = 0;
  *out = f;
  return SBBF_OK;
}

sbbf_status sbbf_wrap(uint32_t* d_words, uint32_t num_blocks, sbbf_t** out) {
  return sbbf_wrap_lanes(d_words, num_blocks, 8, out);
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
  if (f->scratch) {
    cudaError_t e = cudaFree(f->scratch);
    if (e != cudaSuccess) st = record_cuda(e);
  }
  if (f->status) {
    cudaError_t e = cudaFree(f->status);
    if (e != cudaSuccess) st = record_cuda(e);
  }
  std::free(f);
  return st;
}

namespace {
__global__ void or_status_kernel(unsigned* status, unsigned bits) { atomicOr(status, bits); }
}  // namespace

sbbf_status sbbf_device_status(sbbf_t* f, sbbf_stream_t stream) {
  if (!f) return SBBF_EINVAL;
  if (!f->status) return SBBF_OK;  // no partitioned pass has run on this filter
  unsigned bits = 0;
  SBBF_CUDA(cudaMemcpyAsync(&bits, f->status, sizeof bits, cudaMemcpyDeviceToHost, stream));
  SBBF_CUDA(cudaStreamSynchronize(stream));
  if (bits == 0) return SBBF_OK;
  SBBF_CUDA(cudaMemsetAsync(f->status, 0, sizeof bits, stream));
  return SBBF_ETIMEOUT;
}

sbbf_status sbbf_record_device_status(sbbf_t* f, uint32_t bits, sbbf_stream_t stream) {
  if (!f || !on_device(f)) return SBBF_EINVAL;
  const sbbf_status st = ensure_scratch(f, 0);  // allocates the word on first use
  if (st != SBBF_OK) return st;
  if (bits == 0) return SBBF_OK;
  or_status_kernel<<<1, 1, 0, stream>>>(f->status, bits);
  return launch_status();
}

uint32_t sbbf_num_blocks(const sbbf_t* f) { return f ? f->num_blocks : 0; }

uint32_t sbbf_lanes(const sbbf_t* f) { return f ? f->lanes : 0; }

sbbf_status sbbf_device_words(const sbbf_t* f, uint32_t** d_words, size_t* bytes) {
  if (!f) return SBBF_EINVAL;
  if (d_words) *d_words = f->words;
  if (bytes) *bytes = filter_bytes(f);
  return SBBF_OK;
}

sbbf_status sbbf_clear(sbbf_t* f, sbbf_stream_t stream) {
  SBBF_TRACE();
  if (!f || !on_device(f)) return SBBF_EINVAL;
  return launch_clear(f->words, filter_words(f), stream);
}

sbbf_status sbbf_insert_hashes(sbbf_t* f, const uint64_t* d_hashes, size_t n,
                               sbbf_stream_t stream) {
  SBBF_TRACE();
  if (!f || !on_device(f)) return SBBF_EINVAL;
  if (n == 0) return SBBF_OK;
  if (!d_hashes || (reinterpret_cast<uintptr_t>(d_hashes) & 7)) return SBBF_EINVAL;
  if (want_partition(f, n, false)) {
    const sbbf_status st = ensure_scratch(f, partition_scratch_bytes(f->num_blocks, n, false));
    if (st == SBBF_OK)
      return launch_insert_partitioned(f->words, f->num_blocks, d_hashes, n, f->scratch, f->status,
                                       stream);
    if (st != SBBF_ENOMEM || f->partition_mode == SBBF_PARTITION_ON) return st;
    // automatic mode without room for the scratch: insert unpartitioned
  }
  return launch_insert_filter(f, d_hashes, n, stream);
}

sbbf_status sbbf_region_passes(const sbbf_t* f, size_t n, int lookup, uint32_t* passes) {
  if (!f || !passes) return SBBF_EINVAL;
  *passes = region_passes(f, n, lookup != 0);
  return SBBF_OK;
}

sbbf_status sbbf_set_partitioning(sbbf_t* f, int mode) {
  if (!f || (mode != SBBF_PARTITION_AUTO && mode != SBBF_PARTITION_OFF &&
             mode != SBBF_PARTITION_ON && mode != SBBF_PARTITION_REGIONS))
    return SBBF_EINVAL;
  f->partition_mode = mode;
  return SBBF_OK;
}

sbbf_status sbbf_find_hashes(const sbbf_t* f, const uint64_t* d_hashes, size_t n,
                             uint32_t* d_out_bits, sbbf_stream_t stream) {
  SBBF_TRACE();
  if (!f || !on_device(f)) return SBBF_EINVAL;
  if (n == 0) return SBBF_OK;
  if (!d_hashes || !d_out_bits || (reinterpret_cast<uintptr_t>(d_hashes) & 7) ||
      (reinterpret_cast<uintptr_t>(d_out_bits) & 3))
    return SBBF_EINVAL;
  if (want_partition(f, n, true)) {
    const sbbf_status st =
        ensure_scratch(const_cast<sbbf_t*>(f), partition_scratch_bytes(f->num_blocks, n, true));
    if (st == SBBF_OK)
      return launch_find_partitioned(f->words, f->num_blocks, d_hashes, n, d_out_bits, f->scratch,
                                     f->status, stream);
    if (st != SBBF_ENOMEM || f->partition_mode == SBBF_PARTITION_ON) return st;
  }
  return launch_find_filter(f, d_hashes, n, d_out_bits, stream);
}

sbbf_status sbbf_union(sbbf_t* dst, const sbbf_t* src, sbbf_stream_t stream) {
  SBBF_TRACE();
  if (!dst || !src || dst->num_blocks != src->num_blocks || dst->lanes != src->lanes)
    return SBBF_EINVAL;
  if (!on_device(dst) || !on_device(src)) return SBBF_EINVAL;
  if (dst->words == src->words) return SBBF_OK;  // x | x == x
  return launch_union(dst->words, src->words, filter_words(dst), stream);
}

sbbf_status sbbf_copy_to_host(const sbbf_t* f, uint32_t* h_words, size_t bytes,
                              sbbf_stream_t stream) {
  SBBF_TRACE();
  if (!f || !h_words) return SBBF_EINVAL;
  const size_t need = filter_bytes(f);
  if (bytes < need) return SBBF_EINVAL;
  SBBF_CUDA(cudaMemcpyAsync(h_words, f->words, need, cudaMemcpyDeviceToHost, stream));
  SBBF_CUDA(cudaStreamSynchronize(stream));
  return SBBF_OK;
}

}  // extern "C"
