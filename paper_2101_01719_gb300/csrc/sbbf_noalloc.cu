// Allocation-free tagged lookup over several filters.
//
// Who needs it: callers that must not call cudaMalloc/cudaFree on this path.
// A serving loop that admits work against a fixed device-memory budget cannot
// let a lookup grab memory behind the budget's back; a framework whose caching
// allocator already reserved the device memory would see an allocation here
// fail or fragment its pool; and cudaFree synchronises the whole device, which
// a latency-critical caller cannot afford.  This entry point therefore keeps
// its only scratch -- the filter directory derived from the caller's sizes and
// the invalid-id counter -- in one file-scope __device__ array that every GPU
// loading the library holds until the process exits.
//
// The array is shared by every call: each call rewrites the directory entries
// it uses and zeroes the counter before its lookup kernel runs.  Two calls
// that overlap on the GPU (different streams, no ordering between them) race
// on the array and may return wrong answers; order such calls on one stream.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "sbbf.h"
#include "sbbf_host.cuh"
#include "sbbf_kernels.cuh"
#include "sbbf_launch.cuh"

namespace sbbf {
namespace {

constexpr size_t kCounterBytes = 256;  // invalid-id counter, padded to the alignment
constexpr size_t kScratchBytes =
    kCounterBytes + sizeof(FilterRef) * static_cast<size_t>(SBBF_NOALLOC_MAX_FILTERS);

// The scratch: [0, 8) invalid-id counter, [256, ...) directory entries.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// Tagged form over a directory built on the device from caller sizes: an id
// past the set or a filter of zero blocks is an invalid key (skipped, counted).
struct TaggedDeviceDir {
  static constexpr int kMinBlocks = 3;
  const uint32_t* ids;
  const FilterRef* dir;
  uint32_t n_filters;
  unsigned long long* invalid;
  uint32_t bad;

  __device__ __forceinline__ void begin_chunk(uint64_t) {}
  __device__ __forceinline__ uint64_t block(uint64_t k, uint64_t h) {
    const uint32_t t = __ldg(ids + k);
    if (t >= n_filters) {
      ++bad;
      return kNoBlock64;
    }
    const FilterRef r = load_ref(dir, t);
    if (r.num_blocks == 0) {
      ++bad;
      return kNoBlock64;
    }
    return r.base + block_of(h, r.num_blocks);
  }
  __device__ __forceinline__ void finish() const {
    unsigned long long c = bad;
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xFFFFFFFFu, c, o);
    if (lane_id() == 0 && c) atomicAdd(invalid, c);
  }
};

// One CTA of 1024 threads: dir[t] = {sum of sizes before t, sizes[t]} by a
// block-wide exclusive scan in chunks of 1024, and counter = 0.
__global__ void __launch_bounds__(1024)
    build_directory_kernel(const uint32_t* __restrict__ sizes, uint32_t n_filters,
                           FilterRef* __restrict__ dir, unsigned long long* __restrict__ counter) {
  __shared__ unsigned long long warp_total[32];
  __shared__ unsigned long long carry;
  const unsigned lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) {
    carry = 0;
    *counter = 0;
  }
  __syncthreads();
  for (uint32_t start = 0; start < n_filters; start += blockDim.x) {
    const uint32_t t = start + threadIdx.x;
    const unsigned long long v = t < n_filters ? sizes[t] : 0ull;
    unsigned long long x = v;  // inclusive scan within the warp
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long y = __shfl_up_sync(0xFFFFFFFFu, x, o);
      if (lane >= static_cast<unsigned>(o)) x += y;
    }
    if (lane == 31) warp_total[warp] = x;
    __syncthreads();
    if (warp == 0) {  // inclusive scan of the 32 warp totals
      unsigned long long s = warp_total[lane];
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xFFFFFFFFu, s, o);
        if (lane >= static_cast<unsigned>(o)) s += y;
      }
      warp_total[lane] = s;
    }
    __syncthreads();
    const unsigned long long before_warp = warp > 0 ? warp_total[warp - 1] : 0ull;
    if (t < n_filters) {
      FilterRef r;
      r.base = carry + before_warp + x - v;
      r.num_blocks = static_cast<uint32_t>(v);
      r.reserved = 0;
      dir[t] = r;
    }
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) carry += warp_total[31];
    __syncthreads();
  }
}

std::mutex g_setup_mu;
constexpr int kMaxDevices = 64;
unsigned char* g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device, looked up once
// per device with that device current (host code cannot use the symbol
// itself: on the host it names a stand-in, not device memory).
sbbf_status scratch_address(unsigned char** out) {
  const int d = current_device();
  if (d < 0 || d >= kMaxDevices) return SBBF_EINVAL;
  std::lock_guard<std::mutex> lock(g_setup_mu);
  if (!g_scratch_addr[d]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return record_cuda(e);
    g_scratch_addr[d] = static_cast<unsigned char*>(p);
  }
  *out = g_scratch_addr[d];
  return SBBF_OK;
}

}  // namespace
}  // namespace sbbf

using namespace sbbf;

extern "C" sbbf_status sbbf_multi_find_noalloc(const uint32_t* d_arena,
                                               const uint32_t* d_num_blocks, uint32_t n_filters,
                                               const uint64_t* d_hashes, const uint32_t* d_ids,
                                               size_t n, uint32_t* d_out_bits,
                                               unsigned long long* d_invalid_count,
                                               sbbf_stream_t stream) {
  SBBF_TRACE();
  if (n_filters == 0 || !d_arena || !d_num_blocks) return SBBF_EINVAL;
  if (n_filters > SBBF_NOALLOC_MAX_FILTERS) return SBBF_ERANGE;
  if (n > 0 && (!d_hashes || !d_ids || !d_out_bits)) return SBBF_EINVAL;
  if ((reinterpret_cast<uintptr_t>(d_arena) & 31) || (reinterpret_cast<uintptr_t>(d_num_blocks) & 3) ||
      (reinterpret_cast<uintptr_t>(d_hashes) & 7) || (reinterpret_cast<uintptr_t>(d_ids) & 3) ||
      (reinterpret_cast<uintptr_t>(d_out_bits) & 3) ||
      (reinterpret_cast<uintptr_t>(d_invalid_count) & 7))
    return SBBF_EINVAL;
  unsigned char* scratch = nullptr;
  sbbf_status st = scratch_address(&scratch);
  if (st != SBBF_OK) return st;
  auto* counter = reinterpret_cast<unsigned long long*>(scratch);
  auto* dir = reinterpret_cast<FilterRef*>(scratch + kCounterBytes);

  build_directory_kernel<<<1, 1024, 0, stream>>>(d_num_blocks, n_filters, dir, counter);
  st = launch_status();
  if (st != SBBF_OK) return st;
  if (n > 0) {
    auto kernel = find_kernel<TaggedDeviceDir, false, 2, false>;
    const int occ = cached_occupancy(reinterpret_cast<const void*>(kernel), 256);
    const uint64_t groups = (n + 63) / 64;
    const TaggedDeviceDir res{d_ids, dir, n_filters, counter, 0};
    kernel<<<grid_for(groups, (256 / 32) * 2, occ), 256, 0, stream>>>(d_arena, res, d_hashes, n,
                                                                      d_out_bits, nullptr);
    st = launch_status();
    if (st != SBBF_OK) return st;
  }
  if (d_invalid_count)
    SBBF_CUDA(cudaMemcpyAsync(d_invalid_count, counter, sizeof(unsigned long long),
                              cudaMemcpyDeviceToDevice, stream));
  return SBBF_OK;
}
