// Host-side helpers shared by the library's translation units: status
// bookkeeping, device properties and launch sizing.
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <cstddef>
#include <cstdint>

#include "sbbf.h"

namespace sbbf {

// Names the enclosing scope for profilers and tracers (an NVTX range: the
// entry point's name around its kernels; nothing happens unless a tool such
// as ncu --nvtx or nsys is attached).
struct TraceRange {
  explicit TraceRange(const char* name) { nvtxRangePushA(name); }
  ~TraceRange() { nvtxRangePop(); }
  TraceRange(const TraceRange&) = delete;
  TraceRange& operator=(const TraceRange&) = delete;
};
#define SBBF_TRACE() ::sbbf::TraceRange sbbf_trace_range_(__func__)
#define SBBF_TRACE_NAMED(name) ::sbbf::TraceRange sbbf_trace_range_(name)

// Runs an entry point's body and maps any C++ exception from the host-side
// bookkeeping (container growth, thread creation) to SBBF_ENOMEM: nothing
// throws across the C ABI.
template <class F>
sbbf_status guarded(F&& body) noexcept {
  try {
    return body();
  } catch (...) {
    return SBBF_ENOMEM;
  }
}

// Records a failing CUDA call for sbbf_last_cuda_error() and maps it.
sbbf_status record_cuda(cudaError_t e);

#define SBBF_CUDA(call)                                   \
  do {                                                    \
    cudaError_t _e = (call);                              \
    if (_e != cudaSuccess) return ::sbbf::record_cuda(_e); \
  } while (0)

// Checks the launch just enqueued.
inline sbbf_status launch_status() {
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? SBBF_OK : record_cuda(e);
}

// Streaming multiprocessors of the current device (cached per device).
int sm_count();
int current_device();

// Resident CTAs per SM of `kernel` at `threads` threads and `smem` bytes of
// dynamic shared memory (cached by the caller in a static).
template <typename K>
int occupancy(K kernel, int threads, size_t smem = 0) {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, threads, smem) !=
          cudaSuccess ||
      n < 1)
    n = 1;
  return n;
}

// Grid for `work_items` independent items, each CTA taking `per_cta`, capped
// at `resident` CTAs per SM on every SM (the kernels loop over the rest).
inline unsigned grid_for(uint64_t work_items, uint64_t per_cta, int resident) {
  uint64_t want = (work_items + per_cta - 1) / per_cta;
  uint64_t cap = static_cast<uint64_t>(sm_count()) * static_cast<uint64_t>(resident);
  if (want > cap) want = cap;
  if (want < 1) want = 1;
  return static_cast<unsigned>(want);
}

}  // namespace sbbf

// The single-filter handle (opaque to callers).
struct sbbf_filter {
  uint32_t *words;      // device, num_blocks * lanes uint32
  uint32_t num_blocks;
  uint32_t lanes;       // 32-bit words per block: 8 (the paper's), 4 or 16
  int device;
  int owns;             // 1: allocated by the library
  int partition_mode;   // SBBF_PARTITION_*
  void *scratch;        // partitioned-insert scratch (library-owned), or NULL
  size_t scratch_bytes;
  unsigned *status;     // device status word of the partitioned passes (allocated with
                        // the first scratch; read and cleared by sbbf_device_status)
};

namespace sbbf {

// Partitioned path for filters larger than L2 (sbbf_partition.cu) and the
// single-filter policy that selects it (sbbf_single.cu).
uint64_t partition_scratch_bytes(uint32_t num_blocks, uint64_t n, bool with_index);
sbbf_status launch_insert_partitioned(uint32_t* words, uint32_t num_blocks, const uint64_t* hashes,
                                      uint64_t n, void* scratch, unsigned* status,
                                      cudaStream_t s);
sbbf_status launch_find_partitioned(const uint32_t* words, uint32_t num_blocks,
                                    const uint64_t* hashes, uint64_t n, uint32_t* d_out,
                                    void* scratch, unsigned* status, cudaStream_t s);
// True when a batch of n keys (a lookup batch when `lookup`) should take the
// partitioned path: the filter's mode, its size and the batch's keys per
// block.
bool want_partition(const sbbf_filter* f, uint64_t n, bool lookup);
// Region passes an insert or lookup of n hashes takes under the filter's
// mode (1: none).
uint32_t region_passes(const sbbf_filter* f, uint64_t n, bool lookup);
// Grows the filter's scratch (cudaMalloc, synchronous) to at least `bytes`;
// the first call also allocates the filter's zeroed device status word.
sbbf_status ensure_scratch(sbbf_filter* f, size_t bytes);

// Words and bytes of a filter's bit array.
inline uint64_t filter_words(const sbbf_filter* f) {
  return static_cast<uint64_t>(f->num_blocks) * f->lanes;
}
inline uint64_t filter_bytes(const sbbf_filter* f) { return filter_words(f) * 4; }

// Unpartitioned insert / lookup of device hashes for any lane count: by
// region passes where the filter's mode asks for them (region_passes), else
// in one pass.  Callers whose hashes are read from host memory pass
// regions = false: every region pass would read them again over the link.
sbbf_status launch_insert_filter(const sbbf_filter* f, const uint64_t* d_hashes, uint64_t n,
                                 cudaStream_t s, bool regions = true);
sbbf_status launch_find_filter(const sbbf_filter* f, const uint64_t* d_hashes, uint64_t n,
                               uint32_t* d_out, cudaStream_t s, bool regions = true);

}  // namespace sbbf
