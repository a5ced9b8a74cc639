// Status codes, CUDA error bookkeeping and device properties.
#include <cuda_runtime.h>

#include <atomic>

#include "sbbf.h"
#include "sbbf_host.cuh"

namespace sbbf {

static thread_local int g_last_cuda_error = 0;

sbbf_status record_cuda(cudaError_t e) {
  g_last_cuda_error = static_cast<int>(e);
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();  // not sticky: clear it so later calls are unaffected
    return SBBF_ENOMEM;
  }
  return SBBF_ECUDA;
}

int current_device() {
  int d = 0;
  if (cudaGetDevice(&d) != cudaSuccess) d = 0;
  return d;
}

int sm_count() {
  constexpr int kMaxDevices = 64;
  static std::atomic<int> cache[kMaxDevices];
  int d = current_device();
  if (d < 0 || d >= kMaxDevices) d = 0;
  int v = cache[d].load(std::memory_order_relaxed);
  if (v <= 0) {
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, d) != cudaSuccess ||
        v <= 0)
      v = 1;
    cache[d].store(v, std::memory_order_relaxed);
  }
  return v;
}

}  // namespace sbbf

extern "C" {

const char *sbbf_status_string(int status) {
  switch (status) {
    case SBBF_OK: return "SBBF_OK";
    case SBBF_EINVAL: return "SBBF_EINVAL: invalid argument";
    case SBBF_ENOMEM: return "SBBF_ENOMEM: allocation failed";
    case SBBF_ECUDA: return "SBBF_ECUDA: CUDA runtime error";
    case SBBF_EBUSY: return "SBBF_EBUSY: admission refused";
    case SBBF_ETIMEOUT: return "SBBF_ETIMEOUT: device wait reached its deadline";
    case SBBF_ERANGE: return "SBBF_ERANGE: size beyond the stated maximum";
    default: return "SBBF_?: unknown status";
  }
}

int sbbf_last_cuda_error(void) { return sbbf::g_last_cuda_error; }

uint32_t sbbf_version(void) { return (1u << 16) | 0u; }

}  // extern "C"
