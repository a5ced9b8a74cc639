// Host-buffer entry points, two ways of moving the data:
//   direct: the insert and lookup kernels read the hashes from page-locked
//     host memory and write the result bits into it through the device's
//     mapping of that memory (on GB300, over NVLink-C2C to the Grace host),
//     so no staging copy runs at all;
//   staged: the hashes are copied to the device in chunks on two internal
//     streams, so that the copy of chunk c+1 overlaps the kernel of chunk c
//     and the result copy of chunk c-1.
// The pipe's mode picks one (automatic: direct when every host buffer of the
// call is device-mapped page-locked memory).
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdlib>

#include "sbbf.h"
#include "sbbf_host.cuh"

struct sbbf_host_pipe {
  size_t chunk;
  int mode;  // SBBF_PIPE_*
  uint64_t* d_keys[2];
  uint32_t* d_bits[2];
  cudaStream_t s[2];
  cudaEvent_t start;
  cudaEvent_t done[2];
  int device;
};

using namespace sbbf;

static void pipe_free(sbbf_host_pipe_t* p) {
  for (int i = 0; i < 2; ++i) {
    if (p->d_keys[i]) cudaFree(p->d_keys[i]);
    if (p->d_bits[i]) cudaFree(p->d_bits[i]);
    if (p->s[i]) cudaStreamDestroy(p->s[i]);
    if (p->done[i]) cudaEventDestroy(p->done[i]);
  }
  if (p->start) cudaEventDestroy(p->start);
  std::free(p);
}

// Runs `body(chunk_index, offset, count, stream_slot)` over the chunks, then
// joins both internal streams back into `stream` and waits for it.
template <typename Body>
static sbbf_status run_chunks(sbbf_host_pipe_t* p, size_t n, cudaStream_t stream, Body body) {
  SBBF_CUDA(cudaEventRecord(p->start, stream));
  for (int i = 0; i < 2; ++i) SBBF_CUDA(cudaStreamWaitEvent(p->s[i], p->start, 0));
  size_t c = 0;
  for (size_t off = 0; off < n; off += p->chunk, ++c) {
    const size_t cnt = n - off < p->chunk ? n - off : p->chunk;
    sbbf_status st = body(off, cnt, static_cast<int>(c & 1));
    if (st != SBBF_OK) return st;
  }
  for (int i = 0; i < 2; ++i) {
    SBBF_CUDA(cudaEventRecord(p->done[i], p->s[i]));
    SBBF_CUDA(cudaStreamWaitEvent(stream, p->done[i], 0));
  }
  SBBF_CUDA(cudaStreamSynchronize(stream));
  return SBBF_OK;
}

// Device address of host memory h when it is page-locked memory mapped into
// the device's address space, else nullptr.
static const void* mapped(const void* h) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, h) != cudaSuccess) {
    cudaGetLastError();  // a pointer CUDA does not know: clear the error it recorded
    return nullptr;
  }
  return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

// Resolves the mode of one call: returns 1 for direct, 0 for staged, or -1
// when direct is required but a buffer is not mapped.
static int use_direct(const sbbf_host_pipe_t* p, const void* h_in, const void* h_out,
                      const void** d_in, void** d_out) {
  if (p->mode == SBBF_PIPE_COPY) return 0;
  *d_in = mapped(h_in);
  *d_out = h_out ? const_cast<void*>(mapped(h_out)) : nullptr;
  const bool ok = *d_in && (!h_out || *d_out);
  if (ok) return 1;
  return p->mode == SBBF_PIPE_DIRECT ? -1 : 0;
}

extern "C" {

sbbf_status sbbf_host_pipe_set_mode(sbbf_host_pipe_t* p, int mode) {
  if (!p || (mode != SBBF_PIPE_AUTO && mode != SBBF_PIPE_COPY && mode != SBBF_PIPE_DIRECT))
    return SBBF_EINVAL;
  p->mode = mode;
  return SBBF_OK;
}

sbbf_status sbbf_host_pipe_create(size_t chunk_hashes, sbbf_host_pipe_t** out) {
  if (!out || chunk_hashes == 0 || (chunk_hashes % 64) != 0) return SBBF_EINVAL;
  *out = nullptr;
  sbbf_host_pipe_t* p = static_cast<sbbf_host_pipe_t*>(std::calloc(1, sizeof(sbbf_host_pipe_t)));
  if (!p) return SBBF_ENOMEM;
  p->chunk = chunk_hashes;
  p->device = current_device();
  cudaError_t e = cudaSuccess;
  for (int i = 0; i < 2 && e == cudaSuccess; ++i) {
    e = cudaMalloc(&p->d_keys[i], chunk_hashes * sizeof(uint64_t));
    if (e == cudaSuccess) e = cudaMalloc(&p->d_bits[i], chunk_hashes / 8);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&p->s[i], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->done[i], cudaEventDisableTiming);
  }
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->start, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    pipe_free(p);
    return record_cuda(e);
  }
  *out = p;
  return SBBF_OK;
}

sbbf_status sbbf_host_pipe_destroy(sbbf_host_pipe_t* p) {
  if (!p) return SBBF_OK;
  cudaError_t e = cudaSuccess;
  for (int i = 0; i < 2; ++i)
    if (p->s[i]) {
      cudaError_t e2 = cudaStreamSynchronize(p->s[i]);
      if (e == cudaSuccess) e = e2;
    }
  pipe_free(p);
  return e == cudaSuccess ? SBBF_OK : record_cuda(e);
}

sbbf_status sbbf_insert_hashes_host(sbbf_t* f, sbbf_host_pipe_t* p, const uint64_t* h_hashes,
                                    size_t n, sbbf_stream_t stream) {
  SBBF_TRACE();
  if (!f || !p || f->device != current_device() || p->device != f->device) return SBBF_EINVAL;
  if (n == 0) return SBBF_OK;
  if (!h_hashes) return SBBF_EINVAL;
  const void* d_in = nullptr;
  void* d_out = nullptr;
  const int direct = use_direct(p, h_hashes, nullptr, &d_in, &d_out);
  if (direct < 0) return SBBF_EINVAL;
  if (direct) {
    const sbbf_status st =
        launch_insert_filter(f, static_cast<const uint64_t*>(d_in), n, stream, false);
    if (st != SBBF_OK) return st;
    SBBF_CUDA(cudaStreamSynchronize(stream));
    return SBBF_OK;
  }
  return run_chunks(p, n, stream, [&](size_t off, size_t cnt, int i) -> sbbf_status {
    SBBF_CUDA(cudaMemcpyAsync(p->d_keys[i], h_hashes + off, cnt * sizeof(uint64_t),
                              cudaMemcpyHostToDevice, p->s[i]));
    return launch_insert_filter(f, p->d_keys[i], cnt, p->s[i]);
  });
}

sbbf_status sbbf_find_hashes_host(const sbbf_t* f, sbbf_host_pipe_t* p, const uint64_t* h_hashes,
                                  size_t n, uint32_t* h_out_bits, sbbf_stream_t stream) {
  SBBF_TRACE();
  if (!f || !p || f->device != current_device() || p->device != f->device) return SBBF_EINVAL;
  if (n == 0) return SBBF_OK;
  if (!h_hashes || !h_out_bits) return SBBF_EINVAL;
  const void* d_in = nullptr;
  void* d_out = nullptr;
  const int direct = use_direct(p, h_hashes, h_out_bits, &d_in, &d_out);
  if (direct < 0) return SBBF_EINVAL;
  if (direct) {
    if (reinterpret_cast<uintptr_t>(d_in) & 7 || reinterpret_cast<uintptr_t>(d_out) & 3)
      return SBBF_EINVAL;
    const sbbf_status st = launch_find_filter(f, static_cast<const uint64_t*>(d_in), n,
                                              static_cast<uint32_t*>(d_out), stream, false);
    if (st != SBBF_OK) return st;
    SBBF_CUDA(cudaStreamSynchronize(stream));
    return SBBF_OK;
  }
  return run_chunks(p, n, stream, [&](size_t off, size_t cnt, int i) -> sbbf_status {
    SBBF_CUDA(cudaMemcpyAsync(p->d_keys[i], h_hashes + off, cnt * sizeof(uint64_t),
                              cudaMemcpyHostToDevice, p->s[i]));
    sbbf_status st = launch_find_filter(f, p->d_keys[i], cnt, p->d_bits[i], p->s[i]);
    if (st != SBBF_OK) return st;
    // off is a multiple of the chunk (a multiple of 64), so word-aligned.
    SBBF_CUDA(cudaMemcpyAsync(h_out_bits + off / 32, p->d_bits[i], ((cnt + 31) / 32) * 4,
                              cudaMemcpyDeviceToHost, p->s[i]));
    return SBBF_OK;
  });
}

}  // extern "C"
