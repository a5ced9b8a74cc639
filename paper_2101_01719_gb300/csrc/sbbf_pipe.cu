// Host-buffer entry points: hashes in host memory are copied to the device in
// chunks on two internal streams, so that the copy of chunk c+1 overlaps the
// kernel of chunk c and the result copy of chunk c-1.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdlib>

#include "sbbf.h"
#include "sbbf_host.cuh"

struct sbbf_host_pipe {
  size_t chunk;
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

extern "C" {

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
  if (!f || !p || f->device != current_device() || p->device != f->device) return SBBF_EINVAL;
  if (n == 0) return SBBF_OK;
  if (!h_hashes) return SBBF_EINVAL;
  return run_chunks(p, n, stream, [&](size_t off, size_t cnt, int i) -> sbbf_status {
    SBBF_CUDA(cudaMemcpyAsync(p->d_keys[i], h_hashes + off, cnt * sizeof(uint64_t),
                              cudaMemcpyHostToDevice, p->s[i]));
    return launch_insert_filter(f, p->d_keys[i], cnt, p->s[i]);
  });
}

sbbf_status sbbf_find_hashes_host(const sbbf_t* f, sbbf_host_pipe_t* p, const uint64_t* h_hashes,
                                  size_t n, uint32_t* h_out_bits, sbbf_stream_t stream) {
  if (!f || !p || f->device != current_device() || p->device != f->device) return SBBF_EINVAL;
  if (n == 0) return SBBF_OK;
  if (!h_hashes || !h_out_bits) return SBBF_EINVAL;
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
