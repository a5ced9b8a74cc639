// Many filters of uneven size in one device arena, served by single launches.
//
// Filter t is the plain filter of num_blocks[t] blocks whose block 0 is arena
// block base[t] (bases are the prefix sums of the sizes), so every filter
// keeps the paper's block selection and mask; only the block index gains an
// offset.  Keys reach their filter either by a per-key uint32 id ("tagged"
// form) or by grouping keys per filter with offsets ("segment" form).  A
// batch of any number of filters is one persistent launch (grid = SMs x
// resident CTAs, grid-stride over 64-key chunks); consecutive chunks belong
// to the same few filters, so in the segment form the filters being worked on
// stay in L2 even when the arena does not.
//
// The shape of those launches (CTA size, lanes per key, loads in flight) is
// picked per multi-filter set by an autotuner that checks each candidate's
// result bit for bit against the default shape before timing it.  A CUDA
// graph holds the batched insert -> lookup pair so a whole batch is one graph
// launch whose kernel arguments are updated in place.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "sbbf.h"
#include "sbbf_host.cuh"
#include "sbbf_launch.cuh"

namespace sbbf {
sbbf_status launch_clear(uint32_t* dst, uint64_t n_words, cudaStream_t s);
}  // namespace sbbf

struct sbbf_multi_set {
  uint32_t* words;                 // arena, total_blocks * 8 uint32
  uint64_t total_blocks;
  uint32_t n_filters;
  sbbf::FilterRef* d_dir;          // device directory
  std::vector<sbbf::FilterRef> h_dir;
  unsigned long long* d_invalid;   // keys with an id >= n_filters since the last read
  unsigned long long* d_tiles;     // work counters of the in-order schedule: [0] insert, [1] find
  int device;
  sbbf::Tuning tune_find_seg, tune_insert_seg, tune_find_tag, tune_insert_tag;
};

struct sbbf_multi_graph {
  sbbf_multi_t* m;
  cudaGraph_t graph;
  cudaGraphExec_t exec;
  cudaGraphNode_t memset_node, insert_node, find_node;
  sbbf::Tuning ti, tf;
};

using namespace sbbf;

namespace {

__global__ void mismatch_kernel(const uint32_t* __restrict__ a, const uint32_t* __restrict__ b,
                                uint64_t n, unsigned long long* __restrict__ count) {
  const uint64_t stride = static_cast<uint64_t>(gridDim.x) * blockDim.x;
  unsigned long long c = 0;
  for (uint64_t i = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += stride)
    c += a[i] != b[i];
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xFFFFFFFFu, c, o);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(count, c);
}

bool on_device(const sbbf_multi_t* m) { return m && m->device == current_device(); }

Segments seg_resolver(const sbbf_multi_t* m, const uint64_t* d_offsets) {
  Segments r{};
  r.offsets = d_offsets;
  r.dir = m->d_dir;
  r.n_filters = m->n_filters;
  return r;  // empty cached range: the first chunk searches
}

Tagged tag_resolver(const sbbf_multi_t* m, const uint32_t* d_ids) {
  return Tagged{d_ids, m->d_dir, m->n_filters, m->d_invalid, 0};
}

// ---- autotuner ----------------------------------------------------------------

std::vector<Tuning> candidates(int op) {
  std::vector<Tuning> c;
  for (int threads : {128, 256, 512}) {
    if (op == 0) {
      for (int lanes : {8, 1}) c.push_back(Tuning{threads, lanes, 1, 0});
    } else {
      for (int lanes : {1, 8})
        for (int unroll : {1, 2, 4})
          for (int l1 : {0, 1}) c.push_back(Tuning{threads, lanes, unroll, l1});
    }
  }
  return c;
}

using CacheKey = std::tuple<std::string, int, int, int, int>;  // gpu, op, form, log2 blocks, log2 n

std::mutex g_tune_mu;
std::map<CacheKey, Tuning> g_tune_cache;

int ilog2(uint64_t v) {
  int r = 0;
  while (v > 1) {
    v >>= 1;
    ++r;
  }
  return r;
}

std::string gpu_name() {
  cudaDeviceProp p;
  if (cudaGetDeviceProperties(&p, current_device()) != cudaSuccess) return "?";
  return std::string(p.name);
}

struct DeviceBuf {
  void* p = nullptr;
  ~DeviceBuf() {
    if (p) cudaFree(p);
  }
  cudaError_t alloc(size_t bytes) { return cudaMalloc(&p, bytes < 16 ? 16 : bytes); }
  template <typename T>
  T* as() const {
    return static_cast<T*>(p);
  }
};

struct Events {
  cudaEvent_t a = nullptr, b = nullptr;
  ~Events() {
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
  }
};

// Runs `run(t)` for each candidate shape; `check()` must report 0 mismatches
// against the default shape's result before the candidate is timed.  Keeps
// the fastest verified candidate (the default when nothing beats it).
template <typename Run, typename Prep, typename Check>
sbbf_status search(int op, Tuning def, cudaStream_t s, Run run, Prep prep, Check check,
                   Tuning* best_out, float* best_ms_out) {
  Events ev;
  SBBF_CUDA(cudaEventCreate(&ev.a));
  SBBF_CUDA(cudaEventCreate(&ev.b));
  Tuning best = def;
  float best_ms = 1e30f;
  for (const Tuning& t : candidates(op)) {
    SBBF_CUDA(prep());
    sbbf_status st = run(t);
    if (st != SBBF_OK) return st;
    uint64_t bad = 0;
    st = check(&bad);
    if (st != SBBF_OK) return st;
    if (bad != 0) continue;  // never pick a shape whose result differs
    float ms_min = 1e30f;
    for (int rep = 0; rep < 3; ++rep) {
      SBBF_CUDA(prep());
      SBBF_CUDA(cudaEventRecord(ev.a, s));
      st = run(t);
      if (st != SBBF_OK) return st;
      SBBF_CUDA(cudaEventRecord(ev.b, s));
      SBBF_CUDA(cudaEventSynchronize(ev.b));
      float ms = 0;
      SBBF_CUDA(cudaEventElapsedTime(&ms, ev.a, ev.b));
      ms_min = std::min(ms_min, ms);
    }
    if (ms_min < best_ms) {
      best_ms = ms_min;
      best = t;
    }
  }
  *best_out = best;
  if (best_ms_out) *best_ms_out = best_ms;
  return SBBF_OK;
}

sbbf_status count_mismatch(const uint32_t* a, const uint32_t* b, uint64_t n,
                           unsigned long long* d_count, cudaStream_t s, uint64_t* out) {
  SBBF_CUDA(cudaMemsetAsync(d_count, 0, sizeof(unsigned long long), s));
  mismatch_kernel<<<grid_for(n, 256, 8), 256, 0, s>>>(a, b, n, d_count);
  sbbf_status st = launch_status();
  if (st != SBBF_OK) return st;
  unsigned long long h = 0;
  SBBF_CUDA(cudaMemcpyAsync(&h, d_count, sizeof(h), cudaMemcpyDeviceToHost, s));
  SBBF_CUDA(cudaStreamSynchronize(s));
  *out = h;
  return SBBF_OK;
}

}  // namespace

extern "C" {

sbbf_status sbbf_multi_create(const uint32_t* h_num_blocks, uint32_t n_filters, sbbf_multi_t** out) {
  return guarded([&]() -> sbbf_status {
    if (!out || !h_num_blocks || n_filters == 0) return SBBF_EINVAL;
    *out = nullptr;
    uint64_t total = 0;
    for (uint32_t t = 0; t < n_filters; ++t) {
      if (h_num_blocks[t] == 0) return SBBF_EINVAL;
      total += h_num_blocks[t];
    }
    sbbf_multi_t* m = new (std::nothrow) sbbf_multi_t();
    if (!m) return SBBF_ENOMEM;
    m->n_filters = n_filters;
    m->total_blocks = total;
    m->device = current_device();
    m->tune_find_seg = m->tune_find_tag = kDefaultFind;
    m->tune_insert_seg = m->tune_insert_tag = kDefaultInsert;
    try {
      m->h_dir.resize(n_filters);
    } catch (...) {
      delete m;  // nothing on the device yet
      throw;
    }
    uint64_t base = 0;
    for (uint32_t t = 0; t < n_filters; ++t) {
      m->h_dir[t] = FilterRef{base, h_num_blocks[t], 0};
      base += h_num_blocks[t];
    }
    cudaError_t e = cudaMalloc(&m->words, total * 32);
    if (e == cudaSuccess) e = cudaMalloc(&m->d_dir, sizeof(FilterRef) * n_filters);
    if (e == cudaSuccess) e = cudaMalloc(&m->d_invalid, sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMalloc(&m->d_tiles, 2 * sizeof(unsigned long long));
    if (e == cudaSuccess)
      e = cudaMemcpy(m->d_dir, m->h_dir.data(), sizeof(FilterRef) * n_filters,
                     cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(m->d_invalid, 0, sizeof(unsigned long long));
    sbbf_status st = e == cudaSuccess ? SBBF_OK : record_cuda(e);
    if (st == SBBF_OK) st = launch_clear(m->words, total * 8, nullptr);
    if (st == SBBF_OK) {
      e = cudaStreamSynchronize(nullptr);
      if (e != cudaSuccess) st = record_cuda(e);
    }
    if (st != SBBF_OK) {
      sbbf_multi_destroy(m);
      return st;
    }
    *out = m;
    return SBBF_OK;
  });
}

sbbf_status sbbf_multi_destroy(sbbf_multi_t* m) {
  if (!m) return SBBF_OK;
  cudaError_t e = cudaSuccess, e2;
  if (m->words && (e2 = cudaFree(m->words)) != cudaSuccess) e = e2;
  if (m->d_dir && (e2 = cudaFree(m->d_dir)) != cudaSuccess) e = e2;
  if (m->d_invalid && (e2 = cudaFree(m->d_invalid)) != cudaSuccess) e = e2;
  if (m->d_tiles && (e2 = cudaFree(m->d_tiles)) != cudaSuccess) e = e2;
  delete m;
  return e == cudaSuccess ? SBBF_OK : record_cuda(e);
}

uint32_t sbbf_multi_num_filters(const sbbf_multi_t* m) { return m ? m->n_filters : 0; }

sbbf_status sbbf_multi_filter_info(const sbbf_multi_t* m, uint32_t id, uint64_t* base_block,
                                   uint32_t* num_blocks) {
  if (!m || id >= m->n_filters) return SBBF_EINVAL;
  if (base_block) *base_block = m->h_dir[id].base;
  if (num_blocks) *num_blocks = m->h_dir[id].num_blocks;
  return SBBF_OK;
}

sbbf_status sbbf_multi_device_words(const sbbf_multi_t* m, uint32_t** d_words, size_t* bytes) {
  if (!m) return SBBF_EINVAL;
  if (d_words) *d_words = m->words;
  if (bytes) *bytes = static_cast<size_t>(m->total_blocks) * 32;
  return SBBF_OK;
}

sbbf_status sbbf_multi_clear(sbbf_multi_t* m, sbbf_stream_t stream) {
  SBBF_TRACE();
  if (!on_device(m)) return SBBF_EINVAL;
  return launch_clear(m->words, m->total_blocks * 8, stream);
}

sbbf_status sbbf_multi_copy_to_host(const sbbf_multi_t* m, uint32_t* h_words, size_t bytes,
                                    sbbf_stream_t stream) {
  SBBF_TRACE();
  if (!m || !h_words) return SBBF_EINVAL;
  const size_t need = static_cast<size_t>(m->total_blocks) * 32;
  if (bytes < need) return SBBF_EINVAL;
  SBBF_CUDA(cudaMemcpyAsync(h_words, m->words, need, cudaMemcpyDeviceToHost, stream));
  SBBF_CUDA(cudaStreamSynchronize(stream));
  return SBBF_OK;
}

sbbf_status sbbf_multi_insert(sbbf_multi_t* m, const uint64_t* d_hashes, const uint32_t* d_ids,
                              size_t n, sbbf_stream_t stream) {
  return guarded([&]() -> sbbf_status {
    SBBF_TRACE();
    if (!on_device(m)) return SBBF_EINVAL;
    if (n == 0) return SBBF_OK;
    if (!d_hashes || !d_ids || (reinterpret_cast<uintptr_t>(d_hashes) & 7) ||
        (reinterpret_cast<uintptr_t>(d_ids) & 3))
      return SBBF_EINVAL;
    return launch_insert_t(m->tune_insert_tag, m->words, tag_resolver(m, d_ids), d_hashes, n, stream,
                           m->d_tiles);
  });
}

sbbf_status sbbf_multi_find(const sbbf_multi_t* m, const uint64_t* d_hashes, const uint32_t* d_ids,
                            size_t n, uint32_t* d_out_bits, sbbf_stream_t stream) {
  return guarded([&]() -> sbbf_status {
    SBBF_TRACE();
    if (!on_device(m)) return SBBF_EINVAL;
    if (n == 0) return SBBF_OK;
    if (!d_hashes || !d_ids || !d_out_bits || (reinterpret_cast<uintptr_t>(d_hashes) & 7) ||
        (reinterpret_cast<uintptr_t>(d_ids) & 3) || (reinterpret_cast<uintptr_t>(d_out_bits) & 3))
      return SBBF_EINVAL;
    return launch_find_t(m->tune_find_tag, m->words, tag_resolver(m, d_ids), d_hashes, n,
                         d_out_bits, stream, m->d_tiles + 1);
  });
}

sbbf_status sbbf_multi_insert_segments(sbbf_multi_t* m, const uint64_t* d_hashes,
                                       const uint64_t* d_offsets, size_t n,
                                       sbbf_stream_t stream) {
  return guarded([&]() -> sbbf_status {
    SBBF_TRACE();
    if (!on_device(m)) return SBBF_EINVAL;
    if (n == 0) return SBBF_OK;
    if (!d_hashes || !d_offsets || (reinterpret_cast<uintptr_t>(d_hashes) & 7) ||
        (reinterpret_cast<uintptr_t>(d_offsets) & 7))
      return SBBF_EINVAL;
    return launch_insert_t(m->tune_insert_seg, m->words, seg_resolver(m, d_offsets), d_hashes, n,
                           stream, m->d_tiles);
  });
}

sbbf_status sbbf_multi_find_segments(const sbbf_multi_t* m, const uint64_t* d_hashes,
                                     const uint64_t* d_offsets, size_t n, uint32_t* d_out_bits,
                                     sbbf_stream_t stream) {
  return guarded([&]() -> sbbf_status {
    SBBF_TRACE();
    if (!on_device(m)) return SBBF_EINVAL;
    if (n == 0) return SBBF_OK;
    if (!d_hashes || !d_offsets || !d_out_bits || (reinterpret_cast<uintptr_t>(d_hashes) & 7) ||
        (reinterpret_cast<uintptr_t>(d_offsets) & 7) || (reinterpret_cast<uintptr_t>(d_out_bits) & 3))
      return SBBF_EINVAL;
    return launch_find_t(m->tune_find_seg, m->words, seg_resolver(m, d_offsets), d_hashes, n,
                         d_out_bits, stream, m->d_tiles + 1);
  });
}

sbbf_status sbbf_multi_insert_each(sbbf_multi_t* m, const uint64_t* d_hashes,
                                   const uint64_t* h_offsets, sbbf_stream_t stream) {
  return guarded([&]() -> sbbf_status {
    SBBF_TRACE();
    if (!on_device(m) || !h_offsets || !d_hashes) return SBBF_EINVAL;
    for (uint32_t t = 0; t < m->n_filters; ++t) {
      if (h_offsets[t + 1] < h_offsets[t]) return SBBF_EINVAL;
      const uint64_t cnt = h_offsets[t + 1] - h_offsets[t];
      if (cnt == 0) continue;
      sbbf_status st = launch_insert_t(kDefaultInsert, m->words + 8 * m->h_dir[t].base,
                                       OneFilter{m->h_dir[t].num_blocks}, d_hashes + h_offsets[t],
                                       cnt, stream);
      if (st != SBBF_OK) return st;
    }
    return SBBF_OK;
  });
}

sbbf_status sbbf_multi_find_each(const sbbf_multi_t* m, const uint64_t* d_hashes,
                                 const uint64_t* h_offsets, uint32_t* d_out_bits,
                                 sbbf_stream_t stream) {
  return guarded([&]() -> sbbf_status {
    SBBF_TRACE();
    if (!on_device(m) || !h_offsets || !d_hashes || !d_out_bits) return SBBF_EINVAL;
    for (uint32_t t = 0; t < m->n_filters; ++t) {
      if (h_offsets[t + 1] < h_offsets[t]) return SBBF_EINVAL;
      const uint64_t cnt = h_offsets[t + 1] - h_offsets[t];
      if (cnt == 0) continue;
      if (h_offsets[t] % 32) return SBBF_EINVAL;  // each filter's answers start a fresh word
      Tuning tf = kDefaultFind;
      tf.l1_bypass = static_cast<uint64_t>(m->h_dir[t].num_blocks) * 32 > kL1BypassBytes;
      sbbf_status st = launch_find_t(tf, m->words + 8 * m->h_dir[t].base,
                                     OneFilter{m->h_dir[t].num_blocks}, d_hashes + h_offsets[t], cnt,
                                     d_out_bits + h_offsets[t] / 32, stream);
      if (st != SBBF_OK) return st;
    }
    return SBBF_OK;
  });
}

sbbf_status sbbf_multi_invalid_count(sbbf_multi_t* m, uint64_t* count, sbbf_stream_t stream) {
  if (!on_device(m) || !count) return SBBF_EINVAL;
  unsigned long long h = 0;
  SBBF_CUDA(cudaMemcpyAsync(&h, m->d_invalid, sizeof(h), cudaMemcpyDeviceToHost, stream));
  SBBF_CUDA(cudaMemsetAsync(m->d_invalid, 0, sizeof(h), stream));
  SBBF_CUDA(cudaStreamSynchronize(stream));
  *count = h;
  return SBBF_OK;
}

sbbf_status sbbf_multi_get_tuning(const sbbf_multi_t* m, int op, int form, int* threads,
                                  int* lanes, int* unroll, int* l1_bypass) {
  if (!m || (op != SBBF_OP_INSERT && op != SBBF_OP_FIND) ||
      (form != SBBF_FORM_SEGMENTS && form != SBBF_FORM_TAGGED))
    return SBBF_EINVAL;
  const Tuning& t = op == SBBF_OP_INSERT
                        ? (form == SBBF_FORM_SEGMENTS ? m->tune_insert_seg : m->tune_insert_tag)
                        : (form == SBBF_FORM_SEGMENTS ? m->tune_find_seg : m->tune_find_tag);
  if (threads) *threads = t.threads;
  if (lanes) *lanes = t.lanes;
  if (unroll) *unroll = t.unroll;
  if (l1_bypass) *l1_bypass = t.l1_bypass;
  return SBBF_OK;
}

sbbf_status sbbf_multi_set_tuning(sbbf_multi_t* m, int op, int form, int threads, int lanes,
                                  int unroll, int l1_bypass) {
  return guarded([&]() -> sbbf_status {
    const Tuning t{threads, lanes, unroll, l1_bypass};
    if (!m || !tuning_valid(t) || (op != SBBF_OP_INSERT && op != SBBF_OP_FIND) ||
        (form != SBBF_FORM_SEGMENTS && form != SBBF_FORM_TAGGED))
      return SBBF_EINVAL;
    Tuning& dst = op == SBBF_OP_INSERT
                      ? (form == SBBF_FORM_SEGMENTS ? m->tune_insert_seg : m->tune_insert_tag)
                      : (form == SBBF_FORM_SEGMENTS ? m->tune_find_seg : m->tune_find_tag);
    dst = t;
    return SBBF_OK;
  });
}

sbbf_status sbbf_multi_tune(sbbf_multi_t* m, int op, int form, const uint64_t* d_hashes,
                            const void* d_offsets_or_ids, size_t n, sbbf_stream_t stream,
                            float* best_ms) {
  return guarded([&]() -> sbbf_status {
    SBBF_TRACE();
    if (!on_device(m) || !d_hashes || !d_offsets_or_ids || n == 0) return SBBF_EINVAL;
    if ((op != SBBF_OP_INSERT && op != SBBF_OP_FIND) ||
        (form != SBBF_FORM_SEGMENTS && form != SBBF_FORM_TAGGED))
      return SBBF_EINVAL;
    const uint64_t n_s = std::min<uint64_t>(n, 1ull << 24);  // tuning sample: a prefix
    const CacheKey key{gpu_name(), op, form, ilog2(m->total_blocks), ilog2(n_s)};
    Tuning& dst = op == SBBF_OP_INSERT
                      ? (form == SBBF_FORM_SEGMENTS ? m->tune_insert_seg : m->tune_insert_tag)
                      : (form == SBBF_FORM_SEGMENTS ? m->tune_find_seg : m->tune_find_tag);
    {
      std::lock_guard<std::mutex> lock(g_tune_mu);
      auto it = g_tune_cache.find(key);
      if (it != g_tune_cache.end()) {
        dst = it->second;
        if (best_ms) *best_ms = -1.0f;
        return SBBF_OK;
      }
    }
    cudaStream_t s = stream;
    DeviceBuf cnt, tiles;
    SBBF_CUDA(cnt.alloc(sizeof(unsigned long long)));
    SBBF_CUDA(tiles.alloc(sizeof(unsigned long long)));
    unsigned long long* tile_ctr = tiles.as<unsigned long long>();

    // Sample offsets (segment form): the prefix of n_s keys, clipped.
    DeviceBuf d_off_s;
    const uint64_t* off_s = nullptr;
    uint64_t blocks_touched = m->total_blocks;
    if (form == SBBF_FORM_SEGMENTS) {
      std::vector<uint64_t> h_off(m->n_filters + 1);
      SBBF_CUDA(cudaMemcpyAsync(h_off.data(), d_offsets_or_ids, 8 * h_off.size(),
                                cudaMemcpyDeviceToHost, s));
      SBBF_CUDA(cudaStreamSynchronize(s));
      uint32_t last = 0;
      for (auto& o : h_off) o = std::min<uint64_t>(o, n_s);
      for (uint32_t t = 0; t < m->n_filters; ++t)
        if (h_off[t] < n_s) last = t;
      blocks_touched = m->h_dir[last].base + m->h_dir[last].num_blocks;
      SBBF_CUDA(d_off_s.alloc(8 * h_off.size()));
      SBBF_CUDA(cudaMemcpyAsync(d_off_s.p, h_off.data(), 8 * h_off.size(), cudaMemcpyHostToDevice, s));
      SBBF_CUDA(cudaStreamSynchronize(s));
      off_s = d_off_s.as<uint64_t>();
    }
    const uint32_t* ids = static_cast<const uint32_t*>(d_offsets_or_ids);
    Tuning best = dst;
    sbbf_status st;
    if (op == SBBF_OP_FIND) {
      const uint64_t words = (n_s + 31) / 32;
      DeviceBuf ref, got;
      SBBF_CUDA(ref.alloc(4 * words));
      SBBF_CUDA(got.alloc(4 * words));
      auto run_into = [&](const Tuning& t, uint32_t* out) -> sbbf_status {
        return form == SBBF_FORM_SEGMENTS
                   ? launch_find_t(t, m->words, seg_resolver(m, off_s), d_hashes, n_s, out, s,
                                   tile_ctr)
                   : launch_find_t(t, m->words, tag_resolver(m, ids), d_hashes, n_s, out, s,
                                   tile_ctr);
      };
      st = run_into(kDefaultFind, ref.as<uint32_t>());
      if (st != SBBF_OK) return st;
      st = search(
          op, kDefaultFind, s, [&](const Tuning& t) { return run_into(t, got.as<uint32_t>()); },
          [&]() { return cudaSuccess; },
          [&](uint64_t* bad) {
            return count_mismatch(ref.as<uint32_t>(), got.as<uint32_t>(), words,
                                  cnt.as<unsigned long long>(), s, bad);
          },
          &best, best_ms);
    } else {
      // Inserts run into scratch copies of the touched part of the arena.
      const uint64_t n_words = blocks_touched * 8;
      DeviceBuf ref, scratch;
      if (ref.alloc(4 * n_words) != cudaSuccess || scratch.alloc(4 * n_words) != cudaSuccess) {
        cudaGetLastError();
        return SBBF_ENOMEM;
      }
      auto run_into = [&](const Tuning& t, uint32_t* arena) -> sbbf_status {
        return form == SBBF_FORM_SEGMENTS
                   ? launch_insert_t(t, arena, seg_resolver(m, off_s), d_hashes, n_s, s, tile_ctr)
                   : launch_insert_t(t, arena, tag_resolver(m, ids), d_hashes, n_s, s, tile_ctr);
      };
      st = launch_clear(ref.as<uint32_t>(), n_words, s);
      if (st == SBBF_OK) st = run_into(kDefaultInsert, ref.as<uint32_t>());
      if (st != SBBF_OK) return st;
      st = search(
          op, kDefaultInsert, s, [&](const Tuning& t) { return run_into(t, scratch.as<uint32_t>()); },
          [&]() {
            return launch_clear(scratch.as<uint32_t>(), n_words, s) == SBBF_OK ? cudaSuccess
                                                                               : cudaErrorUnknown;
          },
          [&](uint64_t* bad) {
            return count_mismatch(ref.as<uint32_t>(), scratch.as<uint32_t>(), n_words,
                                  cnt.as<unsigned long long>(), s, bad);
          },
          &best, best_ms);
      // the tagged sample also counted its invalid ids once per run: reset
      if (form == SBBF_FORM_TAGGED)
        SBBF_CUDA(cudaMemsetAsync(m->d_invalid, 0, sizeof(unsigned long long), s));
    }
    if (st != SBBF_OK) return st;
    if (op == SBBF_OP_FIND && form == SBBF_FORM_TAGGED)
      SBBF_CUDA(cudaMemsetAsync(m->d_invalid, 0, sizeof(unsigned long long), s));
    SBBF_CUDA(cudaStreamSynchronize(s));
    dst = best;
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune_cache[key] = best;
    return SBBF_OK;
  });
}

// ---- CUDA graph: batched inserts then lookups, one graph launch ---------------

sbbf_status sbbf_multi_graph_create(sbbf_multi_t* m, sbbf_multi_graph_t** out) {
  return guarded([&]() -> sbbf_status {
    if (!on_device(m) || !out) return SBBF_EINVAL;
    *out = nullptr;
    sbbf_multi_graph_t* g = new (std::nothrow) sbbf_multi_graph_t();
    if (!g) return SBBF_ENOMEM;
    g->m = m;
    g->ti = m->tune_insert_seg;
    g->tf = m->tune_find_seg;
    auto fail = [&](cudaError_t e) {
      if (g->exec) cudaGraphExecDestroy(g->exec);
      if (g->graph) cudaGraphDestroy(g->graph);
      delete g;
      return record_cuda(e);
    };
    cudaError_t e = cudaGraphCreate(&g->graph, 0);
    if (e != cudaSuccess) return fail(e);
    // Both work counters are zeroed by a memset node ahead of the two kernels.
    cudaMemsetParams mp = {};
    mp.dst = m->d_tiles;
    mp.value = 0;
    mp.elementSize = 4;
    mp.width = 4;  // 16 bytes: both 64-bit counters
    mp.height = 1;
    mp.pitch = 0;
    e = cudaGraphAddMemsetNode(&g->memset_node, g->graph, nullptr, 0, &mp);
    if (e != cudaSuccess) return fail(e);
    // Placeholder arguments; every launch sets the real ones.
    Segments r = seg_resolver(m, nullptr);
    uint32_t* words = m->words;
    HashInput h(nullptr);
    uint64_t n = 0;
    uint32_t* o = nullptr;
    unsigned long long* ti = m->d_tiles;
    unsigned long long* tf = m->d_tiles + 1;
    void* iargs[] = {&words, &r, &h, &n, &ti};
    void* fargs[] = {&words, &r, &h, &n, &o, &tf};
    cudaKernelNodeParams ip = {};
    ip.func = reinterpret_cast<void*>(g->ti.lanes == 8 ? insert_kernel<Segments, true>
                                                       : insert_kernel<Segments, false>);
    ip.gridDim = dim3(1);
    ip.blockDim = dim3(g->ti.threads);
    ip.kernelParams = iargs;
    e = cudaGraphAddKernelNode(&g->insert_node, g->graph, &g->memset_node, 1, &ip);
    if (e != cudaSuccess) return fail(e);
    cudaKernelNodeParams fp = {};
    fp.func = reinterpret_cast<void*>(find_kernel_for<Segments>(g->tf));
    fp.gridDim = dim3(1);
    fp.blockDim = dim3(g->tf.threads);
    fp.kernelParams = fargs;
    e = cudaGraphAddKernelNode(&g->find_node, g->graph, &g->insert_node, 1, &fp);
    if (e != cudaSuccess) return fail(e);
    e = cudaGraphInstantiate(&g->exec, g->graph, 0);
    if (e != cudaSuccess) return fail(e);
    *out = g;
    return SBBF_OK;
  });
}

sbbf_status sbbf_multi_graph_destroy(sbbf_multi_graph_t* g) {
  if (!g) return SBBF_OK;
  if (g->exec) cudaGraphExecDestroy(g->exec);
  if (g->graph) cudaGraphDestroy(g->graph);
  delete g;
  return SBBF_OK;
}

sbbf_status sbbf_multi_graph_launch(sbbf_multi_graph_t* g, const uint64_t* d_ins,
                                    const uint64_t* d_ins_offsets, size_t n_ins,
                                    const uint64_t* d_q, const uint64_t* d_q_offsets, size_t n_q,
                                    uint32_t* d_out_bits, sbbf_stream_t stream) {
  return guarded([&]() -> sbbf_status {
    SBBF_TRACE();
    if (!g || !on_device(g->m)) return SBBF_EINVAL;
    if ((n_ins && (!d_ins || !d_ins_offsets)) || (n_q && (!d_q || !d_q_offsets || !d_out_bits)))
      return SBBF_EINVAL;
    if ((reinterpret_cast<uintptr_t>(d_ins) & 7) || (reinterpret_cast<uintptr_t>(d_q) & 7) ||
        (reinterpret_cast<uintptr_t>(d_ins_offsets) & 7) ||
        (reinterpret_cast<uintptr_t>(d_q_offsets) & 7) ||
        (reinterpret_cast<uintptr_t>(d_out_bits) & 3))
      return SBBF_EINVAL;
    sbbf_multi_t* m = g->m;
    Segments ri = seg_resolver(m, d_ins_offsets), rf = seg_resolver(m, d_q_offsets);
    uint32_t* words = m->words;
    HashInput hi(d_ins), hq(d_q);
    uint64_t ni = n_ins, nq = n_q;
    uint32_t* o = d_out_bits;
    unsigned long long* ti = m->d_tiles;
    unsigned long long* tf = m->d_tiles + 1;
    void* iargs[] = {&words, &ri, &hi, &ni, &ti};
    void* fargs[] = {&words, &rf, &hq, &nq, &o, &tf};
    cudaKernelNodeParams ip = {}, fp = {};
    SBBF_CUDA(cudaGraphKernelNodeGetParams(g->insert_node, &ip));
    SBBF_CUDA(cudaGraphKernelNodeGetParams(g->find_node, &fp));
    const int occ_i = cached_occupancy(ip.func, g->ti.threads);
    // n == 0 launches one CTA whose loop body never runs.
    ip.gridDim = dim3(grid_for((ni + 63) / 64, g->ti.threads / 32, occ_i));
    fp.gridDim = dim3(find_grid(g->tf, nq, fp.func));
    ip.kernelParams = iargs;
    fp.kernelParams = fargs;
    ip.extra = nullptr;
    fp.extra = nullptr;
    SBBF_CUDA(cudaGraphExecKernelNodeSetParams(g->exec, g->insert_node, &ip));
    SBBF_CUDA(cudaGraphExecKernelNodeSetParams(g->exec, g->find_node, &fp));
    SBBF_CUDA(cudaGraphLaunch(g->exec, stream));
    return SBBF_OK;
  });
}

}  // extern "C"
