// Serving: many resident filters, requests arriving over time, continuous
// batching under a device-memory budget.
//
// A request is one insert or lookup of n hashes on one filter.  Requests
// queue per filter in arrival order.  A scheduler thread owns the GPU stream;
// whenever fewer than `max_inflight_windows` windows are on the GPU it forms
// the next window: it visits the filters in the order of their oldest queued
// request and, for each filter it can make resident within the budget, takes
// that filter's queued requests in order (at most four runs of one
// operation, so a window has at most four phases), up to
// `max_window_requests` requests and `max_window_keys` hashes per window.  One admission thus
// serves a filter's whole backlog, and a filter that cannot be admitted yet
// holds back only its own requests.  Requests that arrive while earlier
// windows run are admitted into the next window as slots and memory free up,
// and all requests of a window run in one kernel launch.
//
// Result semantics are those of serial replay in arrival order: a lookup sees
// exactly the inserts on its filter that arrived before it.  Within a window
// the requests of each filter are split into phases at every change of
// operation (insert run, lookup run, insert run, ...); phase p of all filters
// runs in one launch, phases in order, so inserts that arrived later never
// reach an earlier lookup and every earlier insert does.
//
// Residency: a filter lives in device memory while admitted; to admit another
// filter under the budget the scheduler evicts the least recently used
// resident filter that the forming window does not use: its words are copied
// to pinned host memory and its device memory freed, both ordered on the
// stream after every window that used it.  A filter never written is
// admitted by zero-filling.  The budget counts resident filters plus the
// device-resident hash and result buffers of admitted requests.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdint>
#include <cstring>
#include <deque>
#include <mutex>
#include <set>
#include <thread>
#include <utility>
#include <vector>

#include "sbbf.h"
#include "sbbf_device.cuh"
#include "sbbf_host.cuh"

namespace sbbf {
sbbf_status launch_insert(uint32_t* words, uint32_t num_blocks, const uint64_t* d_hashes,
                          uint64_t n, cudaStream_t s);
sbbf_status launch_find(const uint32_t* words, uint32_t num_blocks, const uint64_t* d_hashes,
                        uint64_t n, uint32_t* d_out, cudaStream_t s);
sbbf_status launch_clear(uint32_t* dst, uint64_t n_words, cudaStream_t s);

namespace {

// Device descriptor of one admitted request (40 bytes).
struct ReqDesc {
  const uint64_t* hashes;
  uint32_t* out;
  uint32_t* words;
  uint64_t n;
  uint32_t num_blocks;
  uint32_t op;
};

// ---- the window kernel ------------------------------------------------------
//
// Work unit: one 64-hash chunk of one request; chunk_off[r] is the first
// chunk of request r (prefix sums of ceil(n_r / 64)).  Inserts use 8 lanes per
// key (red.or.b32 per lane), lookups one lane per key (256-bit block load);
// results are packed per request from its own first output word.

__global__ void __launch_bounds__(256)
    serve_kernel(const ReqDesc* __restrict__ reqs, const uint64_t* __restrict__ chunk_off,
                 uint32_t n_reqs, uint64_t chunk_begin, uint64_t chunk_end) {
  const unsigned lane = lane_id();
  const uint64_t warp = (static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const uint64_t n_warps = (static_cast<uint64_t>(gridDim.x) * blockDim.x) >> 5;
  const uint64_t pk = policy_evict_first();
  const uint32_t seed = lane_seed(lane & 7);
  const int group_base = static_cast<int>(lane & ~7u);
  uint32_t r = 0;
  uint64_t r_lo = 0, r_hi = 0;  // cached chunk range of request r
  for (uint64_t u = chunk_begin + warp; u < chunk_end; u += n_warps) {
    if (!(u >= r_lo && u < r_hi)) {  // last r with chunk_off[r] <= u
      uint32_t lo = 0, hi = n_reqs;
      while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (__ldg(chunk_off + mid) <= u) lo = mid; else hi = mid;
      }
      r = lo;
      r_lo = __ldg(chunk_off + r);
      r_hi = __ldg(chunk_off + r + 1);
    }
    const ReqDesc d = reqs[r];
    const uint64_t k = (u - r_lo) * 64 + 2 * lane;
    const bool vec = (reinterpret_cast<uintptr_t>(d.hashes) & 15) == 0;
    uint64_t h0 = 0, h1 = 0;
    if (vec && k + 1 < d.n) {
      load_keys2(d.hashes + k, pk, h0, h1);
    } else {
      if (k < d.n) h0 = load_key1(d.hashes + k, pk);
      if (k + 1 < d.n) h1 = load_key1(d.hashes + k + 1, pk);
    }
    const uint64_t b0 = k < d.n ? block_of(h0, d.num_blocks) : ~0ull;
    const uint64_t b1 = k + 1 < d.n ? block_of(h1, d.num_blocks) : ~0ull;
    if (d.op == SBBF_OP_INSERT) {
      uint32_t* const word_j = d.words + (lane & 7);
      const uint32_t x0 = static_cast<uint32_t>(h0), x1 = static_cast<uint32_t>(h1);
#pragma unroll
      for (int rr = 0; rr < 16; ++rr) {
        const int src = group_base + (rr >> 1);
        const uint32_t x = __shfl_sync(0xFFFFFFFFu, (rr & 1) ? x1 : x0, src);
        const uint64_t b = __shfl_sync(0xFFFFFFFFu, (rr & 1) ? b1 : b0, src);
        if (b != ~0ull) red_or(word_j + 8ull * b, 1u << bit_index(x, seed));
      }
    } else {
      uint32_t w0[8], w1[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) w0[i] = w1[i] = 0;
      if (b0 != ~0ull) load_block(d.words + 8ull * b0, pk, w0);
      if (b1 != ~0ull) load_block(d.words + 8ull * b1, pk, w1);
      const uint32_t r0 = block_has(w0, static_cast<uint32_t>(h0));
      const uint32_t r1 = block_has(w1, static_cast<uint32_t>(h1));
      const uint32_t v = (r0 | (r1 << 1)) << (2 * (lane & 15));
      const uint32_t lo = __reduce_or_sync(0xFFFFFFFFu, lane < 16 ? v : 0u);
      const uint32_t hi = __reduce_or_sync(0xFFFFFFFFu, lane >= 16 ? v : 0u);
      const uint64_t word = (u - r_lo) * 2;
      const uint64_t n_out = (d.n + 31) >> 5;
      const uint32_t lo1[1] = {lo}, hi1[1] = {hi};
      store_answers<1>(d.out, n_out, word, lo1, hi1, lane, false,
                       (reinterpret_cast<uintptr_t>(d.out) & 7) == 0);
    }
  }
}

uint64_t now_ns() {
  return static_cast<uint64_t>(std::chrono::duration_cast<std::chrono::nanoseconds>(
                                   std::chrono::steady_clock::now().time_since_epoch())
                                   .count());
}

bool device_resident(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Runs of one operation a filter may contribute to one window; each run is
// a phase (a launch), so this bounds the launches of a window.
constexpr int kMaxRunsPerFilter = 4;
// Windows after an eviction or a refused admission during which filters
// drain their whole backlog instead of kMaxRunsPerFilter runs.
constexpr int kPressureWindows = 16;

// A non-resident filter whose oldest request has waited this long is
// admitted in the same pass as the resident filters and may evict a filter
// that still has queued requests.
constexpr uint64_t kAdmitAgeNs = 50000000;

struct Pending {
  sbbf_request_t req;
  uint64_t ticket;
  uint64_t dev_bytes;  // device-resident payload + result bytes (budgeted)
  uint64_t t_submit;   // steady-clock ns at submission
};

struct FilterState {
  uint32_t num_blocks = 0;
  uint32_t* d_words = nullptr;  // device copy while resident
  uint32_t* h_words = nullptr;  // pinned host copy after an eviction
  bool written = false;         // ever inserted into
  bool host_valid = false;      // h_words equals the current contents
  uint64_t last_use = 0;        // window sequence number of its last use
  uint64_t bytes() const { return static_cast<uint64_t>(num_blocks) * 32; }
};

struct WindowSlot {
  ReqDesc* h_desc = nullptr;  // pinned staging
  uint64_t* h_off = nullptr;
  ReqDesc* d_desc = nullptr;
  uint64_t* d_off = nullptr;
  cudaEvent_t done = nullptr;
  bool busy = false;
};

struct Window {
  int slot;
  std::vector<uint64_t> tickets;
  uint64_t dev_bytes;
  uint64_t keys;
};

}  // namespace
}  // namespace sbbf

using namespace sbbf;

struct sbbf_server {
  sbbf_server_config_t cfg;
  int device = 0;
  cudaStream_t stream = nullptr;
  std::mutex mu;
  std::condition_variable cv;
  // Queued requests per filter in arrival order, and the filters ordered by
  // the ticket of their oldest queued request.
  std::vector<std::deque<Pending>> queues;
  std::set<std::pair<uint64_t, uint32_t>> heads;
  uint64_t n_pending = 0;
  int pressure = 0;  // windows left in "memory pressure" mode (see launch_window)
  std::vector<FilterState> filters;
  std::vector<uint64_t> done_ns;   // per ticket: completion time, 0 while pending
  std::vector<int> status;         // per ticket: SBBF_OK or an error
  std::deque<Window> inflight;
  std::vector<WindowSlot> slots;
  uint64_t resident_bytes = 0, inflight_bytes = 0, window_seq = 0;
  sbbf_server_stats_t stats = {};
  sbbf_status error = SBBF_OK;  // sticky device error
  bool stop = false;
  bool paused = false;          // serial replay owns the stream
  std::thread worker;
};

namespace {

// Frees device memory of filter f after copying its words to pinned host
// memory; both stream-ordered after all earlier work.
sbbf_status evict(sbbf_server_t* s, uint32_t f) {
  FilterState& st = s->filters[f];
  if (st.written && !st.host_valid) {  // write back only what changed since admission
    if (!st.h_words) {
      cudaError_t e = cudaMallocHost(&st.h_words, st.bytes());
      if (e != cudaSuccess) {
        st.h_words = nullptr;
        return record_cuda(e);
      }
    }
    SBBF_CUDA(cudaMemcpyAsync(st.h_words, st.d_words, st.bytes(), cudaMemcpyDeviceToHost,
                              s->stream));
    st.host_valid = true;
    ++s->stats.writebacks;
  }
  SBBF_CUDA(cudaFreeAsync(st.d_words, s->stream));
  st.d_words = nullptr;
  s->resident_bytes -= st.bytes();
  ++s->stats.evictions;
  return SBBF_OK;
}

sbbf_status admit(sbbf_server_t* s, uint32_t f) {
  FilterState& st = s->filters[f];
  cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&st.d_words), st.bytes(), s->stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    st.d_words = nullptr;
    return SBBF_ENOMEM;
  }
  if (st.written && st.h_words) {
    // host_valid holds: the host copy was written back at the last eviction
    SBBF_CUDA(cudaMemcpyAsync(st.d_words, st.h_words, st.bytes(), cudaMemcpyHostToDevice,
                              s->stream));
  } else {
    sbbf_status rc = launch_clear(st.d_words, static_cast<uint64_t>(st.num_blocks) * 8, s->stream);
    if (rc != SBBF_OK) return rc;
  }
  s->resident_bytes += st.bytes();
  ++s->stats.admissions;
  return SBBF_OK;
}

// Makes filter f resident within the budget, evicting LRU filters not in
// `in_window`.  `extra` is the budgeted bytes the caller adds besides.
// Returns SBBF_EBUSY when the budget cannot be met now.
sbbf_status make_resident(sbbf_server_t* s, uint32_t f, uint64_t extra,
                          const std::vector<char>& in_window, bool evict_queued = true) {
  FilterState& st = s->filters[f];
  const uint64_t need = (st.d_words ? 0 : st.bytes()) + extra;
  while (s->resident_bytes + s->inflight_bytes + need > s->cfg.budget_bytes) {
    // Least recently used resident filter outside the forming window,
    // preferring filters with no queued requests (they will not be needed
    // back soon).
    int victim = -1;
    for (size_t i = 0; i < s->filters.size(); ++i) {
      const FilterState& c = s->filters[i];
      if (!c.d_words || in_window[i] || i == f) continue;
      if (!evict_queued && !s->queues[i].empty()) continue;
      if (victim < 0) {
        victim = static_cast<int>(i);
        continue;
      }
      const FilterState& v = s->filters[victim];
      const bool c_idle = s->queues[i].empty(), v_idle = s->queues[victim].empty();
      if ((c_idle && !v_idle) || (c_idle == v_idle && c.last_use < v.last_use))
        victim = static_cast<int>(i);
    }
    if (victim < 0) return SBBF_EBUSY;
    sbbf_status rc = evict(s, static_cast<uint32_t>(victim));
    if (rc != SBBF_OK) return rc;
  }
  if (!st.d_words) {
    sbbf_status rc = admit(s, f);
    if (rc != SBBF_OK) return rc == SBBF_ENOMEM ? SBBF_EBUSY : rc;
  }
  return SBBF_OK;
}

// Forms and launches one window from the pending requests (lock held).
sbbf_status launch_window(sbbf_server_t* s, bool* launched) {
  SBBF_TRACE_NAMED("sbbf_server_window");
  *launched = false;
  int slot = -1;
  for (size_t i = 0; i < s->slots.size(); ++i)
    if (!s->slots[i].busy) {
      slot = static_cast<int>(i);
      break;
    }
  if (slot < 0) return SBBF_OK;
  WindowSlot& ws = s->slots[slot];
  std::vector<char> in_window(s->filters.size(), 0);
  std::vector<Pending> taken;
  uint64_t keys = 0, bytes = 0;
  // Filters in the order of their oldest queued request; each admitted filter
  // brings as many of its queued requests (in order) as the window holds, so
  // one admission serves a filter's whole backlog.  A filter that cannot be
  // made resident now keeps its requests queued; other filters proceed.
  // Pass 0 takes resident filters (and non-resident ones that waited longer
  // than kAdmitAgeNs); pass 1 admits the others, evicting only then.
  std::vector<std::pair<uint64_t, uint32_t>> done_heads, new_heads;
  const uint64_t now = now_ns();
  bool full = false;
  for (int pass = 0; pass < 2 && !full; ++pass) {
  size_t scanned = 0;
  const size_t scan_limit = static_cast<size_t>(s->cfg.max_window_requests) + 64;
  for (auto it = s->heads.begin(); it != s->heads.end() &&
                                   taken.size() < s->cfg.max_window_requests &&
                                   scanned < scan_limit;
       ++it, ++scanned) {
    const uint32_t f = it->second;
    if (in_window[f]) continue;  // taken in pass 0
    std::deque<Pending>& q = s->queues[f];
    const bool resident = s->filters[f].d_words != nullptr;
    const bool aged = now - q.front().t_submit >= kAdmitAgeNs;
    if (pass == 0 && !resident && !aged) continue;
    if (!taken.empty() && keys + q.front().req.n > s->cfg.max_window_keys) {
      full = true;
      break;
    }
    // Only a request that waited kAdmitAgeNs may push out a filter that
    // still has queued requests; otherwise backlogged filters drain first.
    const uint64_t evictions_before = s->stats.evictions;
    sbbf_status rc = make_resident(s, f, bytes + q.front().dev_bytes, in_window, aged);
    if (s->stats.evictions != evictions_before) s->pressure = kPressureWindows;
    if (rc == SBBF_EBUSY) {
      ++s->stats.admission_waits;
      s->pressure = kPressureWindows;
      continue;
    }
    if (rc != SBBF_OK) return rc;
    in_window[f] = 1;
    int runs = 0;
    uint32_t last_op = ~0u;
    // Under memory pressure a resident filter drains its whole backlog, so
    // each admission serves as many requests as possible.
    const int max_runs = s->pressure > 0 ? 1 << 30 : kMaxRunsPerFilter;
    while (!q.empty() && taken.size() < s->cfg.max_window_requests) {
      const Pending& p = q.front();
      if (!taken.empty() && keys + p.req.n > s->cfg.max_window_keys) break;
      if (p.req.op != last_op) {  // a new run of this filter: one more phase
        if (runs == max_runs) break;
        ++runs;
        last_op = p.req.op;
      }
      if (s->resident_bytes + s->inflight_bytes + bytes + p.dev_bytes > s->cfg.budget_bytes) break;
      keys += p.req.n;
      bytes += p.dev_bytes;
      taken.push_back(p);
      q.pop_front();
      --s->n_pending;
    }
    done_heads.push_back(*it);
    if (!q.empty()) new_heads.push_back({q.front().ticket, f});
  }
  if (taken.size() >= s->cfg.max_window_requests) full = true;
  }
  for (const auto& h : done_heads) s->heads.erase(h);
  for (const auto& h : new_heads) s->heads.insert(h);
  if (taken.empty()) return SBBF_OK;
  if (s->pressure > 0) --s->pressure;
  const uint64_t seq = ++s->window_seq;
  // Phases: per filter, a new phase at every change of operation.
  std::vector<int> last_op(s->filters.size(), -1), phase_of(s->filters.size(), 0);
  std::vector<int> phase(taken.size());
  int n_phases = 1;
  for (size_t i = 0; i < taken.size(); ++i) {
    const uint32_t f = taken[i].req.filter;
    if (last_op[f] >= 0 && static_cast<int>(taken[i].req.op) != last_op[f]) ++phase_of[f];
    last_op[f] = static_cast<int>(taken[i].req.op);
    phase[i] = phase_of[f];
    n_phases = std::max(n_phases, phase[i] + 1);
    s->filters[f].last_use = seq;
    if (taken[i].req.op == SBBF_OP_INSERT) {
      s->filters[f].written = true;
      s->filters[f].host_valid = false;
    }
  }
  std::vector<size_t> order(taken.size());
  for (size_t i = 0; i < order.size(); ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t b) { return phase[a] < phase[b]; });
  // Descriptors, chunk offsets and per-phase ranges.
  std::vector<uint32_t> phase_first(n_phases + 1, 0);
  uint64_t chunks = 0;
  for (size_t j = 0; j < order.size(); ++j) {
    const Pending& p = taken[order[j]];
    const FilterState& st = s->filters[p.req.filter];
    ws.h_desc[j] = ReqDesc{p.req.d_hashes, p.req.d_out_bits, st.d_words, p.req.n, st.num_blocks,
                           p.req.op};
    ws.h_off[j] = chunks;
    chunks += (p.req.n + 63) / 64;
    phase_first[phase[order[j]] + 1] = static_cast<uint32_t>(j + 1);
  }
  ws.h_off[order.size()] = chunks;
  for (int p = 1; p <= n_phases; ++p) phase_first[p] = std::max(phase_first[p], phase_first[p - 1]);
  const size_t nr = order.size();
  SBBF_CUDA(cudaMemcpyAsync(ws.d_desc, ws.h_desc, nr * sizeof(ReqDesc), cudaMemcpyHostToDevice,
                            s->stream));
  SBBF_CUDA(cudaMemcpyAsync(ws.d_off, ws.h_off, (nr + 1) * sizeof(uint64_t),
                            cudaMemcpyHostToDevice, s->stream));
  static int occ = occupancy(serve_kernel, 256);
  for (int p = 0; p < n_phases; ++p) {
    const uint32_t a = phase_first[p], b = phase_first[p + 1];
    if (a == b) continue;
    const uint64_t c0 = ws.h_off[a], c1 = ws.h_off[b];
    if (c1 == c0) continue;
    serve_kernel<<<grid_for(c1 - c0, 8, occ), 256, 0, s->stream>>>(
        ws.d_desc, ws.d_off, static_cast<uint32_t>(nr), c0, c1);
    sbbf_status rc = launch_status();
    if (rc != SBBF_OK) return rc;
    ++s->stats.launches;
  }
  SBBF_CUDA(cudaEventRecord(ws.done, s->stream));
  ws.busy = true;
  Window w;
  w.slot = slot;
  w.dev_bytes = bytes;
  w.keys = keys;
  for (const Pending& p : taken) w.tickets.push_back(p.ticket);
  s->inflight_bytes += bytes;
  s->inflight.push_back(std::move(w));
  ++s->stats.windows;
  s->stats.requests += taken.size();
  s->stats.keys += keys;
  s->stats.phases += static_cast<uint64_t>(n_phases);
  *launched = true;
  return SBBF_OK;
}

// Retires finished windows in order (lock held).
void collect(sbbf_server_t* s) {
  while (!s->inflight.empty()) {
    Window& w = s->inflight.front();
    WindowSlot& ws = s->slots[w.slot];
    const cudaError_t e = cudaEventQuery(ws.done);
    if (e == cudaErrorNotReady) break;
    const uint64_t t = now_ns();
    const int st = e == cudaSuccess ? SBBF_OK : record_cuda(e);
    if (st != SBBF_OK) s->error = static_cast<sbbf_status>(st);
    for (uint64_t tk : w.tickets) {
      s->done_ns[tk] = t;
      s->status[tk] = st;
    }
    s->inflight_bytes -= w.dev_bytes;
    ws.busy = false;
    s->inflight.pop_front();
  }
}

void worker_loop(sbbf_server_t* s) {
  cudaSetDevice(s->device);
  std::unique_lock<std::mutex> lk(s->mu);
  for (;;) {
    collect(s);
    if (s->stop && s->n_pending == 0 && s->inflight.empty()) break;
    bool launched = false;
    if (!s->paused && s->n_pending > 0 &&
        s->inflight.size() < s->cfg.max_inflight_windows && s->error == SBBF_OK) {
      const sbbf_status rc = guarded([&] { return launch_window(s, &launched); });
      if (rc != SBBF_OK) s->error = rc;  // sticky: waiters return it
    }
    if (launched) {
      s->cv.notify_all();
      continue;
    }
    if (s->inflight.empty()) {
      s->cv.notify_all();
      s->cv.wait_for(lk, std::chrono::milliseconds(2));
    } else {
      lk.unlock();  // a window is on the GPU: poll again shortly
      std::this_thread::sleep_for(std::chrono::microseconds(2));
      lk.lock();
    }
  }
  s->cv.notify_all();
}

void free_server(sbbf_server_t* s) {
  for (FilterState& f : s->filters) {
    if (f.d_words) cudaFree(f.d_words);
    if (f.h_words) cudaFreeHost(f.h_words);
  }
  for (WindowSlot& w : s->slots) {
    if (w.h_desc) cudaFreeHost(w.h_desc);
    if (w.h_off) cudaFreeHost(w.h_off);
    if (w.d_desc) cudaFree(w.d_desc);
    if (w.d_off) cudaFree(w.d_off);
    if (w.done) cudaEventDestroy(w.done);
  }
  if (s->stream) cudaStreamDestroy(s->stream);
  delete s;
}

sbbf_status wait_ticket(sbbf_server_t* s, std::unique_lock<std::mutex>& lk, uint64_t ticket,
                        uint64_t deadline) {
  while (s->done_ns[ticket] == 0) {
    if (s->error != SBBF_OK) return s->error;
    if (deadline && now_ns() >= deadline) return SBBF_ETIMEOUT;
    s->cv.wait_for(lk, std::chrono::microseconds(200));
  }
  return static_cast<sbbf_status>(s->status[ticket]);
}

}  // namespace

namespace {

// Makes room for one more element ahead of the push_back, so that the push
// cannot throw after other state changed; the capacity grows geometrically
// (a bare reserve(size() + 1) reallocates and copies on every call).
template <class V>
void reserve_one_more(V& v) {
  if (v.size() == v.capacity()) v.reserve(v.capacity() ? 2 * v.capacity() : 64);
}

}  // namespace

extern "C" {

sbbf_status sbbf_server_create(const sbbf_server_config_t* cfg, sbbf_server_t** out) {
  if (!cfg || !out || cfg->max_window_requests == 0 || cfg->max_window_keys == 0 ||
      cfg->max_inflight_windows == 0 || cfg->max_pending_requests == 0)
    return SBBF_EINVAL;
  *out = nullptr;
  sbbf_server_t* s = new (std::nothrow) sbbf_server_t();
  if (!s) return SBBF_ENOMEM;
  s->cfg = *cfg;
  s->device = current_device();
  cudaError_t e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
  s->slots.resize(cfg->max_inflight_windows);
  for (WindowSlot& w : s->slots) {
    const size_t nr = cfg->max_window_requests;
    if (e == cudaSuccess) e = cudaMallocHost(&w.h_desc, nr * sizeof(ReqDesc));
    if (e == cudaSuccess) e = cudaMallocHost(&w.h_off, (nr + 1) * sizeof(uint64_t));
    if (e == cudaSuccess) e = cudaMalloc(&w.d_desc, nr * sizeof(ReqDesc));
    if (e == cudaSuccess) e = cudaMalloc(&w.d_off, (nr + 1) * sizeof(uint64_t));
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&w.done, cudaEventDisableTiming);
  }
  if (e != cudaSuccess) {
    free_server(s);
    return record_cuda(e);
  }
  // Keep freed filter memory in the stream-ordered pool between evictions.
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, s->device) == cudaSuccess) {
    uint64_t keep = UINT64_MAX;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
  }
  try {
    s->worker = std::thread(worker_loop, s);
  } catch (...) {
    free_server(s);
    return SBBF_ENOMEM;
  }
  *out = s;
  return SBBF_OK;
}

sbbf_status sbbf_server_destroy(sbbf_server_t* s) {
  if (!s) return SBBF_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    s->paused = false;
  }
  s->cv.notify_all();
  if (s->worker.joinable()) s->worker.join();
  const cudaError_t e = cudaStreamSynchronize(s->stream);
  free_server(s);
  return e == cudaSuccess ? SBBF_OK : record_cuda(e);
}

sbbf_status sbbf_server_add_filter(sbbf_server_t* s, uint32_t num_blocks, uint32_t* id) {
  return guarded([&]() -> sbbf_status {
    if (!s || !id || num_blocks == 0) return SBBF_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    FilterState f;
    f.num_blocks = num_blocks;
    reserve_one_more(s->filters);
    reserve_one_more(s->queues);
    s->filters.push_back(f);
    s->queues.emplace_back();
    *id = static_cast<uint32_t>(s->filters.size() - 1);
    return SBBF_OK;
  });
}

sbbf_status sbbf_server_submit(sbbf_server_t* s, const sbbf_request_t* r, uint64_t* ticket) {
  return guarded([&]() -> sbbf_status {
    if (!s || !r || !ticket) return SBBF_EINVAL;
    if (r->op != SBBF_OP_INSERT && r->op != SBBF_OP_FIND) return SBBF_EINVAL;
    if (r->n > 0 && (!r->d_hashes || (r->op == SBBF_OP_FIND && !r->d_out_bits))) return SBBF_EINVAL;
    if ((reinterpret_cast<uintptr_t>(r->d_hashes) & 7) || (reinterpret_cast<uintptr_t>(r->d_out_bits) & 3))
      return SBBF_EINVAL;
    Pending p;
    p.req = *r;
    p.dev_bytes = 0;
    p.t_submit = now_ns();
    if (r->n && device_resident(r->d_hashes)) p.dev_bytes += 8 * r->n;
    if (r->n && r->op == SBBF_OP_FIND && device_resident(r->d_out_bits)) p.dev_bytes += 4 * ((r->n + 31) / 32);
    {
      std::lock_guard<std::mutex> lk(s->mu);
      if (r->filter >= s->filters.size()) return SBBF_EINVAL;
      if (s->error != SBBF_OK) return s->error;
      if (s->n_pending >= s->cfg.max_pending_requests) return SBBF_EBUSY;
      if (s->filters[r->filter].bytes() + p.dev_bytes > s->cfg.budget_bytes) return SBBF_EBUSY;
      p.ticket = s->done_ns.size();
      // every step that can throw comes before the first change of state
      reserve_one_more(s->done_ns);
      reserve_one_more(s->status);
      if (r->n > 0) {
        std::deque<Pending>& q = s->queues[r->filter];
        const bool was_empty = q.empty();
        q.push_back(p);
        if (was_empty) {
          try {
            s->heads.insert({p.ticket, r->filter});
          } catch (...) {
            q.pop_back();
            throw;
          }
        }
        ++s->n_pending;
      }
      s->done_ns.push_back(r->n == 0 ? now_ns() : 0);
      s->status.push_back(SBBF_OK);
      *ticket = p.ticket;
    }
    s->cv.notify_all();
    return SBBF_OK;
  });
}

sbbf_status sbbf_server_poll(sbbf_server_t* s, uint64_t ticket, int* done) {
  return guarded([&]() -> sbbf_status {
    if (!s || !done) return SBBF_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    if (ticket >= s->done_ns.size()) return SBBF_EINVAL;
    *done = s->done_ns[ticket] != 0;
    return *done ? static_cast<sbbf_status>(s->status[ticket]) : SBBF_OK;
  });
}

sbbf_status sbbf_server_wait(sbbf_server_t* s, uint64_t ticket, uint64_t timeout_ns) {
  return guarded([&]() -> sbbf_status {
    if (!s) return SBBF_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    if (ticket >= s->done_ns.size()) return SBBF_EINVAL;
    return wait_ticket(s, lk, ticket, timeout_ns ? now_ns() + timeout_ns : 0);
  });
}

sbbf_status sbbf_server_drain(sbbf_server_t* s, uint64_t timeout_ns) {
  return guarded([&]() -> sbbf_status {
    if (!s) return SBBF_EINVAL;
    const uint64_t deadline = timeout_ns ? now_ns() + timeout_ns : 0;
    std::unique_lock<std::mutex> lk(s->mu);
    while (s->n_pending > 0 || !s->inflight.empty()) {
      if (s->error != SBBF_OK) return s->error;
      if (deadline && now_ns() >= deadline) return SBBF_ETIMEOUT;
      s->cv.wait_for(lk, std::chrono::microseconds(200));
    }
    return s->error;
  });
}

sbbf_status sbbf_server_copy_filter(sbbf_server_t* s, uint32_t id, uint32_t* h_words, size_t bytes) {
  return guarded([&]() -> sbbf_status {
    if (!s || !h_words) return SBBF_EINVAL;
    sbbf_status rc = sbbf_server_drain(s, 0);
    if (rc != SBBF_OK) return rc;
    std::lock_guard<std::mutex> lk(s->mu);
    if (id >= s->filters.size()) return SBBF_EINVAL;
    const FilterState& f = s->filters[id];
    if (bytes < f.bytes()) return SBBF_EINVAL;
    if (f.d_words) {
      SBBF_CUDA(cudaMemcpyAsync(h_words, f.d_words, f.bytes(), cudaMemcpyDeviceToHost, s->stream));
      SBBF_CUDA(cudaStreamSynchronize(s->stream));
    } else {
      SBBF_CUDA(cudaStreamSynchronize(s->stream));  // a pending eviction copy
      if (f.written && f.h_words) std::memcpy(h_words, f.h_words, f.bytes());
      else std::memset(h_words, 0, f.bytes());
    }
    return SBBF_OK;
  });
}

sbbf_status sbbf_server_prefill(sbbf_server_t* s, uint32_t id, const uint64_t* d_hashes, size_t n) {
  return guarded([&]() -> sbbf_status {
    if (!s) return SBBF_EINVAL;
    sbbf_status rc = sbbf_server_drain(s, 0);
    if (rc != SBBF_OK) return rc;
    std::lock_guard<std::mutex> lk(s->mu);
    if (id >= s->filters.size() || (n && !d_hashes)) return SBBF_EINVAL;
    std::vector<char> none(s->filters.size(), 0);
    rc = make_resident(s, id, 0, none);
    if (rc != SBBF_OK) return rc;
    FilterState& f = s->filters[id];
    f.written = true;
    f.host_valid = false;
    f.last_use = ++s->window_seq;
    rc = launch_insert(f.d_words, f.num_blocks, d_hashes, n, s->stream);
    if (rc != SBBF_OK) return rc;
    SBBF_CUDA(cudaStreamSynchronize(s->stream));
    return SBBF_OK;
  });
}

sbbf_status sbbf_server_stats(sbbf_server_t* s, sbbf_server_stats_t* out) {
  return guarded([&]() -> sbbf_status {
    if (!s || !out) return SBBF_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    *out = s->stats;
    out->resident_bytes = s->resident_bytes;
    return SBBF_OK;
  });
}

sbbf_status sbbf_server_replay(sbbf_server_t* s, const sbbf_request_t* reqs,
                               const uint64_t* arrival_ns, size_t n, uint64_t* latency_ns) {
  return guarded([&]() -> sbbf_status {
    if (!s || (n && (!reqs || !arrival_ns || !latency_ns))) return SBBF_EINVAL;
    std::vector<uint64_t> tickets(n);
    const uint64_t t0 = now_ns();
    for (size_t i = 0; i < n; ++i) {
      while (now_ns() < t0 + arrival_ns[i]) {
      }  // arrival time of request i
      sbbf_status rc;
      while ((rc = sbbf_server_submit(s, &reqs[i], &tickets[i])) == SBBF_EBUSY &&
             s->cfg.max_pending_requests > 0) {
        std::this_thread::sleep_for(std::chrono::microseconds(5));  // queue full: back-pressure
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->error != SBBF_OK) return s->error;
        if (s->filters[reqs[i].filter].bytes() > s->cfg.budget_bytes) return SBBF_EBUSY;
      }
      if (rc != SBBF_OK) return rc;
    }
    std::unique_lock<std::mutex> lk(s->mu);
    for (size_t i = 0; i < n; ++i) {
      sbbf_status rc = wait_ticket(s, lk, tickets[i], 0);
      if (rc != SBBF_OK) return rc;
      latency_ns[i] = s->done_ns[tickets[i]] - (t0 + arrival_ns[i]);
    }
    return SBBF_OK;
  });
}

sbbf_status sbbf_server_replay_serial(sbbf_server_t* s, const sbbf_request_t* reqs,
                                      const uint64_t* arrival_ns, size_t n,
                                      uint64_t* latency_ns) {
  return guarded([&]() -> sbbf_status {
    if (!s || (n && (!reqs || !arrival_ns || !latency_ns))) return SBBF_EINVAL;
    sbbf_status rc = sbbf_server_drain(s, 0);
    if (rc != SBBF_OK) return rc;
    {
      std::lock_guard<std::mutex> lk(s->mu);
      s->paused = true;  // this thread owns the stream until the replay ends
    }
    constexpr size_t kEvents = 1024;
    std::vector<cudaEvent_t> ev(kEvents, nullptr);
    cudaError_t e = cudaSuccess;
    for (auto& x : ev)
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&x, cudaEventDisableTiming);
    size_t done = 0, launched = 0;  // only recorded events are ever queried
    const uint64_t t0 = now_ns();
    auto retire = [&](bool block) -> sbbf_status {  // stamps finished requests in order
      while (done < launched) {
        const cudaError_t q = block ? cudaEventSynchronize(ev[done % kEvents])
                                    : cudaEventQuery(ev[done % kEvents]);
        if (q == cudaErrorNotReady) return SBBF_OK;
        if (q != cudaSuccess) return record_cuda(q);
        latency_ns[done] = now_ns() - (t0 + arrival_ns[done]);
        ++done;
        if (block) return SBBF_OK;
      }
      return SBBF_OK;
    };
    rc = e == cudaSuccess ? SBBF_OK : record_cuda(e);
    for (size_t i = 0; i < n && rc == SBBF_OK; ++i) {
      while (now_ns() < t0 + arrival_ns[i]) {
        rc = retire(false);
        if (rc != SBBF_OK) break;
      }
      if (rc != SBBF_OK) break;
      while (i - done >= kEvents && rc == SBBF_OK) rc = retire(true);  // event ring full
      if (rc != SBBF_OK) break;
      std::lock_guard<std::mutex> lk(s->mu);
      const sbbf_request_t& r = reqs[i];
      if (r.filter >= s->filters.size()) {
        rc = SBBF_EINVAL;
        break;
      }
      std::vector<char> none(s->filters.size(), 0);
      rc = make_resident(s, r.filter, 0, none);
      if (rc != SBBF_OK) break;
      FilterState& f = s->filters[r.filter];
      f.last_use = ++s->window_seq;
      if (r.n) {
        if (r.op == SBBF_OP_INSERT) {
          f.written = true;
          f.host_valid = false;
          rc = launch_insert(f.d_words, f.num_blocks, r.d_hashes, r.n, s->stream);
        } else {
          rc = launch_find(f.d_words, f.num_blocks, r.d_hashes, r.n, r.d_out_bits, s->stream);
        }
        ++s->stats.launches;
      }
      if (rc == SBBF_OK) {
        const cudaError_t er = cudaEventRecord(ev[i % kEvents], s->stream);
        if (er != cudaSuccess) rc = record_cuda(er);
        else launched = i + 1;
      }
    }
    while (rc == SBBF_OK && done < launched) rc = retire(true);
    for (auto& x : ev)
      if (x) cudaEventDestroy(x);
    {
      std::lock_guard<std::mutex> lk(s->mu);
      s->paused = false;
    }
    s->cv.notify_all();
    return rc;
  });
}

}  // extern "C"
