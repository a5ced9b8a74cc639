// Filters to and from host byte buffers (not in the paper, whose adopters
// store filters on disk; see the list of systems using the design).
//
// Native checkpoint format: a 64-byte little-endian header, then the filter
// words in the library's layout.
//   0  'S' 'B' 'B' 'F'
//   4  u32 format version (1)
//   8  u32 lanes (4, 8 or 16 words per block)
//  12  u32 num_blocks
//  16  u64 layout digest: XXH64 (seed 0) of the lanes' seeds as little-endian
//      uint32, lane 0 first -- a filter only means something with the seeds
//      and lane order it was built with, so a change of either is detected
//  24  u64 payload bytes (num_blocks * lanes * 4)
//  32  u64 XXH64 (seed 0) of the payload
//  40  24 zero bytes
//
// Parquet's Bloom-filter format: a Thrift compact-protocol BloomFilterHeader
// {1: i32 numBytes, 2: algorithm {1: BLOCK {}}, 3: hash {1: XXHASH {}},
// 4: compression {1: UNCOMPRESSED {}}} followed by numBytes of bitset.
// Parquet's blocks are eight little-endian uint32 words like this library's,
// but it lists the eight salts in the order the paper's text prints the
// appendix constants, which swaps each adjacent pair of the appendix's
// little-endian lane order: Parquet word 2j + 1 is this library's word 2j and
// vice versa.  Export and import apply that swap on the device.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdlib>
#include <cstring>

#include "sbbf.h"
#include "sbbf_device.cuh"
#include "sbbf_host.cuh"
#include "sbbf_keys.cuh"

namespace sbbf {

constexpr size_t kNativeHeader = 64;
constexpr uint32_t kFormatVersion = 1;
constexpr size_t kStagingBytes = 64ull << 20;

// Lane seeds on the host, for the layout digest (lanes 0..7: appendix seeds;
// 8..15: the sixteen-lane extension).
constexpr uint32_t kHostSeeds[16] = {
    SBBF_SEED0,  SBBF_SEED1,  SBBF_SEED2,  SBBF_SEED3,  SBBF_SEED4,  SBBF_SEED5,
    SBBF_SEED6,  SBBF_SEED7,  0xe220a839u, 0x6e789e6bu, 0x06c45d19u, 0xf88bb8a9u,
    0x1b39896bu, 0x53cb9f0du, 0x2c829abfu, 0xc584133bu};

static void put32(uint8_t* p, uint32_t v) {
  for (int i = 0; i < 4; ++i) p[i] = static_cast<uint8_t>(v >> (8 * i));
}
static void put64(uint8_t* p, uint64_t v) {
  for (int i = 0; i < 8; ++i) p[i] = static_cast<uint8_t>(v >> (8 * i));
}
static uint32_t get32(const uint8_t* p) {
  uint32_t v = 0;
  for (int i = 3; i >= 0; --i) v = (v << 8) | p[i];
  return v;
}
static uint64_t get64(const uint8_t* p) {
  uint64_t v = 0;
  for (int i = 7; i >= 0; --i) v = (v << 8) | p[i];
  return v;
}

static uint64_t layout_digest(uint32_t lanes) {
  uint8_t b[64];
  for (uint32_t i = 0; i < lanes; ++i) put32(b + 4 * i, kHostSeeds[i]);
  return xxh::hash_bytes_host(b, 4ull * lanes, 0);
}

// out[i] = in[i] with its two 32-bit halves exchanged (words 2j <-> 2j+1);
// in == out is allowed.
__global__ void swap_pairs_kernel(const uint2* in, uint2* out, uint64_t n2) {
  const uint64_t stride = static_cast<uint64_t>(gridDim.x) * blockDim.x;
  for (uint64_t i = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n2;
       i += stride) {
    const uint2 v = in[i];
    out[i] = make_uint2(v.y, v.x);
  }
}

static sbbf_status launch_swap(const uint32_t* in, uint32_t* out, uint64_t n_words,
                               cudaStream_t s) {
  static int occ = occupancy(swap_pairs_kernel, 256);
  const uint64_t n2 = n_words / 2;
  swap_pairs_kernel<<<grid_for(n2, 256, occ), 256, 0, s>>>(reinterpret_cast<const uint2*>(in),
                                                            reinterpret_cast<uint2*>(out), n2);
  return launch_status();
}

// ---- Thrift compact protocol (the subset a BloomFilterHeader needs) ------------

struct ThriftReader {
  const uint8_t* p;
  size_t n, i;
  bool ok;

  uint8_t byte() {
    if (i >= n) {
      ok = false;
      return 0;
    }
    return p[i++];
  }
  uint64_t varint() {
    uint64_t v = 0;
    for (int sh = 0; sh < 64; sh += 7) {
      const uint8_t b = byte();
      if (!ok) return 0;
      v |= static_cast<uint64_t>(b & 0x7f) << sh;
      if (!(b & 0x80)) return v;
    }
    ok = false;
    return 0;
  }
  int64_t zigzag() {
    const uint64_t v = varint();
    return static_cast<int64_t>(v >> 1) ^ -static_cast<int64_t>(v & 1);
  }
  // Reads a field header; false at the struct's stop byte or on error.
  bool field(int& id, int& type, int& last) {
    const uint8_t b = byte();
    if (!ok || b == 0) return false;
    type = b & 0x0f;
    const int delta = b >> 4;
    id = delta ? last + delta : static_cast<int>(zigzag());
    last = id;
    return ok;
  }
  void skip(int type, int depth) {
    if (depth > 32) {
      ok = false;
      return;
    }
    switch (type) {
      case 1: case 2: return;          // bool in a field header
      case 3: byte(); return;          // byte
      case 4: case 5: case 6: varint(); return;  // i16, i32, i64
      case 7: advance(8); return;      // double
      case 8: advance(varint()); return;  // binary
      case 9: case 10: {               // list, set
        const uint8_t h = byte();
        uint64_t size = h >> 4;
        if (size == 15) size = varint();
        if (!ok || size > n - i) {
          ok = false;
          return;
        }
        const int et = h & 0x0f;
        for (uint64_t k = 0; k < size && ok; ++k) {
          if (et == 1 || et == 2) byte();  // bool elements take a byte each
          else skip(et, depth + 1);
        }
        return;
      }
      case 11: {  // map
        const uint64_t size = varint();
        if (!ok || size > n - i) {
          ok = false;
          return;
        }
        if (size == 0) return;
        const uint8_t kv = byte();
        for (uint64_t k = 0; k < size && ok; ++k) {
          skip(kv >> 4, depth + 1);
          skip(kv & 0x0f, depth + 1);
        }
        return;
      }
      case 12: {  // struct
        int id, t, last = 0;
        while (field(id, t, last)) skip(t, depth + 1);
        return;
      }
      default: ok = false;
    }
  }
  void advance(uint64_t k) {
    if (k > n - i) {
      ok = false;
      return;
    }
    i += k;
  }
  // A union struct whose member must be field 1 (itself an empty struct in
  // the header's unions).  Returns the member's id, or -1 on error.
  int union_member() {
    int id, t, last = 0, member = -1;
    while (field(id, t, last)) {
      if (t != 12 || member != -1) {
        ok = false;
        return -1;
      }
      member = id;
      skip(t, 1);
    }
    return ok ? member : -1;
  }
};

}  // namespace sbbf

using namespace sbbf;

extern "C" {

size_t sbbf_serialized_size(const sbbf_t* f) {
  return f ? kNativeHeader + static_cast<size_t>(filter_bytes(f)) : 0;
}

sbbf_status sbbf_serialize(const sbbf_t* f, void* h_buf, size_t bytes, sbbf_stream_t stream) {
  SBBF_TRACE();
  if (!f || !h_buf) return SBBF_EINVAL;
  const size_t payload = filter_bytes(f);
  if (bytes < kNativeHeader + payload) return SBBF_EINVAL;
  uint8_t* out = static_cast<uint8_t*>(h_buf);
  SBBF_CUDA(cudaMemcpyAsync(out + kNativeHeader, f->words, payload, cudaMemcpyDeviceToHost,
                            stream));
  SBBF_CUDA(cudaStreamSynchronize(stream));
  std::memset(out, 0, kNativeHeader);
  std::memcpy(out, "SBBF", 4);
  put32(out + 4, kFormatVersion);
  put32(out + 8, f->lanes);
  put32(out + 12, f->num_blocks);
  put64(out + 16, layout_digest(f->lanes));
  put64(out + 24, payload);
  put64(out + 32, xxh::hash_bytes_host(out + kNativeHeader, payload, 0));
  return SBBF_OK;
}

sbbf_status sbbf_deserialize(const void* h_buf, size_t bytes, sbbf_t** out) {
  SBBF_TRACE();
  if (!h_buf || !out) return SBBF_EINVAL;
  *out = nullptr;
  const uint8_t* in = static_cast<const uint8_t*>(h_buf);
  if (bytes < kNativeHeader || std::memcmp(in, "SBBF", 4) != 0) return SBBF_EINVAL;
  const uint32_t version = get32(in + 4), lanes = get32(in + 8), nb = get32(in + 12);
  if (version != kFormatVersion || (lanes != 4 && lanes != 8 && lanes != 16) || nb == 0)
    return SBBF_EINVAL;
  const uint64_t payload = static_cast<uint64_t>(nb) * lanes * 4;
  if (get64(in + 16) != layout_digest(lanes) || get64(in + 24) != payload) return SBBF_EINVAL;
  for (size_t i = 40; i < kNativeHeader; ++i)
    if (in[i] != 0) return SBBF_EINVAL;
  if (bytes - kNativeHeader < payload) return SBBF_EINVAL;
  if (get64(in + 32) != xxh::hash_bytes_host(in + kNativeHeader, payload, 0)) return SBBF_EINVAL;
  sbbf_t* f = nullptr;
  sbbf_status st = sbbf_create_lanes(nb, lanes, &f);
  if (st != SBBF_OK) return st;
  const cudaError_t e = cudaMemcpy(f->words, in + kNativeHeader, payload, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    sbbf_destroy(f);
    return record_cuda(e);
  }
  *out = f;
  return SBBF_OK;
}

sbbf_status sbbf_parquet_header(uint64_t num_bytes, uint8_t* h_out, size_t cap,
                                size_t* header_len) {
  if (num_bytes == 0 || num_bytes % 32 != 0 || num_bytes > 0x7fffffffull) return SBBF_EINVAL;
  uint8_t b[32];
  size_t k = 0;
  b[k++] = 0x15;  // field 1, i32
  uint64_t z = num_bytes << 1;  // zigzag encoding of a non-negative i32
  do {
    uint8_t c = z & 0x7f;
    z >>= 7;
    if (z) c |= 0x80;
    b[k++] = c;
  } while (z);
  for (int f = 2; f <= 4; ++f) {  // fields 2-4: a union holding member 1, an empty struct
    b[k++] = 0x1c;
    b[k++] = 0x1c;
    b[k++] = 0x00;
    b[k++] = 0x00;
  }
  b[k++] = 0x00;  // end of header
  if (header_len) *header_len = k;
  if (h_out) {
    if (cap < k) return SBBF_EINVAL;
    std::memcpy(h_out, b, k);
  }
  return SBBF_OK;
}

sbbf_status sbbf_parquet_parse_header(const uint8_t* h_buf, size_t bytes, uint64_t* num_bytes,
                                      size_t* header_len) {
  if (!h_buf) return SBBF_EINVAL;
  ThriftReader r{h_buf, bytes, 0, true};
  int id, t, last = 0;
  int64_t nbytes = -1;
  int alg = -1, hash = -1, comp = -1;
  while (r.field(id, t, last)) {
    if (id == 1 && t == 5) nbytes = r.zigzag();
    else if (id == 2 && t == 12) alg = r.union_member();
    else if (id == 3 && t == 12) hash = r.union_member();
    else if (id == 4 && t == 12) comp = r.union_member();
    else r.skip(t, 1);
  }
  if (!r.ok) return SBBF_EINVAL;
  // BLOCK split block algorithm, XXHASH, UNCOMPRESSED; whole 32-byte blocks
  if (nbytes <= 0 || nbytes % 32 != 0 || alg != 1 || hash != 1 || comp != 1) return SBBF_EINVAL;
  if (num_bytes) *num_bytes = static_cast<uint64_t>(nbytes);
  if (header_len) *header_len = r.i;
  return SBBF_OK;
}

size_t sbbf_parquet_size(const sbbf_t* f) {
  if (!f || f->lanes != 8) return 0;
  size_t h = 0;
  if (sbbf_parquet_header(filter_bytes(f), nullptr, 0, &h) != SBBF_OK) return 0;
  return h + static_cast<size_t>(filter_bytes(f));
}

sbbf_status sbbf_export_parquet(const sbbf_t* f, uint8_t* h_buf, size_t bytes, size_t* written,
                                sbbf_stream_t stream) {
  SBBF_TRACE();
  if (!f || !h_buf || f->lanes != 8) return SBBF_EINVAL;
  const uint64_t total = filter_bytes(f);
  size_t h = 0;
  sbbf_status st = sbbf_parquet_header(total, h_buf, bytes, &h);
  if (st != SBBF_OK) return st;
  if (bytes - h < total) return SBBF_EINVAL;
  const size_t chunk = total < kStagingBytes ? total : kStagingBytes;
  uint32_t* staging = nullptr;
  SBBF_CUDA(cudaMalloc(&staging, chunk));
  for (uint64_t off = 0; off < total && st == SBBF_OK; off += chunk) {
    const uint64_t len = total - off < chunk ? total - off : chunk;
    st = launch_swap(f->words + off / 4, staging, len / 4, stream);
    if (st != SBBF_OK) break;
    cudaError_t e = cudaMemcpyAsync(h_buf + h + off, staging, len, cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) st = record_cuda(e);
  }
  const cudaError_t fe = cudaFree(staging);
  if (st != SBBF_OK) return st;
  if (fe != cudaSuccess) return record_cuda(fe);
  if (written) *written = h + total;
  return SBBF_OK;
}

sbbf_status sbbf_import_parquet(const uint8_t* h_buf, size_t bytes, sbbf_t** out,
                                size_t* consumed) {
  SBBF_TRACE();
  if (!h_buf || !out) return SBBF_EINVAL;
  *out = nullptr;
  uint64_t nbytes = 0;
  size_t h = 0;
  sbbf_status st = sbbf_parquet_parse_header(h_buf, bytes, &nbytes, &h);
  if (st != SBBF_OK) return st;
  if (bytes - h < nbytes) return SBBF_EINVAL;
  sbbf_t* f = nullptr;
  st = sbbf_create_lanes(static_cast<uint32_t>(nbytes / 32), 8, &f);
  if (st != SBBF_OK) return st;
  cudaError_t e = cudaMemcpy(f->words, h_buf + h, nbytes, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    st = launch_swap(f->words, f->words, nbytes / 4, nullptr);
    if (st == SBBF_OK) {
      e = cudaStreamSynchronize(nullptr);
      if (e != cudaSuccess) st = record_cuda(e);
    }
  } else {
    st = record_cuda(e);
  }
  if (st != SBBF_OK) {
    sbbf_destroy(f);
    return st;
  }
  *out = f;
  if (consumed) *consumed = h + nbytes;
  return SBBF_OK;
}

}  // extern "C"
