// Where a key's 64-bit hash comes from.
//
// The paper's operations take a 64-bit hash per key, and it leaves the key
// hash open: the key is hashed once, to 64 bits, before block selection.
// Besides taking the caller's hashes, the kernels can hash raw keys in the
// same pass with XXH64 (the hash Parquet's split block filters use, seed 0
// there).  XXH64 here follows its published specification (Y. Collet, xxHash,
// XXH64): inputs of 32 bytes or more run four accumulators over 32-byte
// stripes; then the length is added, 8-, 4- and 1-byte tail steps follow, and
// a final avalanche mixes the result.  Bytes are read little-endian.
//
// A key source provides pair(k, n, pol, h0, h1): the hashes of keys k and
// k + 1 (k even; a key at or past n yields 0, which the kernels never use).
#pragma once

#include <cstdint>

#include "sbbf_device.cuh"

namespace sbbf {

namespace xxh {
constexpr uint64_t kP1 = 0x9E3779B185EBCA87ull;
constexpr uint64_t kP2 = 0xC2B2AE3D27D4EB4Full;
constexpr uint64_t kP3 = 0x165667B19E3779F9ull;
constexpr uint64_t kP4 = 0x85EBCA77C2B2AE63ull;
constexpr uint64_t kP5 = 0x27D4EB2F165667C5ull;

__host__ __device__ __forceinline__ uint64_t rotl(uint64_t x, int r) { return (x << r) | (x >> (64 - r)); }

__host__ __device__ __forceinline__ uint64_t round(uint64_t acc, uint64_t lane) {
  return rotl(acc + lane * kP2, 31) * kP1;
}

__host__ __device__ __forceinline__ uint64_t avalanche(uint64_t h) {
  h ^= h >> 33;
  h *= kP2;
  h ^= h >> 29;
  h *= kP3;
  return h ^ (h >> 32);
}

// Tail step for one 8-byte word.
__host__ __device__ __forceinline__ uint64_t step8(uint64_t acc, uint64_t v) {
  return rotl(acc ^ round(0, v), 27) * kP1 + kP4;
}

// Tail step for one 4-byte word.
__host__ __device__ __forceinline__ uint64_t step4(uint64_t acc, uint32_t v) {
  return rotl(acc ^ (static_cast<uint64_t>(v) * kP1), 23) * kP2 + kP3;
}

__host__ __device__ __forceinline__ uint64_t step1(uint64_t acc, uint32_t byte) {
  return rotl(acc ^ (static_cast<uint64_t>(byte) * kP5), 11) * kP1;
}

// XXH64 of one 8-byte key (its little-endian bytes).
__device__ __forceinline__ uint64_t hash8(uint64_t key, uint64_t seed) {
  return avalanche(step8(seed + kP5 + 8, key));
}

// XXH64 of one 4-byte key.
__device__ __forceinline__ uint64_t hash4(uint32_t key, uint64_t seed) {
  return avalanche(step4(seed + kP5 + 4, key));
}

// Reads 8 (or 4) bytes at any byte address from the aligned words that hold
// them: every word read holds at least one of the requested bytes, so no read
// leaves the words the key occupies.
__device__ __forceinline__ uint64_t read8(const uint8_t* p) {
  const uintptr_t a = reinterpret_cast<uintptr_t>(p);
  const unsigned o = a & 7;
  const uint64_t* q = reinterpret_cast<const uint64_t*>(a - o);
  const uint64_t lo = __ldg(q);
  if (o == 0) return lo;
  return (lo >> (8 * o)) | (__ldg(q + 1) << (64 - 8 * o));
}

__device__ __forceinline__ uint32_t read4(const uint8_t* p) {
  const uintptr_t a = reinterpret_cast<uintptr_t>(p);
  const unsigned o = a & 3;
  const uint32_t* q = reinterpret_cast<const uint32_t*>(a - o);
  const uint32_t lo = __ldg(q);
  if (o == 0) return lo;
  return (lo >> (8 * o)) | (__ldg(q + 1) << (32 - 8 * o));
}

// XXH64 of len bytes at p (global memory).
static __device__ __noinline__ uint64_t hash_bytes(const uint8_t* p, uint64_t len, uint64_t seed) {
  uint64_t i = 0, acc;
  if (len >= 32) {
    uint64_t v1 = seed + kP1 + kP2, v2 = seed + kP2, v3 = seed, v4 = seed - kP1;
    for (; i + 32 <= len; i += 32) {
      v1 = round(v1, read8(p + i));
      v2 = round(v2, read8(p + i + 8));
      v3 = round(v3, read8(p + i + 16));
      v4 = round(v4, read8(p + i + 24));
    }
    acc = rotl(v1, 1) + rotl(v2, 7) + rotl(v3, 12) + rotl(v4, 18);
    acc = (acc ^ round(0, v1)) * kP1 + kP4;
    acc = (acc ^ round(0, v2)) * kP1 + kP4;
    acc = (acc ^ round(0, v3)) * kP1 + kP4;
    acc = (acc ^ round(0, v4)) * kP1 + kP4;
  } else {
    acc = seed + kP5;
  }
  acc += len;
  for (; i + 8 <= len; i += 8) acc = step8(acc, read8(p + i));
  if (i + 4 <= len) {
    acc = step4(acc, read4(p + i));
    i += 4;
  }
  for (; i < len; ++i) acc = step1(acc, __ldg(p + i));
  return avalanche(acc);
}
// XXH64 of len bytes in host memory (checksums of serialized filters).
inline uint64_t hash_bytes_host(const uint8_t* p, uint64_t len, uint64_t seed) {
  auto rd8 = [](const uint8_t* q) {
    uint64_t v = 0;
    for (int i = 7; i >= 0; --i) v = (v << 8) | q[i];
    return v;
  };
  uint64_t i = 0, acc;
  if (len >= 32) {
    uint64_t v1 = seed + kP1 + kP2, v2 = seed + kP2, v3 = seed, v4 = seed - kP1;
    for (; i + 32 <= len; i += 32) {
      v1 = round(v1, rd8(p + i));
      v2 = round(v2, rd8(p + i + 8));
      v3 = round(v3, rd8(p + i + 16));
      v4 = round(v4, rd8(p + i + 24));
    }
    acc = rotl(v1, 1) + rotl(v2, 7) + rotl(v3, 12) + rotl(v4, 18);
    acc = (acc ^ round(0, v1)) * kP1 + kP4;
    acc = (acc ^ round(0, v2)) * kP1 + kP4;
    acc = (acc ^ round(0, v3)) * kP1 + kP4;
    acc = (acc ^ round(0, v4)) * kP1 + kP4;
  } else {
    acc = seed + kP5;
  }
  acc += len;
  for (; i + 8 <= len; i += 8) acc = step8(acc, rd8(p + i));
  if (i + 4 <= len) {
    acc = step4(acc, static_cast<uint32_t>(p[i]) | (static_cast<uint32_t>(p[i + 1]) << 8) |
                         (static_cast<uint32_t>(p[i + 2]) << 16) |
                         (static_cast<uint32_t>(p[i + 3]) << 24));
    i += 4;
  }
  for (; i < len; ++i) acc = step1(acc, p[i]);
  return avalanche(acc);
}
}  // namespace xxh

// The caller's 64-bit hashes (the paper's input).
struct HashInput {
  static constexpr bool kHeavy = false;  // see BytesInput
  const uint64_t* hashes;
  __host__ __device__ HashInput(const uint64_t* p = nullptr) : hashes(p) {}
  __device__ __forceinline__ void pair(uint64_t k, uint64_t n, uint64_t pol, uint64_t& h0,
                                       uint64_t& h1) const {
    const bool vec = (reinterpret_cast<uintptr_t>(hashes) & 15) == 0;
    if (vec && k + 1 < n) {
      load_keys2(hashes + k, pol, h0, h1);
    } else {
      h0 = k < n ? load_key1(hashes + k, pol) : 0;
      h1 = k + 1 < n ? load_key1(hashes + k + 1, pol) : 0;
    }
  }
};

// 8-byte keys (8-byte aligned), hashed with XXH64.
struct Key64Input {
  static constexpr bool kHeavy = false;
  const uint64_t* keys;
  uint64_t seed;
  __device__ __forceinline__ void pair(uint64_t k, uint64_t n, uint64_t pol, uint64_t& h0,
                                       uint64_t& h1) const {
    HashInput(keys).pair(k, n, pol, h0, h1);
    h0 = xxh::hash8(h0, seed);
    h1 = xxh::hash8(h1, seed);
  }
};

// 4-byte keys (4-byte aligned), hashed with XXH64.  Keys k and k + 1 (k even)
// share one 8-byte word when the array is 8-byte aligned.
struct Key32Input {
  static constexpr bool kHeavy = false;
  const uint32_t* keys;
  uint64_t seed;
  __device__ __forceinline__ void pair(uint64_t k, uint64_t n, uint64_t pol, uint64_t& h0,
                                       uint64_t& h1) const {
    uint32_t a = 0, b = 0;
    if ((reinterpret_cast<uintptr_t>(keys) & 7) == 0 && k + 1 < n) {
      const uint64_t w = load_key1(reinterpret_cast<const uint64_t*>(keys + k), pol);
      a = static_cast<uint32_t>(w);
      b = static_cast<uint32_t>(w >> 32);
    } else {
      if (k < n) a = __ldg(keys + k);
      if (k + 1 < n) b = __ldg(keys + k + 1);
    }
    h0 = xxh::hash4(a, seed);
    h1 = xxh::hash4(b, seed);
  }
};

// Variable-length keys: key k is data[offsets[k], offsets[k + 1]).
struct BytesInput {
  // A per-key loop with a call: kernels reading this source are not held to
  // a register cap below 128 per thread.
  static constexpr bool kHeavy = true;
  const uint8_t* data;
  const uint64_t* offsets;  // n + 1 non-decreasing byte offsets
  uint64_t seed;
  __device__ __forceinline__ void pair(uint64_t k, uint64_t n, uint64_t, uint64_t& h0,
                                       uint64_t& h1) const {
    h0 = h1 = 0;
    if (k >= n) return;
    const uint64_t o0 = __ldg(offsets + k), o1 = __ldg(offsets + k + 1);
    h0 = xxh::hash_bytes(data + o0, o1 - o0, seed);
    if (k + 1 < n) {
      const uint64_t o2 = __ldg(offsets + k + 2);
      h1 = xxh::hash_bytes(data + o1, o2 - o1, seed);
    }
  }
};

}  // namespace sbbf
