// Device-side building blocks of split block Bloom filters
// (Apple, arXiv 2101.01719): block selection, the per-lane multiply-shift
// bit, and the PTX memory operations the kernels are built from.
//
// Filter layout: block b = 8 consecutive uint32 lanes at words [8b, 8b+8);
// one block is one 32-byte DRAM/L2 sector, so one key touches one sector.
#pragma once

#include <cstdint>

namespace sbbf {

constexpr int kLanes = 8;             // eight 32-bit lanes per 256-bit block
constexpr uint32_t kNoBlock = 0xFFFFFFFFu;  // never a valid block (B < 2^32)

// The eight odd multiply-shift seeds in lane order 0..7 (appendix figure:
// the low half of each 64-bit initialiser element is the lower lane).
#define SBBF_SEED0 0x44974d91u
#define SBBF_SEED1 0x47b6137bu
#define SBBF_SEED2 0xa2b7289du
#define SBBF_SEED3 0x8824ad5bu
#define SBBF_SEED4 0x2df1424bu
#define SBBF_SEED5 0x705495c7u
#define SBBF_SEED6 0x5c6bfb31u
#define SBBF_SEED7 0x9efc4947u

__device__ __forceinline__ uint32_t lane_seed(int j) {
  // Selected once per thread; a switch keeps the table out of local memory.
  switch (j & 7) {
    case 0: return SBBF_SEED0;
    case 1: return SBBF_SEED1;
    case 2: return SBBF_SEED2;
    case 3: return SBBF_SEED3;
    case 4: return SBBF_SEED4;
    case 5: return SBBF_SEED5;
    case 6: return SBBF_SEED6;
    default: return SBBF_SEED7;
  }
}

// Appendix block_index: ((h >> 32) * B) >> 32.  Both factors are 32-bit, so
// the result is the high word of a 32x32 -> 64 product.
__device__ __forceinline__ uint32_t block_of(uint64_t h, uint32_t num_blocks) {
  return __umulhi(static_cast<uint32_t>(h >> 32), num_blocks);
}

// Intro / appendix make_mask: bit index of lane with seed s for low word x,
// (s * x mod 2^32) >> 27, in [0, 32).
__device__ __forceinline__ uint32_t bit_index(uint32_t x, uint32_t s) {
  return (x * s) >> 27;
}

// All eight lanes of a block hold their mask bit (appendix find_hash).
__device__ __forceinline__ bool block_has(const uint32_t w[8], uint32_t x) {
  uint32_t t = (w[0] >> bit_index(x, SBBF_SEED0)) &
               (w[1] >> bit_index(x, SBBF_SEED1)) &
               (w[2] >> bit_index(x, SBBF_SEED2)) &
               (w[3] >> bit_index(x, SBBF_SEED3)) &
               (w[4] >> bit_index(x, SBBF_SEED4)) &
               (w[5] >> bit_index(x, SBBF_SEED5)) &
               (w[6] >> bit_index(x, SBBF_SEED6)) &
               (w[7] >> bit_index(x, SBBF_SEED7));
  return t & 1u;
}

// ---- memory operations ----------------------------------------------------

// L2 policy handles (createpolicy): streamed key data is evicted first so
// that filter sectors stay resident.
__device__ __forceinline__ uint64_t policy_evict_first() {
  uint64_t p;
  asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ uint64_t policy_evict_normal() {
  uint64_t p;
  asm("createpolicy.fractional.L2::evict_normal.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ uint64_t policy_evict_last() {
  uint64_t p;
  asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}

// Two consecutive hashes, 16-byte aligned, read once: no L1 allocation.
__device__ __forceinline__ void load_keys2(const uint64_t* p, uint64_t pol,
                                           uint64_t& a, uint64_t& b) {
  asm("ld.global.nc.L1::no_allocate.L2::cache_hint.v2.u64 {%0, %1}, [%2], %3;"
      : "=l"(a), "=l"(b)
      : "l"(p), "l"(pol));
}

__device__ __forceinline__ uint64_t load_key1(const uint64_t* p, uint64_t pol) {
  uint64_t a;
  asm("ld.global.nc.L1::no_allocate.L2::cache_hint.u64 %0, [%1], %2;"
      : "=l"(a)
      : "l"(p), "l"(pol));
  return a;
}

// One 32-byte block in a single 256-bit load (sm_100+ vector width).
__device__ __forceinline__ void load_block(const uint32_t* p, uint64_t pol,
                                           uint32_t w[8]) {
  asm("ld.global.nc.L2::cache_hint.v8.u32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8], %9;"
      : "=r"(w[0]), "=r"(w[1]), "=r"(w[2]), "=r"(w[3]), "=r"(w[4]),
        "=r"(w[5]), "=r"(w[6]), "=r"(w[7])
      : "l"(p), "l"(pol));
}

// The same load without allocating in L1: for filters much larger than L1 the
// L1 tag/fill work only costs data-pipe cycles.
__device__ __forceinline__ void load_block_na(const uint32_t* p, uint64_t pol,
                                              uint32_t w[8]) {
  asm("ld.global.nc.L1::no_allocate.L2::cache_hint.v8.u32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8], %9;"
      : "=r"(w[0]), "=r"(w[1]), "=r"(w[2]), "=r"(w[3]), "=r"(w[4]),
        "=r"(w[5]), "=r"(w[6]), "=r"(w[7])
      : "l"(p), "l"(pol));
}

__device__ __forceinline__ uint32_t load_word_na(const uint32_t* p, uint64_t pol) {
  uint32_t w;
  asm("ld.global.nc.L1::no_allocate.L2::cache_hint.u32 %0, [%1], %2;"
      : "=r"(w)
      : "l"(p), "l"(pol));
  return w;
}

// One 32-bit lane word of a block.
__device__ __forceinline__ uint32_t load_word(const uint32_t* p, uint64_t pol) {
  uint32_t w;
  asm("ld.global.nc.L2::cache_hint.u32 %0, [%1], %2;" : "=r"(w) : "l"(p), "l"(pol));
  return w;
}

// Fire-and-forget atomic OR performed at L2.
__device__ __forceinline__ void red_or(uint32_t* p, uint32_t v) {
  asm volatile("red.relaxed.gpu.global.or.b32 [%0], %1;" ::"l"(p), "r"(v)
               : "memory");
}

__device__ __forceinline__ void red_or64(unsigned long long* p, unsigned long long v) {
  asm volatile("red.relaxed.gpu.global.or.b64 [%0], %1;" ::"l"(p), "l"(v)
               : "memory");
}

// Mask bits of two adjacent lanes packed little-endian into one 64-bit word
// (the lower lane in the low half).
__device__ __forceinline__ unsigned long long mask_pair(uint32_t x, uint32_t s_lo,
                                                        uint32_t s_hi) {
  return (static_cast<unsigned long long>(1u << bit_index(x, s_hi)) << 32) |
         (1u << bit_index(x, s_lo));
}

__device__ __forceinline__ void store_stream(uint32_t* p, uint32_t v) {
  asm volatile("st.global.cs.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Two or four answer words in one streaming store (8- / 16-byte aligned p).
__device__ __forceinline__ void store_stream2(uint32_t* p, uint32_t a, uint32_t b) {
  asm volatile("st.global.cs.v2.u32 [%0], {%1, %2};" ::"l"(p), "r"(a), "r"(b) : "memory");
}
__device__ __forceinline__ void store_stream4(uint32_t* p, uint32_t a, uint32_t b, uint32_t c,
                                              uint32_t d) {
  asm volatile("st.global.cs.v4.u32 [%0], {%1, %2, %3, %4};" ::"l"(p), "r"(a), "r"(b), "r"(c),
               "r"(d)
               : "memory");
}

// Answer words word0 .. word0 + 2U - 1 of a unit of U groups (lo[u], hi[u]
// for group u), as few stores as the output's alignment allows: one 16-byte
// store per two groups, else one 8-byte store per group, else (and for words
// past the answers' end) word by word.  One store request carries four
// answer words instead of one: measured +5.5% lookups/s on an L2-resident
// filter, where the L1-to-L2 request rate is the bound.
template <int U>
__device__ __forceinline__ void store_answers(uint32_t* out, uint64_t n_out, uint64_t word0,
                                              const uint32_t (&lo)[U], const uint32_t (&hi)[U],
                                              unsigned lane, bool out16, bool out8) {
  if (U % 2 == 0 && out16 && word0 + 2 * U <= n_out) {
#pragma unroll
    for (int p = 0; p < U / 2; ++p)
      if (lane == static_cast<unsigned>(p))
        store_stream4(out + word0 + 4 * p, lo[2 * p], hi[2 * p], lo[2 * p + 1], hi[2 * p + 1]);
    return;
  }
#pragma unroll
  for (int u = 0; u < U; ++u) {
    const uint64_t w = word0 + 2 * u;
    if (out8 && w + 2 <= n_out) {
      if (lane == static_cast<unsigned>(u)) store_stream2(out + w, lo[u], hi[u]);
    } else {
      if (lane == 0 && w < n_out) store_stream(out + w, lo[u]);
      if (lane == 1 && w + 1 < n_out) store_stream(out + w + 1, hi[u]);
    }
  }
}

__device__ __forceinline__ unsigned lane_id() {
  unsigned l;
  asm("mov.u32 %0, %%laneid;" : "=r"(l));
  return l;
}

}  // namespace sbbf
