// A bare lookup loop over 256M streamed keys into a 1 MiB filter, with and
// without each part of the library's lookup: L2 cache-hint policies, the full
// eight-lane test, and the packed answers stored as two 4-byte words per 64
// keys or as one 16-byte store per 128 keys.  Prints G keys/s per variant.
//   nvcc -gencode arch=compute_103a,code=sm_103a -O3 -o /tmp/as answer_stores.cu && /tmp/as
#include <cstdio>
#include <cstdint>
#include <cuda_runtime.h>
#define CK(x) do { cudaError_t e_ = (x); if (e_ != cudaSuccess) { std::printf("%s: %s\n", #x, cudaGetErrorString(e_)); return 1; } } while (0)
__device__ __forceinline__ uint64_t pol_first() { uint64_t p; asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p)); return p; }
__device__ __forceinline__ uint64_t pol_last() { uint64_t p; asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p)); return p; }
template <bool H> __device__ __forceinline__ void ldk2(const uint64_t* p, uint64_t pol, uint64_t& a, uint64_t& b) {
  if (H) asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.v2.u64 {%0, %1}, [%2], %3;" : "=l"(a), "=l"(b) : "l"(p), "l"(pol));
  else asm volatile("ld.global.nc.L1::no_allocate.v2.u64 {%0, %1}, [%2];" : "=l"(a), "=l"(b) : "l"(p));
}
template <bool H> __device__ __forceinline__ void ldb(const uint32_t* p, uint64_t pol, uint32_t w[8]) {
  if (H) asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.v8.u32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8], %9;"
               : "=r"(w[0]), "=r"(w[1]), "=r"(w[2]), "=r"(w[3]), "=r"(w[4]), "=r"(w[5]), "=r"(w[6]), "=r"(w[7]) : "l"(p), "l"(pol));
  else asm volatile("ld.global.nc.L1::no_allocate.v8.u32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(w[0]), "=r"(w[1]), "=r"(w[2]), "=r"(w[3]), "=r"(w[4]), "=r"(w[5]), "=r"(w[6]), "=r"(w[7]) : "l"(p));
}
__device__ __forceinline__ uint32_t blk(uint64_t h, uint32_t nb) { return __umulhi(static_cast<uint32_t>(h >> 32), nb); }
template <bool F> __device__ __forceinline__ uint32_t test(const uint32_t w[8], uint64_t h) {
  const uint32_t x = static_cast<uint32_t>(h);
  if (F) return (w[0] >> ((x * 0x44974d91u) >> 27)) & (w[1] >> ((x * 0x47b6137bu) >> 27)) & (w[2] >> ((x * 0xa2b7289du) >> 27)) &
                (w[3] >> ((x * 0x8824ad5bu) >> 27)) & (w[4] >> ((x * 0x2df1424bu) >> 27)) & (w[5] >> ((x * 0x705495c7u) >> 27)) &
                (w[6] >> ((x * 0x5c6bfb31u) >> 27)) & (w[7] >> ((x * 0x9efc4947u) >> 27)) & 1u;
  return (w[0] >> ((x * 0x44974d91u) >> 27)) & (w[3] >> ((x * 0x8824ad5bu) >> 27)) & (w[7] >> ((x * 0x9efc4947u) >> 27)) & 1u;
}
// S: 0 = count only; 1 = two 4-byte streaming stores per group (lanes 0, 1); 2 = one 16-byte store per two groups
template <bool H, bool F, int S>
__global__ void __launch_bounds__(256) kA(const uint64_t* __restrict__ keys, uint64_t n, const uint32_t* __restrict__ f, uint32_t nb, uint32_t* out, uint32_t* bits) {
  const unsigned lane = threadIdx.x & 31;
  const uint64_t warp = (blockIdx.x * 256ull + threadIdx.x) >> 5, nwarps = gridDim.x * 8ull;
  const uint64_t pk = pol_first(), pf = pol_last();
  uint32_t acc = 0;
  for (uint64_t c = warp; c * 128 < n; c += nwarps) {
    uint64_t h[4];
    ldk2<H>(keys + c * 128 + 2 * lane, pk, h[0], h[1]);
    ldk2<H>(keys + c * 128 + 64 + 2 * lane, pk, h[2], h[3]);
    uint32_t w[4][8];
#pragma unroll
    for (int e = 0; e < 4; ++e) ldb<H>(f + 8ull * blk(h[e], nb), pf, w[e]);
    uint32_t r[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) r[e] = test<F>(w[e], h[e]);
    if constexpr (S == 0) {
      acc += r[0] + r[1] + r[2] + r[3];
      continue;
    } else {
    uint32_t wd[4];
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const uint32_t v = (r[2 * u] | (r[2 * u + 1] << 1)) << (2 * (lane & 15));
      wd[2 * u] = __reduce_or_sync(0xFFFFFFFFu, lane < 16 ? v : 0u);
      wd[2 * u + 1] = __reduce_or_sync(0xFFFFFFFFu, lane >= 16 ? v : 0u);
    }
    if (S == 1) {
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        if (lane == 0) __stcs(bits + 4 * c + 2 * u, wd[2 * u]);
        if (lane == 1) __stcs(bits + 4 * c + 2 * u + 1, wd[2 * u + 1]);
      }
    } else {
      if (lane == 0) __stcs(reinterpret_cast<uint4*>(bits + 4 * c), make_uint4(wd[0], wd[1], wd[2], wd[3]));
    }
    }
  }
  if (S == 0) { const uint32_t s = __reduce_add_sync(0xFFFFFFFFu, acc); if (lane == 0) atomicAdd(out, s); }
}
__global__ void fill(uint64_t* k, uint64_t n) {
  for (uint64_t i = blockIdx.x * 256ull + threadIdx.x; i < n; i += gridDim.x * 256ull) {
    uint64_t z = (i + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull; z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    k[i] = z ^ (z >> 31);
  }
}
template <bool H, bool F, int S> int run(const char* name, const uint64_t* keys, uint64_t n, const uint32_t* f, uint32_t nb, uint32_t* out, uint32_t* bits, int grid) {
  cudaEvent_t a, b; CK(cudaEventCreate(&a)); CK(cudaEventCreate(&b));
  float best = 0;
  for (int rep = 0; rep < 3; ++rep) {
    CK(cudaEventRecord(a)); kA<H, F, S><<<grid, 256>>>(keys, n, f, nb, out, bits); CK(cudaEventRecord(b)); CK(cudaEventSynchronize(b));
    float ms; CK(cudaEventElapsedTime(&ms, a, b)); const float r = n / ms / 1e6; if (r > best) best = r;
  }
  std::printf("%-44s %7.1f G keys/s\n", name, best);
  return 0;
}
int main() {
  int sms = 0; CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0));
  const uint64_t n = 1ull << 28; const uint32_t nb = 32768;
  uint64_t* keys; uint32_t *f, *out, *bits;
  CK(cudaMalloc(&keys, n * 8)); CK(cudaMalloc(&f, nb * 32)); CK(cudaMalloc(&out, 8)); CK(cudaMalloc(&bits, n / 8));
  CK(cudaMemset(f, 0x5a, nb * 32)); fill<<<sms * 8, 256>>>(keys, n); CK(cudaDeviceSynchronize());
  const int grid = sms * 6;
  run<false, false, 0>("plain loads, 3-lane test, count", keys, n, f, nb, out, bits, grid);
  run<true, false, 0>("cache hints, 3-lane test, count", keys, n, f, nb, out, bits, grid);
  run<false, true, 0>("plain loads, 8-lane test, count", keys, n, f, nb, out, bits, grid);
  run<false, true, 1>("plain loads, 8-lane test, 2x4-byte stores", keys, n, f, nb, out, bits, grid);
  run<false, true, 2>("plain loads, 8-lane test, 16-byte store", keys, n, f, nb, out, bits, grid);
  run<true, true, 1>("cache hints, 8-lane test, 2x4-byte stores", keys, n, f, nb, out, bits, grid);
  run<true, true, 2>("cache hints, 8-lane test, 16-byte store", keys, n, f, nb, out, bits, grid);
  return 0;
}
