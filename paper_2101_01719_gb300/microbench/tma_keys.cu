// Lookup-shaped loop: 256M streamed 8-byte keys, each selecting a random
// 32-byte block of a 1 MiB buffer.  A: keys by 128-bit L1-no-allocate loads.
// B: keys by per-warp cp.async.bulk copies into a 4-deep shared-memory ring
// (every mbarrier wait bounded by the global timer).  Prints G keys/s for
// 4, 6 and 8 CTAs per SM.
//   nvcc -gencode arch=compute_103a,code=sm_103a -O3 -o /tmp/tk tma_keys.cu && /tmp/tk
#include <cstdio>
#include <cstdint>
#include <cuda_runtime.h>
#define CK(x) do { cudaError_t e_ = (x); if (e_ != cudaSuccess) { std::printf("%s: %s\n", #x, cudaGetErrorString(e_)); return 1; } } while (0)

__device__ __forceinline__ void ldk2(const uint64_t* p, uint64_t& a, uint64_t& b) {
  asm volatile("ld.global.nc.L1::no_allocate.v2.u64 {%0, %1}, [%2];" : "=l"(a), "=l"(b) : "l"(p));
}
__device__ __forceinline__ void ldb(const uint32_t* p, uint32_t w[8]) {
  asm volatile("ld.global.nc.L1::no_allocate.v8.u32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(w[0]), "=r"(w[1]), "=r"(w[2]), "=r"(w[3]), "=r"(w[4]), "=r"(w[5]), "=r"(w[6]), "=r"(w[7]) : "l"(p));
}
__device__ __forceinline__ uint32_t blk(uint64_t h, uint32_t nb) { return __umulhi(static_cast<uint32_t>(h >> 32), nb); }
__device__ __forceinline__ uint32_t test(const uint32_t w[8], uint64_t h) {
  const uint32_t x = static_cast<uint32_t>(h);
  return (w[0] >> ((x * 0x44974d91u) >> 27)) & (w[3] >> ((x * 0x8824ad5bu) >> 27)) & (w[7] >> ((x * 0x9efc4947u) >> 27)) & 1u;
}

// A: grid-stride over 128-key chunks per warp
__global__ void __launch_bounds__(256) kA(const uint64_t* __restrict__ keys, uint64_t n, const uint32_t* __restrict__ f, uint32_t nb, uint32_t* out) {
  const unsigned lane = threadIdx.x & 31;
  const uint64_t warp = (blockIdx.x * 256ull + threadIdx.x) >> 5, nwarps = gridDim.x * 8ull;
  uint32_t acc = 0;
  for (uint64_t c = warp; c * 128 < n; c += nwarps) {
    uint64_t h[4];
    ldk2(keys + c * 128 + 2 * lane, h[0], h[1]);
    ldk2(keys + c * 128 + 64 + 2 * lane, h[2], h[3]);
    uint32_t w[4][8];
#pragma unroll
    for (int e = 0; e < 4; ++e) ldb(f + 8ull * blk(h[e], nb), w[e]);
#pragma unroll
    for (int e = 0; e < 4; ++e) acc += test(w[e], h[e]);
  }
  const uint32_t s = __reduce_add_sync(0xFFFFFFFFu, acc);
  if (lane == 0) atomicAdd(out, s);
}

__device__ __forceinline__ uint32_t su32(const void* p) { return static_cast<uint32_t>(__cvta_generic_to_shared(p)); }
__device__ __forceinline__ uint64_t gns() { uint64_t t; asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t)); return t; }

constexpr int kStages = 4;
// B: warp w owns chunks w, w + nwarps, ...; lane 0 keeps kStages - 1 copies ahead
__global__ void __launch_bounds__(256) kB(const uint64_t* __restrict__ keys, uint64_t n, const uint32_t* __restrict__ f, uint32_t nb, uint32_t* out, uint32_t* err) {
  __shared__ __align__(16) uint64_t s_keys[8][kStages][128];
  __shared__ __align__(8) unsigned long long s_bar[8][kStages];
  const unsigned lane = threadIdx.x & 31, wic = threadIdx.x >> 5;
  const uint64_t warp = (blockIdx.x * 256ull + threadIdx.x) >> 5, nwarps = gridDim.x * 8ull;
  const uint64_t n_chunks = n / 128;  // n a multiple of 128 here
  if (lane == 0) {
    for (int s = 0; s < kStages; ++s) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&s_bar[wic][s])) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncwarp();
  auto issue = [&](uint64_t c, int s) {
    const uint32_t bar = su32(&s_bar[wic][s]);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(1024u) : "memory");
    asm volatile("cp.async.bulk.shared::cta.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(su32(&s_keys[wic][s][0])), "l"(keys + c * 128), "r"(1024u), "r"(bar) : "memory");
  };
  uint32_t acc = 0;
  if (lane == 0)
    for (int s = 0; s < kStages - 1; ++s) { const uint64_t c = warp + s * nwarps; if (c < n_chunks) issue(c, s); }
  uint32_t parity = 0;
  int s = 0;
  for (uint64_t c = warp; c < n_chunks; c += nwarps) {
    // issue the copy kStages - 1 chunks ahead into the slot freed last step
    const uint64_t ca = c + (kStages - 1) * nwarps;
    const int sa = (s + kStages - 1) % kStages;
    __syncwarp();
    if (lane == 0 && ca < n_chunks) issue(ca, sa);
    const uint32_t bar = su32(&s_bar[wic][s]);
    const uint64_t t0 = gns();
    for (;;) {
      uint32_t done;
      asm volatile("{ .reg .pred p; mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }" : "=r"(done) : "r"(bar), "r"((parity >> s) & 1) : "memory");
      if (done) break;
      if (gns() - t0 > 2000000000ull) { if (lane == 0) atomicAdd(err, 1u); return; }
    }
    parity ^= 1u << s;
    uint64_t h[4];
    const uint4 v0 = *reinterpret_cast<const uint4*>(&s_keys[wic][s][2 * lane]);
    const uint4 v1 = *reinterpret_cast<const uint4*>(&s_keys[wic][s][64 + 2 * lane]);
    h[0] = (uint64_t(v0.y) << 32) | v0.x; h[1] = (uint64_t(v0.w) << 32) | v0.z;
    h[2] = (uint64_t(v1.y) << 32) | v1.x; h[3] = (uint64_t(v1.w) << 32) | v1.z;
    uint32_t w[4][8];
#pragma unroll
    for (int e = 0; e < 4; ++e) ldb(f + 8ull * blk(h[e], nb), w[e]);
#pragma unroll
    for (int e = 0; e < 4; ++e) acc += test(w[e], h[e]);
    s = (s + 1) % kStages;
  }
  const uint32_t sum = __reduce_add_sync(0xFFFFFFFFu, acc);
  if (lane == 0) atomicAdd(out, sum);
}

__global__ void fill(uint64_t* k, uint64_t n) {
  for (uint64_t i = blockIdx.x * 256ull + threadIdx.x; i < n; i += gridDim.x * 256ull) {
    uint64_t z = (i + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull; z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    k[i] = z ^ (z >> 31);
  }
}

int main() {
  int sms = 0; CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0));
  const uint64_t n = 1ull << 28;
  const uint32_t nb = 32768;
  uint64_t* keys; uint32_t *f, *out, *err;
  CK(cudaMalloc(&keys, n * 8)); CK(cudaMalloc(&f, nb * 32)); CK(cudaMalloc(&out, 8)); CK(cudaMalloc(&err, 8));
  CK(cudaMemset(f, 0x5a, nb * 32)); CK(cudaMemset(err, 0, 8));
  fill<<<sms * 8, 256>>>(keys, n); CK(cudaDeviceSynchronize());
  cudaEvent_t a, b; CK(cudaEventCreate(&a)); CK(cudaEventCreate(&b));
  float ms;
  for (int occ : {4, 6, 8}) {
    for (int rep = 0; rep < 3; ++rep) {
      CK(cudaMemset(out, 0, 8));
      CK(cudaEventRecord(a)); kA<<<sms * occ, 256>>>(keys, n, f, nb, out); CK(cudaEventRecord(b)); CK(cudaEventSynchronize(b));
      CK(cudaEventElapsedTime(&ms, a, b));
      uint32_t ha = 0; CK(cudaMemcpy(&ha, out, 4, cudaMemcpyDeviceToHost));
      if (rep == 2) std::printf("A occ %d: %7.1f G keys/s (hits %u)\n", occ, n / ms / 1e6, ha);
      CK(cudaMemset(out, 0, 8));
      CK(cudaEventRecord(a)); kB<<<sms * occ, 256>>>(keys, n, f, nb, out, err); CK(cudaEventRecord(b)); CK(cudaEventSynchronize(b));
      CK(cudaEventElapsedTime(&ms, a, b));
      uint32_t hb = 0, he = 0; CK(cudaMemcpy(&hb, out, 4, cudaMemcpyDeviceToHost)); CK(cudaMemcpy(&he, err, 4, cudaMemcpyDeviceToHost));
      if (rep == 2) std::printf("B occ %d: %7.1f G keys/s (hits %u, timeouts %u)\n", occ, n / ms / 1e6, hb, he);
    }
  }
  return 0;
}
