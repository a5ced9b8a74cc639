// Random 32-byte block access ceilings on the current GPU.
//
// Every filter operation touches one random 32-byte block, so the fastest a
// lookup or insert kernel can go is bounded by how many random blocks the
// memory system serves per second.  This program measures that, with no
// hashing beyond index generation:
//   read32  one 256-bit load per random block (the lookup access)
//   read64  two adjacent blocks (64 bytes) per random position
//   red8    eight lanes each red.or one word of a random block (the insert access)
//   smem    random 32-byte reads from a CTA's shared memory
//   dsmem   random 32-byte reads from other CTAs' shared memory in a cluster
// over buffers from L2-resident (1 MiB) to 32 GiB.
//
// Build and run:  nvcc -gencode arch=compute_103a,code=sm_103a -O3 -o rs random_sector.cu && ./rs
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>

namespace cg = cooperative_groups;

#define CK(x)                                                                        \
  do {                                                                               \
    cudaError_t e_ = (x);                                                            \
    if (e_ != cudaSuccess) {                                                         \
      std::printf("error %s at line %d: %s\n", #x, __LINE__, cudaGetErrorString(e_)); \
      return 1;                                                                      \
    }                                                                                \
  } while (0)

__device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Random block index in [0, nblk) for (thread, draw).
__device__ __forceinline__ uint32_t draw(uint64_t t, uint64_t i, uint32_t nblk) {
  const uint64_t h = mix64(t * 0x9E3779B97F4A7C15ull + i * 0x632BE59BD9B4E019ull);
  return __umulhi(static_cast<uint32_t>(h >> 32), nblk);
}

__device__ __forceinline__ void load32(const uint32_t* p, uint32_t w[8]) {
  asm volatile("ld.global.nc.v8.u32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(w[0]), "=r"(w[1]), "=r"(w[2]), "=r"(w[3]), "=r"(w[4]), "=r"(w[5]),
                 "=r"(w[6]), "=r"(w[7])
               : "l"(p));
}

// Cache-path variants of the same 256-bit load: 0 = ld.global.nc (L1
// allocating), 1 = ld.global.nc.L1::no_allocate, 2 = ld.global.cg (L2 only).
template <int kPath>
__device__ __forceinline__ void load32v(const uint32_t* p, uint32_t w[8]) {
  if (kPath == 1) {
    asm volatile("ld.global.nc.L1::no_allocate.v8.u32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(w[0]), "=r"(w[1]), "=r"(w[2]), "=r"(w[3]), "=r"(w[4]), "=r"(w[5]),
                   "=r"(w[6]), "=r"(w[7])
                 : "l"(p));
  } else if (kPath == 2) {
    asm volatile("ld.global.cg.v8.u32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(w[0]), "=r"(w[1]), "=r"(w[2]), "=r"(w[3]), "=r"(w[4]), "=r"(w[5]),
                   "=r"(w[6]), "=r"(w[7])
                 : "l"(p));
  } else {
    load32(p, w);
  }
}

template <int U, int kPath>
__global__ void read32p(const uint32_t* __restrict__ f, uint32_t nblk, int iters, uint32_t* out) {
  const uint64_t t = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x;
  uint32_t acc = 0;
  for (int i = 0; i < iters; ++i) {
    uint32_t w[U][8];
#pragma unroll
    for (int u = 0; u < U; ++u) load32v<kPath>(f + 8ull * draw(t, i * U + u, nblk), w[u]);
#pragma unroll
    for (int u = 0; u < U; ++u) acc ^= w[u][0] ^ w[u][7];
  }
  if (acc == 0x12345678u) out[0] = acc;
}

template <int U>
__global__ void read32(const uint32_t* __restrict__ f, uint32_t nblk, int iters, uint32_t* out) {
  const uint64_t t = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x;
  uint32_t acc = 0;
  for (int i = 0; i < iters; ++i) {
    uint32_t w[U][8];
#pragma unroll
    for (int u = 0; u < U; ++u) load32(f + 8ull * draw(t, i * U + u, nblk), w[u]);
#pragma unroll
    for (int u = 0; u < U; ++u) acc ^= w[u][0] ^ w[u][7];
  }
  if (acc == 0x12345678u) out[0] = acc;  // keeps the loads live
}

__global__ void read64(const uint32_t* __restrict__ f, uint32_t npairs, int iters, uint32_t* out) {
  const uint64_t t = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x;
  uint32_t acc = 0;
  for (int i = 0; i < iters; ++i) {
    uint32_t w0[8], w1[8];
    const uint64_t b = draw(t, i, npairs);
    load32(f + 16ull * b, w0);
    load32(f + 16ull * b + 8, w1);
    acc ^= w0[0] ^ w1[7];
  }
  if (acc == 0x12345678u) out[0] = acc;
}

__global__ void red8(uint32_t* __restrict__ f, uint32_t nblk, int iters) {
  const uint64_t t = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x;
  const uint32_t j = threadIdx.x & 7;
  for (int i = 0; i < iters; ++i) {
    const uint32_t b = draw(t >> 3, i, nblk);
    const uint32_t m = 1u << ((j * 4u + static_cast<uint32_t>(i)) & 31u);
    asm volatile("red.relaxed.gpu.global.or.b32 [%0], %1;" ::"l"(f + 8ull * b + j), "r"(m)
                 : "memory");
  }
}

extern __shared__ uint4 smem4[];

__global__ void smem_read(const uint32_t* __restrict__ f, uint32_t nblk, int iters,
                          uint32_t* out) {
  for (uint32_t i = threadIdx.x; i < 2 * nblk; i += blockDim.x)
    smem4[i] = reinterpret_cast<const uint4*>(f)[i];
  __syncthreads();
  const uint64_t t = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x;
  uint32_t acc = 0;
  for (int i = 0; i < iters; ++i) {
    const uint32_t b = draw(t, i, nblk);
    const uint4 a = smem4[2 * b], c = smem4[2 * b + 1];
    acc ^= a.x ^ a.w ^ c.x ^ c.w;
  }
  if (acc == 0x12345678u) out[0] = acc;
}

__global__ void dsmem_read(const uint32_t* __restrict__ f, uint32_t nblk, int iters,
                           uint32_t* out) {
  cg::cluster_group cluster = cg::this_cluster();
  const uint32_t csize = cluster.num_blocks();
  for (uint32_t i = threadIdx.x; i < 2 * nblk; i += blockDim.x)
    smem4[i] = reinterpret_cast<const uint4*>(f)[i];
  cluster.sync();
  const uint64_t t = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x;
  uint32_t acc = 0;
  for (int i = 0; i < iters; ++i) {
    const uint32_t b = draw(t, i, nblk);
    const uint32_t rank = draw(t, i + 1000003, csize);
    const uint4* p = cluster.map_shared_rank(smem4, rank);
    const uint4 a = p[2 * b], c = p[2 * b + 1];
    acc ^= a.x ^ a.w ^ c.x ^ c.w;
  }
  cluster.sync();  // no CTA leaves while others still read its shared memory
  if (acc == 0x12345678u) out[0] = acc;
}

int main() {
  int sms = 0;
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0));
  const uint64_t max_bytes = 32ull << 30;
  uint32_t *f = nullptr, *out = nullptr;
  CK(cudaMalloc(&f, max_bytes));
  CK(cudaMalloc(&out, 64));
  CK(cudaMemset(f, 0x5a, max_bytes));
  CK(cudaDeviceSynchronize());
  cudaEvent_t a, b;
  CK(cudaEventCreate(&a));
  CK(cudaEventCreate(&b));
  float ms = 0;
  std::printf("SMs %d\n", sms);
  const uint64_t sizes[] = {1ull << 20, 64ull << 20, 128ull << 20, 512ull << 20, 4ull << 30,
                            (32ull << 30) - 32};
  for (uint64_t bytes : sizes) {
    const uint32_t nblk = static_cast<uint32_t>(bytes / 32);
    const int threads = 256, grid = sms * 8;
    read32<4><<<grid, threads>>>(f, nblk, 4, out);
    CK(cudaDeviceSynchronize());
    CK(cudaEventRecord(a));
    read32<4><<<grid, threads>>>(f, nblk, 64, out);
    CK(cudaEventRecord(b));
    CK(cudaEventSynchronize(b));
    CK(cudaEventElapsedTime(&ms, a, b));
    double n = static_cast<double>(grid) * threads * 64 * 4;
    std::printf("read32 %10.1f MiB: %7.1f G blocks/s (%7.1f GB/s of 32-byte blocks)\n",
                bytes / 1048576.0, n / ms / 1e6, 32 * n / ms / 1e6);
    CK(cudaEventRecord(a));
    read64<<<grid, threads>>>(f, nblk / 2, 128, out);
    CK(cudaEventRecord(b));
    CK(cudaEventSynchronize(b));
    CK(cudaEventElapsedTime(&ms, a, b));
    n = static_cast<double>(grid) * threads * 128;
    std::printf("read64 %10.1f MiB: %7.1f G pairs/s  (%7.1f GB/s of 64-byte pairs)\n",
                bytes / 1048576.0, n / ms / 1e6, 64 * n / ms / 1e6);
    CK(cudaEventRecord(a));
    red8<<<grid, threads>>>(f, nblk, 128);
    CK(cudaEventRecord(b));
    CK(cudaEventSynchronize(b));
    CK(cudaEventElapsedTime(&ms, a, b));
    n = static_cast<double>(grid) * threads / 8 * 128;
    std::printf("red8   %10.1f MiB: %7.1f G blocks/s (8 x red.or.b32 per block)\n",
                bytes / 1048576.0, n / ms / 1e6);
  }
  // cache-path variants on an L2-resident 1 MiB buffer
  {
    const uint32_t nblk = 32768;
    const int threads = 256, grid = sms * 8;
    const char* names[3] = {"nc (L1 alloc)", "nc L1::no_allocate", "cg (L2 only)"};
    for (int path = 0; path < 3; ++path) {
      for (int rep = 0; rep < 2; ++rep) {
        CK(cudaEventRecord(a));
        if (path == 0) read32p<4, 0><<<grid, threads>>>(f, nblk, 64, out);
        if (path == 1) read32p<4, 1><<<grid, threads>>>(f, nblk, 64, out);
        if (path == 2) read32p<4, 2><<<grid, threads>>>(f, nblk, 64, out);
        CK(cudaEventRecord(b));
        CK(cudaEventSynchronize(b));
      }
      CK(cudaEventElapsedTime(&ms, a, b));
      const double n = static_cast<double>(grid) * threads * 64 * 4;
      std::printf("read32 1 MiB, %-20s: %7.1f G blocks/s\n", names[path], n / ms / 1e6);
    }
  }
  // shared memory (128 KiB per CTA) and distributed shared memory clusters
  const uint32_t snblk = 4096;
  const int sbytes = static_cast<int>(snblk * 32);
  CK(cudaFuncSetAttribute(smem_read, cudaFuncAttributeMaxDynamicSharedMemorySize, sbytes));
  CK(cudaEventRecord(a));
  smem_read<<<sms, 1024, sbytes>>>(f, snblk, 4096, out);
  CK(cudaEventRecord(b));
  CK(cudaEventSynchronize(b));
  CK(cudaEventElapsedTime(&ms, a, b));
  double n = static_cast<double>(sms) * 1024 * 4096;
  std::printf("smem   128 KiB per CTA: %7.1f G blocks/s\n", n / ms / 1e6);
  CK(cudaFuncSetAttribute(dsmem_read, cudaFuncAttributeMaxDynamicSharedMemorySize, sbytes));
  CK(cudaFuncSetAttribute(dsmem_read, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
  for (int csize : {2, 4, 8, 16}) {
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = csize;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cfg.blockDim = dim3(1024);
    cfg.dynamicSmemBytes = sbytes;
    cfg.gridDim = dim3(csize);
    int nclusters = 0;
    if (cudaOccupancyMaxActiveClusters(&nclusters, dsmem_read, &cfg) != cudaSuccess ||
        nclusters < 1) {
      cudaGetLastError();
      std::printf("dsmem  cluster %2d: not launchable\n", csize);
      continue;
    }
    cfg.gridDim = dim3(nclusters * csize);
    CK(cudaEventRecord(a));
    CK(cudaLaunchKernelEx(&cfg, dsmem_read, static_cast<const uint32_t*>(f), snblk, 1024, out));
    CK(cudaEventRecord(b));
    CK(cudaEventSynchronize(b));
    CK(cudaEventElapsedTime(&ms, a, b));
    n = static_cast<double>(nclusters) * csize * 1024 * 1024;
    std::printf("dsmem  cluster %2d x 128 KiB (%d SMs): %7.1f G blocks/s\n", csize,
                nclusters * csize, n / ms / 1e6);
  }
  CK(cudaEventRecord(a));
  CK(cudaMemcpy(f + (4ull << 30) / 4, f, 4ull << 30, cudaMemcpyDeviceToDevice));
  CK(cudaEventRecord(b));
  CK(cudaEventSynchronize(b));
  CK(cudaEventElapsedTime(&ms, a, b));
  std::printf("copy   4 GiB: %.1f GB/s (read + write)\n", 2.0 * (4ull << 30) / ms / 1e6);
  CK(cudaFree(f));
  CK(cudaFree(out));
  return 0;
}
