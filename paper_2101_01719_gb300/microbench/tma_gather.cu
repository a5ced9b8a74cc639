// Random 32-byte blocks through the TMA gather path.
//
// The filter is viewed as a 2-D tensor of num_blocks rows x 8 uint32 columns
// (one row = one 32-byte block).  cp.async.bulk.tensor...tile::gather4 copies
// four arbitrary rows into shared memory per instruction, tracked by an
// mbarrier, without the per-request L1 data-pipe cost of plain loads.  Each
// warp keeps kStages buffers of 32 blocks in flight; lanes then read their
// block from shared memory.  Every mbarrier wait is bounded; on timeout the
// kernel records an error and stops.
//
// Build and run:
//   nvcc -gencode arch=compute_103a,code=sm_103a -O3 -o tg tma_gather.cu && ./tg
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>

#define CK(x)                                                                        \
  do {                                                                               \
    cudaError_t e_ = (x);                                                            \
    if (e_ != cudaSuccess) {                                                         \
      std::printf("error %s at line %d: %s\n", #x, __LINE__, cudaGetErrorString(e_)); \
      return 1;                                                                      \
    }                                                                                \
  } while (0)

constexpr int kStages = 4;
constexpr int kWarps = 8;
constexpr uint64_t kWaitNs = 200ull * 1000 * 1000;  // give up a wait after 200 ms

__device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t now_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Non-blocking test_wait polled against the global timer: always returns.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  const uint64_t t0 = now_ns();
  for (;;) {
    uint32_t done;
    asm volatile(
        "{ .reg .pred p; mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
    if (now_ns() - t0 > kWaitNs) return false;
  }
}

__global__ void __launch_bounds__(kWarps * 32)
    gather_kernel(const __grid_constant__ CUtensorMap tmap, uint32_t nblk, int iters,
                  uint32_t* out, unsigned* err) {
  __shared__ __align__(128) uint32_t buf[kWarps][kStages][32 * 8];
  __shared__ __align__(8) uint64_t bars[kWarps][kStages];
  const unsigned lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) {
    for (int s = 0; s < kStages; ++s)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&bars[w][s])) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncwarp();
  const uint64_t t = (blockIdx.x * static_cast<uint64_t>(kWarps) + w) * 32;
  // issue round r into stage s: 32 random rows, 8 gather4 copies by lanes 0..7
  auto issue = [&](int s, int r) {
    const uint32_t bar = smem_addr(&bars[w][s]);
    if (lane == 0)
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar),
                   "r"(32u * 32u)
                   : "memory");
    __syncwarp();
    if (lane < 8) {
      int32_t row[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const uint64_t h = mix64((t + lane * 4 + j) * 0x9E3779B97F4A7C15ull + r * 0x632BE59BD9B4E019ull);
        row[j] = static_cast<int32_t>(__umulhi(static_cast<uint32_t>(h >> 32), nblk));
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      asm volatile(
          "cp.async.bulk.tensor.2d.shared::cta.global.tile::gather4.mbarrier::complete_tx::bytes"
          " [%0], [%1, {%2, %3, %4, %5, %6}], [%7];" ::"r"(smem_addr(&buf[w][s][lane * 32])),
          "l"(&tmap), "r"(0), "r"(row[0]), "r"(row[1]), "r"(row[2]), "r"(row[3]), "r"(bar)
          : "memory");
    }
  };
  for (int s = 0; s < kStages && s < iters; ++s) issue(s, s);
  uint32_t acc = 0, phase = 0;
  for (int r = 0; r < iters; ++r) {
    const int s = r % kStages;
    if (!mbar_wait(smem_addr(&bars[w][s]), (phase >> s) & 1)) {
      if (lane == 0) atomicAdd(err, 1u);
      // drain the other stages still in flight (bounded) before leaving
      for (int k = 1; k < kStages && r + k < iters; ++k) {
        const int s2 = (r + k) % kStages;
        mbar_wait(smem_addr(&bars[w][s2]), (phase >> s2) & 1);
      }
      break;
    }
    phase ^= 1u << s;
    const uint4* p = reinterpret_cast<const uint4*>(&buf[w][s][lane * 8]);
    const uint4 a = p[0], b = p[1];
    acc ^= a.x ^ a.w ^ b.x ^ b.w;
    __syncwarp();
    if (r + kStages < iters) issue(s, r + kStages);
  }
  if (acc == 0x12345678u) out[0] = acc;
}

// Hybrid: per round each lane also loads two random blocks with plain 256-bit
// loads (L1 no-allocate) while kTma blocks per warp arrive through gather4,
// to see whether the two paths add up.  kTma = 0 is the plain-load baseline.
template <int kTma>
__global__ void __launch_bounds__(kWarps * 32)
    hybrid_kernel(const __grid_constant__ CUtensorMap tmap, const uint32_t* __restrict__ f,
                  uint32_t nblk, int iters, uint32_t* out, unsigned* err) {
  constexpr int kBuf = kTma > 0 ? kTma * 8 : 8;
  __shared__ __align__(128) uint32_t buf[kWarps][kStages][kBuf];
  __shared__ __align__(8) uint64_t bars[kWarps][kStages];
  const unsigned lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (kTma > 0 && lane == 0) {
    for (int s = 0; s < kStages; ++s)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&bars[w][s])) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncwarp();
  const uint64_t t = (blockIdx.x * static_cast<uint64_t>(kWarps) + w) * 64;
  auto issue = [&](int s, int r) {
    if (kTma == 0) return;
    const uint32_t bar = smem_addr(&bars[w][s]);
    if (lane == 0)
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar),
                   "r"(static_cast<uint32_t>(kTma * 32))
                   : "memory");
    __syncwarp();
    if (lane < kTma / 4) {
      int32_t row[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const uint64_t h = mix64((t + lane * 4 + j) * 0x9E3779B97F4A7C15ull + r * 0x632BE59BD9B4E019ull + 7);
        row[j] = static_cast<int32_t>(__umulhi(static_cast<uint32_t>(h >> 32), nblk));
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      asm volatile(
          "cp.async.bulk.tensor.2d.shared::cta.global.tile::gather4.mbarrier::complete_tx::bytes"
          " [%0], [%1, {%2, %3, %4, %5, %6}], [%7];" ::"r"(smem_addr(&buf[w][s][lane * 32])),
          "l"(&tmap), "r"(0), "r"(row[0]), "r"(row[1]), "r"(row[2]), "r"(row[3]), "r"(bar)
          : "memory");
    }
  };
  for (int s = 0; s < kStages && s < iters; ++s) issue(s, s);
  uint32_t acc = 0, phase = 0;
  for (int r = 0; r < iters; ++r) {
    const int s = r % kStages;
    uint32_t v[2][8];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const uint64_t h = mix64((t + 2 * lane + q) * 0x9E3779B97F4A7C15ull + r * 0xD1B54A32D192ED03ull);
      const uint32_t b = __umulhi(static_cast<uint32_t>(h >> 32), nblk);
      asm volatile("ld.global.nc.L1::no_allocate.v8.u32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                   : "=r"(v[q][0]), "=r"(v[q][1]), "=r"(v[q][2]), "=r"(v[q][3]), "=r"(v[q][4]),
                     "=r"(v[q][5]), "=r"(v[q][6]), "=r"(v[q][7])
                   : "l"(f + 8ull * b));
    }
    if (kTma > 0) {
      if (!mbar_wait(smem_addr(&bars[w][s]), (phase >> s) & 1)) {
        if (lane == 0) atomicAdd(err, 1u);
        for (int k = 1; k < kStages && r + k < iters; ++k) {
          const int s2 = (r + k) % kStages;
          mbar_wait(smem_addr(&bars[w][s2]), (phase >> s2) & 1);
        }
        break;
      }
      phase ^= 1u << s;
#pragma unroll
      for (int q = 0; q < (kTma + 31) / 32; ++q) {
        const int row = q * 32 + static_cast<int>(lane);
        if (row < kTma) {
          const uint4* p = reinterpret_cast<const uint4*>(&buf[w][s][row * 8]);
          const uint4 a = p[0], b = p[1];
          acc ^= a.x ^ a.w ^ b.x ^ b.w;
        }
      }
      __syncwarp();
      if (r + kStages < iters) issue(s, r + kStages);
    }
#pragma unroll
    for (int q = 0; q < 2; ++q) acc ^= v[q][0] ^ v[q][3] ^ v[q][7];
  }
  if (acc == 0x12345678u) out[0] = acc;
}

template <int kTma>
static int run_hybrid(const CUtensorMap& tmap, const uint32_t* f, uint32_t nblk, int sms,
                      uint32_t* out, unsigned* err, cudaEvent_t a, cudaEvent_t b) {
  for (int cps : {2, 4}) {
    const int grid = sms * cps, iters = 512;
    hybrid_kernel<kTma><<<grid, kWarps * 32>>>(tmap, f, nblk, 8, out, err);
    CK(cudaDeviceSynchronize());
    CK(cudaEventRecord(a));
    hybrid_kernel<kTma><<<grid, kWarps * 32>>>(tmap, f, nblk, iters, out, err);
    CK(cudaEventRecord(b));
    CK(cudaEventSynchronize(b));
    float ms = 0;
    CK(cudaEventElapsedTime(&ms, a, b));
    unsigned e = 0;
    CK(cudaMemcpy(&e, err, 4, cudaMemcpyDeviceToHost));
    const double n = static_cast<double>(grid) * kWarps * (64 + kTma) * iters;
    std::printf("hybrid tma=%2d/warp-round %8.1f MiB cta/sm=%d: %7.1f G blocks/s  (timeouts %u)\n",
                kTma, nblk / 32768.0, cps, n / ms / 1e6, e);
  }
  return 0;
}

typedef CUresult (*EncodeTiled)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

int main() {
  int sms = 0;
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0));
  void* fn = nullptr;
  cudaDriverEntryPointQueryResult q;
  CK(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q));
  if (q != cudaDriverEntryPointSuccess || !fn) {
    std::printf("cuTensorMapEncodeTiled not available\n");
    return 1;
  }
  const uint64_t max_blocks = 1ull << 22;  // 128 MiB
  uint32_t *f = nullptr, *out = nullptr;
  unsigned* err = nullptr;
  CK(cudaMalloc(&f, max_blocks * 32));
  CK(cudaMalloc(&out, 64));
  CK(cudaMalloc(&err, 4));
  CK(cudaMemset(f, 0x5a, max_blocks * 32));
  CK(cudaMemset(err, 0, 4));
  cudaEvent_t a, b;
  CK(cudaEventCreate(&a));
  CK(cudaEventCreate(&b));
  for (uint32_t nblk : {32768u, 1u << 20, 1u << 22}) {
    CUtensorMap tmap;
    const cuuint64_t dims[2] = {8, nblk};
    const cuuint64_t strides[1] = {32};
    const cuuint32_t box[2] = {8, 1};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult r = reinterpret_cast<EncodeTiled>(fn)(
        &tmap, CU_TENSOR_MAP_DATA_TYPE_UINT32, 2, f, dims, strides, box, estr,
        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
      std::printf("encode failed: %d\n", static_cast<int>(r));
      return 1;
    }
    for (int cps : {2, 4, 8}) {
      const int grid = sms * cps, iters = 1024;
      gather_kernel<<<grid, kWarps * 32>>>(tmap, nblk, 8, out, err);
      CK(cudaDeviceSynchronize());
      CK(cudaEventRecord(a));
      gather_kernel<<<grid, kWarps * 32>>>(tmap, nblk, iters, out, err);
      CK(cudaEventRecord(b));
      CK(cudaEventSynchronize(b));
      float ms = 0;
      CK(cudaEventElapsedTime(&ms, a, b));
      unsigned e = 0;
      CK(cudaMemcpy(&e, err, 4, cudaMemcpyDeviceToHost));
      const double n = static_cast<double>(grid) * kWarps * 32 * iters;
      std::printf("gather4 %8.1f MiB cta/sm=%d: %7.1f G blocks/s  (wait timeouts %u)\n",
                  nblk / 32768.0, cps, n / ms / 1e6, e);
    }
    if (nblk <= (1u << 20)) {
      if (run_hybrid<0>(tmap, f, nblk, sms, out, err, a, b)) return 1;
      if (run_hybrid<16>(tmap, f, nblk, sms, out, err, a, b)) return 1;
      if (run_hybrid<32>(tmap, f, nblk, sms, out, err, a, b)) return 1;
      if (run_hybrid<24>(tmap, f, nblk, sms, out, err, a, b)) return 1;
    }
  }
  CK(cudaFree(f));
  return 0;
}
