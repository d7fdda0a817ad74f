// Throughput probe of the warp-level INT8 tensor-core instruction
// (mma.sync m16n8k32, s8 x s8 -> s32), used to state the INT8 peak that the
// plane GEMMs' exact-integer rate is compared with.  sm_103a accepts this
// legacy instruction but not tcgen05.mma kind::i8, so it is the only INT8
// tensor path a kernel can issue on this GPU.
//
// Each warp runs `iters` rounds of kChains independent MMAs on register
// operands (no memory traffic in the loop); the accumulators are consumed by
// one guarded store so that the compiler keeps every MMA.
#include "oz2_internal.h"

namespace oz2 {

namespace {

constexpr int kChains = 8;

__device__ __forceinline__ void mma_s8(int (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k32.row.col.s32.s8.s8.s32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
      "{%0, %1, %2, %3};"
      : "+r"(d[0]), "+r"(d[1]), "+r"(d[2]), "+r"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__global__ void __launch_bounds__(256) k_probe_mma_s8(int iters, int* sink) {
  const uint32_t x = threadIdx.x * 0x01010101u + blockIdx.x;
  uint32_t a[4] = {x, x ^ 0x5a5a5a5au, x + 0x01020304u, ~x};
  uint32_t b[2] = {x * 3u, x ^ 0x3c3c3c3cu};
  int acc[kChains][4];
#pragma unroll
  for (int c = 0; c < kChains; ++c)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[c][q] = 0;
#pragma unroll 1
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) mma_s8(acc[c], a, b);
  }
  int s = 0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += acc[c][0] ^ acc[c][1] ^ acc[c][2] ^ acc[c][3];
  if (s == 0x7fffffff) sink[0] = s;    // practically never taken; keeps the MMAs live
}

}  // namespace

}  // namespace oz2

extern "C" int ozaki2_probe_mma_s8(int blocks, int iters, int* sink, double* tops, void* stream) {
  if (blocks <= 0 || iters <= 0 || !sink || !tops) return OZ2_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess) return OZ2_ECUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return OZ2_ECUDA;
  }
  int rc = OZ2_OK;
  oz2::k_probe_mma_s8<<<blocks, 256, 0, s>>>(1, sink);    // warm-up launch
  if (cudaGetLastError() != cudaSuccess || cudaEventRecord(e0, s) != cudaSuccess) rc = OZ2_ECUDA;
  if (!rc) {
    oz2::k_probe_mma_s8<<<blocks, 256, 0, s>>>(iters, sink);
    if (cudaGetLastError() != cudaSuccess || cudaEventRecord(e1, s) != cudaSuccess ||
        cudaEventSynchronize(e1) != cudaSuccess)
      rc = OZ2_ECUDA;
  }
  float ms = 0.f;
  if (!rc && cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) rc = OZ2_ECUDA;
  if (!rc) {
    // one m16n8k32 MMA = 16 x 8 x 32 multiply-adds = 8192 integer operations
    const double ops = 8192.0 * oz2::kChains * (double)iters * (double)blocks * (256 / 32);
    *tops = ops / (ms * 1e-3) / 1e12;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return rc;
}
