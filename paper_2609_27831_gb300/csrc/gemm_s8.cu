// Stages 3-4 of the Ozaki-II flow (Sec. 4.1) with the literal INT8 x INT8 ->
// INT32 product of the paper (Sec. 2.4, Sec. 4.3): the second plane GEMM
// engine, for comparison with the bf16 tcgen05 kernels at equal accuracy.
// sm_103a offers no tcgen05 INT8 form, so this engine issues the warp-level
// mma.sync.m16n8k32.s8.s8.s32; its INT32 accumulators are exact for
// K * 127^2 < 2^31 (every K this library accepts), so no K chunking is needed.
//
// Block = one 128 x 128 half of a (modulus, 128 x 256 output tile) unit, two
// blocks per SM.  The residue planes are bf16 in HBM (as the tcgen05 engines
// read them); each block converts its K-slices to int8 while staging them in
// shared memory (double-buffered through registers), and 8 warps (2 x 4) each
// own a 64 x 32 piece of the tile: 4 x 4 MMAs per K step of 32.  A unit's
// planes run one after the other; each plane's exact sum is reduced mod m and
// added, times its Karatsuba coefficient (one-limb: 1; two-limb:
// -127 P0 + 128 Ps + 16256 P2, Eq. 4), to a running residue kept in shared
// memory (16 bits per output); the result times M_l^{-1} mod m_l is the CRT's
// v_l (Sec. 4.4), stored as the tcgen05 engines store it.
// Entry: {unit index (units in (problem, modulus, tile) order), half, 0, 0}.
#include "oz2_internal.h"

namespace oz2 {

namespace {

constexpr int kS8Threads = 256;
constexpr int kS8Rows = 128;          // rows of A and of B (output columns) per block
constexpr int kS8K = 32;              // K step (one m16n8k32)
constexpr int kS8Stride = 48;         // bytes per staged row: 32 data + 16 pad (conflict-free fragments)

__device__ __forceinline__ void mma_s8(int (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                       uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k32.row.col.s32.s8.s8.s32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
      "{%0, %1, %2, %3};"
      : "+r"(d[0]), "+r"(d[1]), "+r"(d[2]), "+r"(d[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// x mod m for an exact integer |x| < 2^31: x + a multiple of m that makes it
// non-negative and below 2^32, then Barrett reduction with floor(2^32 / m)
// (the quotient estimate is low by at most one, so one correction suffices).
__device__ __forceinline__ uint32_t mod_s32(int x, uint32_t m, uint32_t mu, uint32_t off) {
  const uint32_t y = (uint32_t)x + off;
  const uint32_t q = __umulhi(y, mu);
  uint32_t r = y - q * m;
  return r >= m ? r - m : r;
}
__device__ __forceinline__ uint32_t mod_u32(uint32_t y, uint32_t m, uint32_t mu) {
  const uint32_t q = __umulhi(y, mu);
  uint32_t r = y - q * m;
  return r >= m ? r - m : r;
}

// 8 bf16 integers in [-127, 127] -> 8 int8, packed little-endian in two words
__device__ __forceinline__ uint2 bf16x8_to_s8(uint4 w) {
  auto cv = [](uint32_t h) -> uint32_t {    // one bf16 in the low 16 bits -> its int8 byte
    return (uint32_t)__float2int_rn(__uint_as_float(h << 16)) & 0xffu;
  };
  uint2 o;
  o.x = cv(w.x & 0xffffu) | (cv(w.x >> 16) << 8) | (cv(w.y & 0xffffu) << 16) | (cv(w.y >> 16) << 24);
  o.y = cv(w.z & 0xffffu) | (cv(w.z >> 16) << 8) | (cv(w.w & 0xffffu) << 16) | (cv(w.w >> 16) << 24);
  return o;
}

// The 16-byte chunks of one 128 x 32 bf16 slice that a thread loads: chunk
// c = tid + 256 i (i = 0, 1) covers row c / 4, k offset 8 (c % 4).  Entries at
// rows >= R or k >= K are zero (the plane's K padding is not written).
__device__ __forceinline__ void load_slice(const uint16_t* plane, int64_t Kp, int row0, int R, int k0, int K,
                                           uint4 (&v)[2]) {
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const int c = threadIdx.x + kS8Threads * i;
    const int row = row0 + (c >> 2), k = k0 + 8 * (c & 3);
    uint4 w = make_uint4(0u, 0u, 0u, 0u);
    if (row < R && k < K) {
      w = __ldg(reinterpret_cast<const uint4*>(plane + (int64_t)row * Kp + k));
      const int left = K - k;                     // mask the entries at k >= K
      if (left < 8) {
        uint32_t* ww = reinterpret_cast<uint32_t*>(&w);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          if (2 * q >= left) ww[q] = 0u;
          else if (2 * q + 1 >= left) ww[q] &= 0xffffu;
        }
      }
    }
    v[i] = w;
  }
}
__device__ __forceinline__ void store_slice(uint8_t* s, const uint4 (&v)[2]) {
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const int c = threadIdx.x + kS8Threads * i;
    *reinterpret_cast<uint2*>(s + (c >> 2) * kS8Stride + 8 * (c & 3)) = bf16x8_to_s8(v[i]);
  }
}

__global__ void __launch_bounds__(kS8Threads, 2) k_gemm_s8(const __grid_constant__ DevTables T,
                                                          const int4* __restrict__ list) {
  extern __shared__ __align__(16) uint8_t s8_smem[];
  uint8_t (*sA)[kS8Rows * kS8Stride] = reinterpret_cast<uint8_t (*)[kS8Rows * kS8Stride]>(s8_smem);
  uint8_t (*sB)[kS8Rows * kS8Stride] = sA + 2;
  uint16_t* sRes = reinterpret_cast<uint16_t*>(s8_smem + 4 * kS8Rows * kS8Stride);   // thread t's 64 at t + 256 i
  const int4 e = list[blockIdx.x];
  const Unit u = T.units[e.x];
  const ProbDev& P = T.probs[u.prob];
  const ModConst mc = T.mods[u.ell];
  const uint32_t m = mc.m, mu = mc.mu;
  const uint32_t off = (uint32_t)(((1ull << 31) + m - 1) / m * m);   // multiple of m >= 2^31
  const bool two = u.ell >= P.L1;
  const int g0 = two ? P.L1 + 3 * (u.ell - P.L1) : u.ell;
  const int row0 = u.tm * kBM, col0 = u.tn * kBN + e.y * kS8Rows;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int wm = warp >> 2, wn = warp & 3;          // 2 x 4 warps, 64 x 32 each
  const int gid = lane >> 2, tig = lane & 3;
  const int64_t psA = (int64_t)P.M * P.Kp, psB = (int64_t)P.N * P.Kp;

  const int nplanes = two ? 3 : 1;
  int acc[4][4][4];                                // a plane's exact sums; after the last plane, u_l
  for (int pi = 0; pi < nplanes; ++pi) {
    // planes r0 r0', r1 r1', (r0 + r1)(r0' + r1') with coefficients -127, 16256, 128 (Eq. 4)
    const int g = g0 + pi;
    const uint32_t coef = !two ? 1u : (pi == 0 ? (m - 127u % m) % m : (pi == 1 ? 16256u % m : 128u % m));
    const uint16_t* pa = P.pa + (int64_t)g * psA;
    const uint16_t* pb = P.pb + (int64_t)g * psB;
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[a][b][c] = 0;
    uint4 va[2], vb[2];
    load_slice(pa, P.Kp, row0, P.M, 0, P.K, va);
    load_slice(pb, P.Kp, col0, P.N, 0, P.K, vb);
    __syncthreads();                               // the previous plane's last reads of the buffers
    store_slice(sA[0], va);
    store_slice(sB[0], vb);
    __syncthreads();
    int buf = 0;
    for (int k0 = 0; k0 < P.K; k0 += kS8K) {
      const bool more = k0 + kS8K < P.K;
      if (more) {                                  // the next slices, in flight during the MMAs
        load_slice(pa, P.Kp, row0, P.M, k0 + kS8K, P.K, va);
        load_slice(pb, P.Kp, col0, P.N, k0 + kS8K, P.K, vb);
      }
      const uint8_t* A_ = sA[buf];
      const uint8_t* B_ = sB[buf];
      uint32_t bf[4][2];
#pragma unroll
      for (int nt = 0; nt < 4; ++nt) {
        const uint8_t* bp = B_ + (wn * 32 + nt * 8 + gid) * kS8Stride + 4 * tig;
        bf[nt][0] = *reinterpret_cast<const uint32_t*>(bp);
        bf[nt][1] = *reinterpret_cast<const uint32_t*>(bp + 16);
      }
#pragma unroll
      for (int mt = 0; mt < 4; ++mt) {
        const uint8_t* ap = A_ + (wm * 64 + mt * 16 + gid) * kS8Stride + 4 * tig;
        const uint32_t a0 = *reinterpret_cast<const uint32_t*>(ap);
        const uint32_t a1 = *reinterpret_cast<const uint32_t*>(ap + 8 * kS8Stride);
        const uint32_t a2 = *reinterpret_cast<const uint32_t*>(ap + 16);
        const uint32_t a3 = *reinterpret_cast<const uint32_t*>(ap + 8 * kS8Stride + 16);
#pragma unroll
        for (int nt = 0; nt < 4; ++nt) mma_s8(acc[mt][nt], a0, a1, a2, a3, bf[nt][0], bf[nt][1]);
      }
      if (more) {
        store_slice(sA[buf ^ 1], va);
        store_slice(sB[buf ^ 1], vb);
      }
      __syncthreads();
      buf ^= 1;
    }
    // the plane's exact sums, reduced and weighted into the running residue
    // (each thread reads and writes only its own 64 entries of sRes)
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          uint32_t r = mod_s32(acc[a][b][c], m, mu, off);
          if (coef != 1u) r = mod_u32(r * coef, m, mu);
          uint16_t& slot = sRes[threadIdx.x + kS8Threads * (16 * a + 4 * b + c)];
          if (pi > 0) r = mod_u32(r + slot, m, mu);
          if (pi + 1 < nplanes) slot = (uint16_t)r;
          else acc[a][b][c] = (int)r;                // the unit's u_l, kept for the store
        }
  }
  // v_l = u_l M_l^{-1} mod m_l, stored as the tcgen05 engines store it
  const uint32_t minv = __ldg(crt_view(T.crt_pool, P).Minv + u.ell);
  uint16_t* ub = P.u + (int64_t)u.ell * P.upitch;
#pragma unroll
  for (int mt = 0; mt < 4; ++mt)
#pragma unroll
    for (int nt = 0; nt < 4; ++nt)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int row = row0 + wm * 64 + mt * 16 + gid + 8 * h;
        const int col = col0 + wn * 32 + nt * 8 + 2 * tig;
        if (row >= P.M) continue;
        const uint32_t v0 = mod_u32((uint32_t)acc[mt][nt][2 * h] * minv, m, mu);
        const uint32_t v1 = mod_u32((uint32_t)acc[mt][nt][2 * h + 1] * minv, m, mu);
        if (col < P.N) ub[(int64_t)row * P.N + col] = (uint16_t)v0;
        if (col + 1 < P.N) ub[(int64_t)row * P.N + col + 1] = (uint16_t)v1;
      }
}

}  // namespace

constexpr int kS8Smem = 4 * kS8Rows * kS8Stride + kS8Threads * 64 * 2;   // two double-buffered slices, residues

cudaError_t init_gemm_s8_attributes() {
  return cudaFuncSetAttribute(k_gemm_s8, cudaFuncAttributeMaxDynamicSharedMemorySize, kS8Smem);
}

cudaError_t launch_gemm_s8(const DevTables& t, const int32_t* list, int n, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  k_gemm_s8<<<n, kS8Threads, kS8Smem, s>>>(t, reinterpret_cast<const int4*>(list));
  return cudaGetLastError();
}

}  // namespace oz2
