// Stage 1 and 2 of the Ozaki-II flow (Sec. 4.1): shared exponents per row of A
// and per column of B (Sec. 4.2), integerization a_hat = RNE(a 2^(t-e))
// (Eq. 1) and the centered residues of a_hat for every modulus, written as
// bf16 int8-range planes in the K-major layout of the plane GEMM (Sec. 4.3,
// incl. the balanced base-128 split of two-limb residues, Eq. 4-5).
#include <cuda_bf16.h>
#include <climits>

#include "oz2_internal.h"

namespace oz2 {

// ---------------------------------------------------------------------------
// Exponent scan: e_i = max exp over the nonzero entries of row i of A,
// f_j = max exp over the nonzero entries of column j of B.  The outputs are
// preset to a sentinel below every valid exponent (memset 0x80) and combined
// with atomicMax, so the K range of one line may be split across blocks.
// Block list entry: {problem, side | kpart << 8, first line, kparts}.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_scan(DevTables T, const int4* __restrict__ blk) {
  const int4 b = blk[blockIdx.x];
  const ProbDev& P = T.probs[b.x];
  const int side = b.y & 0xff, kpart = b.y >> 8, kparts = b.w;
  const int K = P.K;
  const int kspan = (K + kparts - 1) / kparts;
  const int k_lo = kpart * kspan, k_hi = min(K, k_lo + kspan);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (side == 0) {
    // rows of A: one warp per row, lanes stride over k
    const int row = b.z + warp;
    if (row >= P.M) return;
    const uint64_t* top = P.a_limbs + (int64_t)(P.nl - 1) * P.a_ps + (int64_t)row * P.a_ld;
    const int32_t* ex = P.a_exp + (int64_t)row * P.a_ld;
    int best = INT_MIN;
    for (int k = k_lo + lane; k < k_hi; k += 32) {
      if (__ldg(top + k) != 0ull) best = max(best, __ldg(ex + k));
    }
    for (int o = 16; o; o >>= 1) best = max(best, __shfl_xor_sync(0xffffffffu, best, o));
    if (lane == 0 && best != INT_MIN) atomicMax(P.e + row, best);
  } else {
    // columns of B: 32 columns per block, the 8 warps split the k range
    __shared__ int red[8][32];
    const int col = b.z + lane;
    int best = INT_MIN;
    if (col < P.N) {
      const uint64_t* top = P.b_limbs + (int64_t)(P.nl - 1) * P.b_ps + col;
      const int32_t* ex = P.b_exp + col;
      for (int k = k_lo + warp; k < k_hi; k += 8) {
        if (__ldg(top + (int64_t)k * P.b_ld) != 0ull) best = max(best, __ldg(ex + (int64_t)k * P.b_ld));
      }
    }
    red[warp][lane] = best;
    __syncthreads();
    if (warp == 0) {
      for (int w = 1; w < 8; ++w) best = max(best, red[w][lane]);
      if (col < P.N && best != INT_MIN) atomicMax(P.f + col, best);
    }
  }
}

// ---------------------------------------------------------------------------
// Integerization + residues.
//
// One thread per element.  With sh = exp - e_line + t - 64 nl (<= 33), the
// magnitude is |a_hat| = floor(sig 2^sh) + rnd, where rnd is the
// round-half-even increment.  floor(sig 2^sh) is assembled as W16 16-bit
// digits; its residue mod m is sum_d dig_d (2^(16 d) mod m) (Sec. 5.3), and the
// increment is added after reduction, so no carry chain is ever formed.
// ---------------------------------------------------------------------------

__device__ __forceinline__ uint32_t barrett32(uint32_t x, uint32_t m, uint32_t mu) {
  // mu = floor(2^32 / m): the quotient estimate is low by at most 1
  uint32_t q = __umulhi(x, mu);
  uint32_t r = x - q * m;
  return r >= m ? r - m : r;
}

__device__ __forceinline__ uint32_t sig_word(const uint32_t* __restrict__ limbs32, int64_t ps,
                                             int64_t off, int nl, int j) {
  // 32-bit word j of the significand (little-endian), 0 outside [0, 2 nl)
  if (j < 0 || j >= 2 * nl) return 0u;
  return __ldg(limbs32 + 2 * ((int64_t)(j >> 1) * ps + off) + (j & 1));
}

// Digits of |a_hat| = floor(sig 2^sh) + rnd for one element, 16 bits each
// (the round-half-even increment rnd is added with a carry through the
// digits).  Returns false for a zero element.
template <int W16>
__device__ __forceinline__ bool element_digits(const uint32_t* __restrict__ limbs32, int64_t ps,
                                               int64_t off, int nl, int exp_el, int e_line, int t,
                                               uint32_t (&dig)[W16]) {
#pragma unroll
  for (int d = 0; d < W16; ++d) dig[d] = 0u;
  const int sh = exp_el - e_line + t - 64 * nl;   // <= t - 64 nl
  // E = sig * 2^64 (two zero words below); bit 0 of floor(sig 2^sh) is bit B of E, B >= 31
  const int B = 64 - sh;
  if (B - 1 >= 64 * nl + 64) return true;       // |a| 2^(t - e) < 1/2: rounds to 0
  const int ws = B >> 5, bs = B & 31;
#pragma unroll
  for (int w = 0; w < W16 / 2; ++w) {
    const uint32_t lo = sig_word(limbs32, ps, off, nl, ws + w - 2);
    const uint32_t hi = sig_word(limbs32, ps, off, nl, ws + w - 1);
    const uint32_t x = __funnelshift_r(lo, hi, bs);
    dig[2 * w] = x & 0xffffu;
    dig[2 * w + 1] = x >> 16;
  }
  // round-half-even: round bit = bit B-1 of E, sticky = the bits below it
  const int rbpos = B - 1;
  const uint32_t rw = sig_word(limbs32, ps, off, nl, (rbpos >> 5) - 2);
  const uint32_t rb = (rw >> (rbpos & 31)) & 1u;
  uint32_t sticky = rw & ((1u << (rbpos & 31)) - 1u);
  for (int j = (rbpos >> 5) - 3; j >= 0 && !sticky; --j) sticky |= sig_word(limbs32, ps, off, nl, j);
  uint32_t c = rb & ((sticky != 0u) | (dig[0] & 1u));
#pragma unroll
  for (int d = 0; d < W16; ++d) {                // |a_hat| <= 2^t fits the W16 digits
    const uint32_t x = dig[d] + c;
    dig[d] = x & 0xffffu;
    c = x >> 16;
  }
  return true;
}

__device__ __forceinline__ uint32_t bf16_bits(int r) {
  return __float_as_uint((float)r) >> 16;         // exact for |r| <= 256
}

// Centered residue of a_hat (sign s) from |a_hat| mod m: symmetric except for
// the even modulus 128, whose tie -64 maps to +64 (range (-m/2, m/2]).
__device__ __forceinline__ int centered(uint32_t r, uint32_t m, bool neg) {
  int x = (2 * r > m) ? (int)r - (int)m : (int)r;
  if (neg) x = -x;
  if (2 * x == -(int)m) x = -x;
  return x;
}

// Two horizontally adjacent elements per thread (k and k + 1): the digit
// table is read once for both, and each plane gets one 32-bit store of two
// bf16 values.  Block: 32 x 8 threads = 64 columns x 8 rows of elements.
template <int W16>
__global__ void __launch_bounds__(256) k_residue(DevTables T, const int4* __restrict__ blk) {
  extern __shared__ __align__(16) uint32_t s_t16[];   // [L][W16], then [L] x {m, mu, c24, 0}
  const int4 b = blk[blockIdx.x];
  const ProbDev& P = T.probs[b.x];
  const int side = b.y;
  const int L = P.L, L1 = P.L1;
  uint4* s_mc = reinterpret_cast<uint4*>(s_t16 + L * W16);
  for (int i = threadIdx.y * 32 + threadIdx.x; i < L * W16; i += 256) {
    const int l = i / W16, d = i - l * W16;
    s_t16[i] = T.t16[(int64_t)l * T.w16max + d];
  }
  for (int l = threadIdx.y * 32 + threadIdx.x; l < L; l += 256) {
    const ModConst mc = T.mods[l];
    s_mc[l] = make_uint4(mc.m, mc.mu, mc.c24, 0u);
  }
  __syncthreads();
  const int R = side ? P.N : P.M;
  const int r = b.z + threadIdx.y;
  const int k = b.w + 2 * threadIdx.x;
  if (r >= R || k >= P.K) return;
  const bool two = k + 1 < P.K;

  const uint64_t* limbs = side ? P.b_limbs : P.a_limbs;
  const int64_t ps = side ? P.b_ps : P.a_ps;
  const int64_t stride_k = side ? P.b_ld : 1;
  const int64_t off0 = side ? ((int64_t)k * P.b_ld + r) : ((int64_t)r * P.a_ld + k);
  const int64_t off1 = off0 + stride_k;
  const int32_t* exps = side ? P.b_exp : P.a_exp;
  const int8_t* signs = side ? P.b_sign : P.a_sign;
  const int nl = P.nl;
  const uint32_t* limbs32 = reinterpret_cast<const uint32_t*>(limbs);
  const int e_line = side ? P.f[r] : P.e[r];

  uint32_t d0[W16], d1[W16];
  bool n0 = false, n1 = false;
  {
    const bool nz = __ldg(limbs + (int64_t)(nl - 1) * ps + off0) != 0ull;
    if (nz) {
      element_digits<W16>(limbs32, ps, off0, nl, __ldg(exps + off0), e_line, P.t, d0);
      n0 = __ldg(signs + off0) != 0;
    } else {
#pragma unroll
      for (int d = 0; d < W16; ++d) d0[d] = 0u;
    }
  }
  {
    const bool nz = two && __ldg(limbs + (int64_t)(nl - 1) * ps + off1) != 0ull;
    if (nz) {
      element_digits<W16>(limbs32, ps, off1, nl, __ldg(exps + off1), e_line, P.t, d1);
      n1 = __ldg(signs + off1) != 0;
    } else {
#pragma unroll
      for (int d = 0; d < W16; ++d) d1[d] = 0u;
    }
  }

  uint16_t* planes = side ? P.pb : P.pa;
  const int64_t plane_stride = (int64_t)R * P.Kp;
  uint16_t* dst = planes + (int64_t)r * P.Kp + k;      // k even, Kp even: 4-byte aligned pairs
  auto put = [&](int x0, int x1) {                     // writes plane at dst, then moves to the next
    if (two) *reinterpret_cast<uint32_t*>(dst) = bf16_bits(x0) | (bf16_bits(x1) << 16);
    else *dst = (uint16_t)bf16_bits(x0);
    dst += plane_stride;
  };
  for (int l = 0; l < L; ++l) {
    const uint4 mcv = s_mc[l];
    struct { uint32_t m, mu, c24; } mc{mcv.x, mcv.y, mcv.z};
    const uint4* tl = reinterpret_cast<const uint4*>(s_t16 + l * W16);
    uint32_t r0, r1;
    if (l < L1) {
      uint32_t a0 = 0u, a1 = 0u;   // digits < 2^16, table < 2^8, <= 132 terms: < 2^32
#pragma unroll
      for (int q = 0; q < W16 / 4; ++q) {
        const uint4 t4 = tl[q];
        a0 += d0[4 * q] * t4.x + d0[4 * q + 1] * t4.y + d0[4 * q + 2] * t4.z + d0[4 * q + 3] * t4.w;
        a1 += d1[4 * q] * t4.x + d1[4 * q + 1] * t4.y + d1[4 * q + 2] * t4.z + d1[4 * q + 3] * t4.w;
      }
      r0 = barrett32(a0, mc.m, mc.mu);
      r1 = barrett32(a1, mc.m, mc.mu);
    } else {
      uint64_t a0 = 0ull, a1 = 0ull;   // < 2^30 * 132 < 2^38
#pragma unroll
      for (int q = 0; q < W16 / 4; ++q) {
        const uint4 t4 = tl[q];
        a0 += (uint64_t)d0[4 * q] * t4.x + (uint64_t)d0[4 * q + 1] * t4.y +
              (uint64_t)d0[4 * q + 2] * t4.z + (uint64_t)d0[4 * q + 3] * t4.w;
        a1 += (uint64_t)d1[4 * q] * t4.x + (uint64_t)d1[4 * q + 1] * t4.y +
              (uint64_t)d1[4 * q + 2] * t4.z + (uint64_t)d1[4 * q + 3] * t4.w;
      }
      r0 = barrett32((uint32_t)(a0 >> 24) * mc.c24 + (uint32_t)(a0 & 0xffffffu), mc.m, mc.mu);
      r1 = barrett32((uint32_t)(a1 >> 24) * mc.c24 + (uint32_t)(a1 & 0xffffffu), mc.m, mc.mu);
    }
    const int x0 = centered(r0, mc.m, n0);
    const int x1 = centered(r1, mc.m, n1);
    if (l < L1) {
      put(x0, x1);                                   // plane l
    } else {
      // balanced base-128 split: r = r0 + 128 r1 with r0 = cen(r mod 128);
      // planes L1 + 3 (l - L1) + {0, 1, 2} = r0, r1, r0 + r1
      const int y0 = x0 & 127, y1 = x1 & 127;
      const int lo0 = y0 > 64 ? y0 - 128 : y0, lo1 = y1 > 64 ? y1 - 128 : y1;
      const int hi0 = (x0 - lo0) >> 7, hi1 = (x1 - lo1) >> 7;
      put(lo0, lo1);
      put(hi0, hi1);
      put(lo0 + hi0, lo1 + hi1);
    }
  }
}

static const int kResidueW16[] = {8, 12, 20, 36, 68, 132};
static const int kNumResidueClasses = 6;

int residue_class_for(int w16) {
  for (int i = 0; i < kNumResidueClasses; ++i)
    if (w16 <= kResidueW16[i]) return i;
  return -1;
}
int residue_class_w16(int cls) { return kResidueW16[cls]; }

cudaError_t launch_scan(const DevTables& t, int /*count*/, const int32_t* blk_rows,
                        const int32_t* blk_cols, int nblk_rows, int nblk_cols, cudaStream_t s) {
  if (nblk_rows) k_scan<<<nblk_rows, 256, 0, s>>>(t, reinterpret_cast<const int4*>(blk_rows));
  if (nblk_cols) k_scan<<<nblk_cols, 256, 0, s>>>(t, reinterpret_cast<const int4*>(blk_cols));
  return cudaGetLastError();
}

template <int W16>
static cudaError_t launch_res_w(const DevTables& t, const int4* blk, int nblk, int smem,
                                cudaStream_t s) {
  k_residue<W16><<<nblk, dim3(32, 8), smem, s>>>(t, blk);
  return cudaGetLastError();
}

// Dynamic shared memory above 48 KB needs an opt-in per kernel; done once,
// before any launch (and so before any stream capture).
cudaError_t init_prep_attributes() {
  const int mx = 200 * 1024;
  cudaError_t e = cudaSuccess;
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_residue<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_residue<12>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_residue<20>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_residue<36>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_residue<68>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_residue<132>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
  return e;
}

cudaError_t launch_residues(const DevTables& t, int cls, const int32_t* blk_list, int nblk,
                            int smem_bytes, cudaStream_t s) {
  const int4* blk = reinterpret_cast<const int4*>(blk_list);
  if (nblk == 0) return cudaSuccess;
  switch (cls) {
    case 0: return launch_res_w<8>(t, blk, nblk, smem_bytes, s);
    case 1: return launch_res_w<12>(t, blk, nblk, smem_bytes, s);
    case 2: return launch_res_w<20>(t, blk, nblk, smem_bytes, s);
    case 3: return launch_res_w<36>(t, blk, nblk, smem_bytes, s);
    case 4: return launch_res_w<68>(t, blk, nblk, smem_bytes, s);
    case 5: return launch_res_w<132>(t, blk, nblk, smem_bytes, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace oz2
