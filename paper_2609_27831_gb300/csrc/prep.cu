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

template <int W16>
__global__ void __launch_bounds__(256) k_residue(DevTables T, const int4* __restrict__ blk) {
  extern __shared__ uint32_t s_t16[];          // [L][W16]
  const int4 b = blk[blockIdx.x];
  const ProbDev& P = T.probs[b.x];
  const int side = b.y;
  const int L = P.L, L1 = P.L1;
  for (int i = threadIdx.y * 32 + threadIdx.x; i < L * W16; i += 256) {
    const int l = i / W16, d = i - l * W16;
    s_t16[i] = T.t16[(int64_t)l * T.w16max + d];
  }
  __syncthreads();
  const int R = side ? P.N : P.M;
  const int r = b.z + threadIdx.y;
  const int k = b.w + threadIdx.x;
  if (r >= R || k >= P.K) return;

  const uint64_t* limbs = side ? P.b_limbs : P.a_limbs;
  const int64_t ps = side ? P.b_ps : P.a_ps;
  const int64_t off = side ? ((int64_t)k * P.b_ld + r) : ((int64_t)r * P.a_ld + k);
  const int32_t* exps = side ? P.b_exp : P.a_exp;
  const int8_t* signs = side ? P.b_sign : P.a_sign;
  const int nl = P.nl;
  const uint32_t* limbs32 = reinterpret_cast<const uint32_t*>(limbs);

  uint32_t dig[W16];
#pragma unroll
  for (int d = 0; d < W16; ++d) dig[d] = 0u;
  uint32_t rnd = 0u;
  bool neg = false;
  const bool nonzero = __ldg(limbs + (int64_t)(nl - 1) * ps + off) != 0ull;
  if (nonzero) {
    const int e_line = side ? P.f[r] : P.e[r];
    const int sh = __ldg(exps + off) - e_line + P.t - 64 * nl;   // <= t - 64 nl
    neg = __ldg(signs + off) != 0;
    // E = sig * 2^64 (two zero words below); mag bit 0 is bit B of E, B >= 31
    const int B = 64 - sh;
    const int nbits_e = 64 * nl + 64;
    if (B - 1 < nbits_e) {
      const int ws = B >> 5, bs = B & 31;
#pragma unroll
      for (int w = 0; w < W16 / 2; ++w) {
        const uint32_t lo = sig_word(limbs32, ps, off, nl, ws + w - 2);
        const uint32_t hi = sig_word(limbs32, ps, off, nl, ws + w - 1);
        const uint32_t x = __funnelshift_r(lo, hi, bs);
        dig[2 * w] = x & 0xffffu;
        dig[2 * w + 1] = x >> 16;
      }
      // round-half-even: round bit = bit B-1 of E, sticky = bits below it
      const int rbpos = B - 1;
      const uint32_t rw = sig_word(limbs32, ps, off, nl, (rbpos >> 5) - 2);
      const uint32_t rb = (rw >> (rbpos & 31)) & 1u;
      uint32_t sticky = rw & ((1u << (rbpos & 31)) - 1u);
      for (int j = (rbpos >> 5) - 3; j >= 0 && !sticky; --j) sticky |= sig_word(limbs32, ps, off, nl, j);
      rnd = rb & ((sticky != 0u) | (dig[0] & 1u));
    }
  }

  uint16_t* planes = side ? P.pb : P.pa;
  const int64_t plane_stride = (int64_t)R * P.Kp;
  uint16_t* dst = planes + (int64_t)r * P.Kp + k;
  for (int l = 0; l < L; ++l) {
    const ModConst mc = T.mods[l];
    const uint32_t* tl = s_t16 + l * W16;
    uint32_t res;
    if (l < L1) {
      uint32_t acc = 0u;   // dig < 2^16, table < 2^8, W16 <= 132 terms: < 2^32
#pragma unroll
      for (int d = 0; d < W16; ++d) acc += dig[d] * tl[d];
      res = barrett32(acc, mc.m, mc.mu);
    } else {
      uint64_t acc = 0ull; // < 2^30 * 132 < 2^38
#pragma unroll
      for (int d = 0; d < W16; ++d) acc += (uint64_t)dig[d] * tl[d];
      const uint32_t y = (uint32_t)(acc >> 24) * mc.c24 + (uint32_t)(acc & 0xffffffu);   // < 2^29
      res = barrett32(y, mc.m, mc.mu);
    }
    res += rnd;
    if (res >= mc.m) res -= mc.m;
    if (neg && res) res = mc.m - res;
    const int rs = (2 * res > mc.m) ? (int)res - (int)mc.m : (int)res;   // (-m/2, m/2]
    if (l < L1) {
      dst[(int64_t)l * plane_stride] = (uint16_t)(__float_as_uint((float)rs) >> 16);
    } else {
      const int x = rs & 127;
      const int r0 = x > 64 ? x - 128 : x;        // cen(r mod 128)
      const int r1 = (rs - r0) >> 7;              // exact
      const int64_t g = L1 + 3 * (l - L1);
      dst[g * plane_stride] = (uint16_t)(__float_as_uint((float)r0) >> 16);
      dst[(g + 1) * plane_stride] = (uint16_t)(__float_as_uint((float)r1) >> 16);
      dst[(g + 2) * plane_stride] = (uint16_t)(__float_as_uint((float)(r0 + r1)) >> 16);
    }
  }
}

static const int kResidueW16[] = {6, 10, 20, 36, 68, 132};
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
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_residue<6>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_residue<10>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
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
    case 0: return launch_res_w<6>(t, blk, nblk, smem_bytes, s);
    case 1: return launch_res_w<10>(t, blk, nblk, smem_bytes, s);
    case 2: return launch_res_w<20>(t, blk, nblk, smem_bytes, s);
    case 3: return launch_res_w<36>(t, blk, nblk, smem_bytes, s);
    case 4: return launch_res_w<68>(t, blk, nblk, smem_bytes, s);
    case 5: return launch_res_w<132>(t, blk, nblk, smem_bytes, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace oz2
