// Stage 1 and 2 of the Ozaki-II flow (Sec. 4.1): shared exponents per row of A
// and per column of B (Sec. 4.2), integerization a_hat = RNE(a 2^(t-e))
// (Eq. 1) and the centered residues of a_hat for every modulus, written as
// bf16 int8-range planes in the K-major layout of the plane GEMM (Sec. 4.3,
// incl. the balanced base-128 split of two-limb residues, Eq. 4-5).
#include <cuda_bf16.h>
#include <algorithm>
#include <climits>

#include "oz2_internal.h"
#include "tc_ptx.cuh"

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

// Plane stores of the CUDA-core residues as global-space stores: the compiler
// then knows they cannot alias the shared-memory tables, and may read the next
// modulus's table row ahead of them (about 1 % at 1024^3, p = 256).
__device__ __forceinline__ void st_plane(uint16_t* p, uint32_t bits) { __stcg(reinterpret_cast<unsigned short*>(p), (unsigned short)bits); }
__device__ __forceinline__ void st_plane2(uint16_t* p, uint32_t v) { __stcg(reinterpret_cast<unsigned int*>(p), v); }
__device__ __forceinline__ void st_plane4(uint16_t* p, uint2 v) { __stcg(reinterpret_cast<uint2*>(p), v); }

// Bytes b0, b1 (sel 0x5140) or b2, b3 (sel 0x7362) of x as an f16 pair (low
// half first): the byte permute puts each byte under the f16 exponent bits of
// 2^10 (0x64), where the mantissa's unit is 1, giving 1024 + b exactly; one
// packed subtraction of 1024 leaves b.
__device__ __forceinline__ uint32_t f16_byte_pair(uint32_t x, uint32_t sel) {
  uint32_t r;
  asm("sub.rn.f16x2 %0, %1, %2;" : "=r"(r) : "r"(__byte_perm(x, 0x64646464u, sel)), "r"(0x64006400u));
  return r;
}

__device__ __forceinline__ uint32_t bf16_bits(int r) {
  // bf16 bits of a small integer (|r| <= 256, exact) without an int->float
  // conversion: 1.5 * 2^23 + r has r in its low mantissa bits
  return __float_as_uint(__int_as_float(0x4B400000 + r) - 12582912.0f) >> 16;
}

// Centered residue of a_hat (sign s) from |a_hat| mod m: symmetric except for
// the even modulus 128, whose tie -64 maps to +64 (range (-m/2, m/2]).
__device__ __forceinline__ int centered(uint32_t r, uint32_t m, bool neg) {
  int x = (2 * r > m) ? (int)r - (int)m : (int)r;
  if (neg) x = -x;
  if (2 * x == -(int)m) x = -x;
  return x;
}

// Words of |a_hat| = floor(sig 2^sh) + rnd for one element (32 bits each,
// the round-half-even increment carried through the words).  A zero element
// gives zero words.
template <int W32>
__device__ __forceinline__ void element_words(const uint64_t* __restrict__ limbs, int64_t ps, int64_t off,
                                              int nl, int exp_el, int e_line, int t, uint32_t (&wd)[W32]) {
#pragma unroll
  for (int w = 0; w < W32; ++w) wd[w] = 0u;
  const int sh = exp_el - e_line + t - 64 * nl;   // <= t - 64 nl
  const int B = 64 - sh;                          // bit of S = sig 2^64 that is bit 0 of the magnitude
  if (B - 1 >= 64 * nl + 64) return;              // |a| 2^(t - e) < 1/2: rounds to 0
  // 64-bit limbs S[j] (S[0] = 0, S[j] = limb j - 1; 0 outside, with no
  // read), all in flight at once: lq - 2 .. lq + W32/2 cover the round bit
  // (limb lq or lq - 1), the first sticky limbs and the words ws .. ws + W32
  // of the magnitude
  auto S = [&](int j) -> uint64_t {
    return (unsigned)(j - 1) < (unsigned)nl ? __ldg(limbs + (int64_t)(j - 1) * ps + off) : 0ull;
  };
  const int ws = B >> 5, bs = B & 31, lq = ws >> 1;
  const bool odd = ws & 1;
  constexpr int NLM = W32 / 2 + 3;
  uint64_t lm[NLM];
#pragma unroll
  for (int q = 0; q < NLM; ++q) lm[q] = S(lq - 2 + q);
  auto word = [&](int x) -> uint32_t {            // word ws + x of S
    const uint32_t a = (x & 1) ? (uint32_t)(lm[2 + (x >> 1)] >> 32) : (uint32_t)lm[2 + (x >> 1)];
    const uint32_t b = (x & 1) ? (uint32_t)lm[2 + ((x + 1) >> 1)] : (uint32_t)(lm[2 + (x >> 1)] >> 32);
    return odd ? b : a;
  };
#pragma unroll
  for (int w = 0; w < W32; ++w) wd[w] = __funnelshift_r(word(w), word(w + 1), bs);
  const int rbpos = B - 1;
  const bool rb_hi = (rbpos >> 6) == lq;          // round bit in limb lq (else lq - 1)
  const uint64_t srb = rb_hi ? lm[2] : lm[1];
  const uint32_t rb = (uint32_t)(srb >> (rbpos & 63)) & 1u;
  uint64_t sticky = (srb & ((1ull << (rbpos & 63)) - 1ull)) | (rb_hi ? lm[1] : 0ull) | lm[0];
  for (int j = lq - 3; j >= 1 && !sticky; --j) sticky |= S(j);
  uint32_t c = rb & ((sticky != 0ull) | (wd[0] & 1u));
#pragma unroll
  for (int w = 0; w < W32; ++w) {                 // |a_hat| <= 2^t fits the W32 words
    const uint32_t x = wd[w] + c;
    c = (c && x == 0u) ? 1u : 0u;
    wd[w] = x;
  }
}

// Elements per thread of the CUDA-core residue kernel: four while their
// words fit in registers, else two.
__host__ __device__ constexpr int residue_ept(int w32) { return w32 <= 10 ? 4 : 2; }

// Centered residue of s |a_hat| mod m from a = sum of the byte products
// (a == |a_hat| mod m, a < 2^23), in fp32: f = s a exactly; q = f / m rounded
// to nearest (the 1.5 2^23 addend rounds; q may be off by one because 1/m is
// rounded), r = f - q m exactly (an fma of integers below 2^24), and one
// step in each direction brings r into (-m/2, m/2] (ties: +m/2).  The result
// is an exact small integer; + 0 turns a -0 into +0.
__device__ __forceinline__ float centered_f32(uint32_t a, bool neg, float mf, float rcp, float hm) {
  float f = __uint_as_float(a | 0x4B000000u) - 8388608.0f;
  if (neg) f = -f;
  const float q = fmaf(f, rcp, 12582912.0f) - 12582912.0f;
  float r = fmaf(-q, mf, f);
  r = r > hm ? r - mf : r;
  r = r <= -hm ? r + mf : r;
  return r + 0.0f;
}

// Residues of EPT elements over all L moduli from their first NW words, and
// the plane writes.  The table row of modulus l holds the packed low bytes of
// 2^(8 b) mod m_l in words [0, W32) and the high bytes in words [W32, 2 W32).
// s_mc[l] = {m, floor(2^32 / m), 1/m (fp32 bits), m/2 (fp32 bits)}.  Byte
// sums stay below 4 NW 255^2 < 2^23 for NW <= 32, so their reduction is done
// in fp32 there (Barrett beyond, with lo + 256 hi < 2^32 for two-limb moduli).
template <int NW, int W32, int EPT>
__device__ __forceinline__ void residue_planes(const uint32_t (&w)[EPT][W32], const bool (&ng)[EPT],
                                               const uint32_t* s_t8, const uint4* s_mc, int L, int L1,
                                               uint16_t* dst, int64_t plane_stride, int nk) {
  static_assert(EPT == 2 || EPT == 4, "two or four elements per thread");
  constexpr int RS = 2 * W32;
  // per element: s a = fma(s, 2^23 + a, -s 2^23) exactly, +0 for a = 0
  float sg[EPT], sb[EPT];
#pragma unroll
  for (int e = 0; e < EPT; ++e) {
    sg[e] = ng[e] ? -1.f : 1.f;
    sb[e] = ng[e] ? 8388608.f : -8388608.f;
  }
  // one plane of the EPT elements: one vector store when all are in range;
  // bits[e] holds the value's bf16 bits in its high half (an exact fp32), two
  // of them packed by one byte permutation
  auto put = [&](const uint32_t (&bits)[EPT]) {
    if (nk == EPT) {
      if (EPT == 4) {
        st_plane4(dst, make_uint2(__byte_perm(bits[0], bits[1], 0x7632), __byte_perm(bits[2], bits[3], 0x7632)));
      } else {
        st_plane2(dst, __byte_perm(bits[0], bits[1], 0x7632));
      }
    } else {
#pragma unroll
      for (int e = 0; e < EPT; ++e)
        if (e < nk) st_plane(dst + e, bits[e] >> 16);
    }
    dst += plane_stride;
  };
  for (int l = 0; l < L; ++l) {
    const uint4 mcv = s_mc[l];
    const uint32_t* tw = s_t8 + l * RS;
    const uint2* tl = reinterpret_cast<const uint2*>(tw);
    if (l < L1) {
      uint32_t a[EPT];
#pragma unroll
      for (int e = 0; e < EPT; ++e) a[e] = 0u;
#pragma unroll
      for (int q = 0; q < NW / 2; ++q) {
        const uint2 t2 = tl[q];
#pragma unroll
        for (int e = 0; e < EPT; ++e) {
          a[e] = __dp4a(w[e][2 * q], t2.x, a[e]);
          a[e] = __dp4a(w[e][2 * q + 1], t2.y, a[e]);
        }
      }
      if (NW & 1) {
        const uint32_t tx = tw[NW - 1];
#pragma unroll
        for (int e = 0; e < EPT; ++e) a[e] = __dp4a(w[e][NW - 1], tx, a[e]);
      }
      uint32_t bits[EPT];
      if constexpr (NW <= 32) {                             // a < 4 NW 255^2 < 2^23: fp32 reduction
        const float mf = (float)mcv.x, rcp = __uint_as_float(mcv.z), hm = __uint_as_float(mcv.w);
        if (mcv.x & 1u) {
          // odd m: a <= 4 NW 255 250 < 0.973 2^23, so |a rcp - a/m| <=
          // a 2^-24 (1 + 2^-29) / m < 1/(2m), while a/m is at least 1/(2m)
          // from every half-integer: the rounded quotient is exact and
          // r = s a - q m is the centered residue, with no correction step
          // (an exact zero is +0: x - x and +0 - 0 m round to +0)
#pragma unroll
          for (int e = 0; e < EPT; ++e) {
            const float f = fmaf(sg[e], __uint_as_float(a[e] | 0x4B000000u), sb[e]);
            const float q = fmaf(f, rcp, 12582912.0f) - 12582912.0f;
            bits[e] = __float_as_uint(fmaf(-q, mf, f));
          }
        } else {                                            // m = 128: ties need the correction
#pragma unroll
          for (int e = 0; e < EPT; ++e) bits[e] = __float_as_uint(centered_f32(a[e], ng[e], mf, rcp, hm));
        }
      } else {
#pragma unroll
        for (int e = 0; e < EPT; ++e) bits[e] = bf16_bits(centered(barrett32(a[e], mcv.x, mcv.y), mcv.x, ng[e])) << 16;
      }
      put(bits);                                            // plane l
    } else {
      // low and high table bytes: x = s_lo + 256 s_hi < 2^32
      uint32_t lo[EPT], hi[EPT];
#pragma unroll
      for (int e = 0; e < EPT; ++e) lo[e] = hi[e] = 0u;
      const uint2* th = tl + W32 / 2;
#pragma unroll
      for (int q = 0; q < NW / 2; ++q) {
        const uint2 t2 = tl[q];
        const uint2 u2 = th[q];
#pragma unroll
        for (int e = 0; e < EPT; ++e) {
          lo[e] = __dp4a(w[e][2 * q], t2.x, lo[e]);
          lo[e] = __dp4a(w[e][2 * q + 1], t2.y, lo[e]);
          hi[e] = __dp4a(w[e][2 * q], u2.x, hi[e]);
          hi[e] = __dp4a(w[e][2 * q + 1], u2.y, hi[e]);
        }
      }
      if (NW & 1) {
        const uint32_t tx = tw[NW - 1], ux = tw[W32 + NW - 1];
#pragma unroll
        for (int e = 0; e < EPT; ++e) {
          lo[e] = __dp4a(w[e][NW - 1], tx, lo[e]);
          hi[e] = __dp4a(w[e][NW - 1], ux, hi[e]);
        }
      }
      // balanced base-128 split: r = r0 + 128 r1 with r0 = cen(r mod 128);
      // planes L1 + 3 (l - L1) + {0, 1, 2} = r0, r1, r0 + r1
      uint32_t b0[EPT], b1[EPT], b2[EPT];
      if constexpr (NW <= 32) {
        // fp32, exact (m odd): lo <= 4 NW 255^2 and hi < lo are below
        // 2^23 / (1 + 2^-29), so their rounded quotients are exact and give
        // centered residues; y = r_lo + 256 r_hi has |y| < 2^21, reduced
        // exactly the same way; then the split with a round-to-nearest
        // quotient by 128 (a tie leaves r0 = -64, moved to +64)
        // Up to 24 words lo <= 24 4 255^2 and 256 |r_hi| <= 256 8095 keep
        // y = s lo + 256 r_hi below 2^23 / (1 + 2^-29): lo needs no reduction
        // of its own.
        const float mf = (float)mcv.x, rcp = __uint_as_float(mcv.z);
#pragma unroll
        for (int e = 0; e < EPT; ++e) {
          const float fl = fmaf(sg[e], __uint_as_float(lo[e] | 0x4B000000u), sb[e]);
          const float fh = fmaf(sg[e], __uint_as_float(hi[e] | 0x4B000000u), sb[e]);
          const float qh = fmaf(fh, rcp, 12582912.0f) - 12582912.0f;
          float yl = fl;
          if constexpr (NW > 24) {
            const float ql = fmaf(fl, rcp, 12582912.0f) - 12582912.0f;
            yl = fmaf(-ql, mf, fl);
          }
          const float y = fmaf(256.f, fmaf(-qh, mf, fh), yl);
          const float q = fmaf(y, rcp, 12582912.0f) - 12582912.0f;
          const float x = fmaf(-q, mf, y);
          float r1 = fmaf(x, 0.0078125f, 12582912.0f) - 12582912.0f;
          float r0 = fmaf(-128.f, r1, x);
          if (r0 <= -64.f) { r0 += 128.f; r1 -= 1.f; }
          b0[e] = __float_as_uint(r0);
          b1[e] = __float_as_uint(r1);
          b2[e] = __float_as_uint(r0 + r1);
        }
      } else {
#pragma unroll
        for (int e = 0; e < EPT; ++e) {
          const int x = centered(barrett32(lo[e] + (hi[e] << 8), mcv.x, mcv.y), mcv.x, ng[e]);
          const int y = x & 127;
          const int r0 = y > 64 ? y - 128 : y;
          const int r1 = (x - r0) >> 7;
          b0[e] = bf16_bits(r0) << 16;
          b1[e] = bf16_bits(r1) << 16;
          b2[e] = bf16_bits(r0 + r1) << 16;
        }
      }
      put(b0);
      put(b1);
      put(b2);
    }
  }
}

// EPT horizontally adjacent elements per thread (k .. k + EPT - 1).  The
// residue of |a_hat| mod m is sum_b beta_b (2^(8 b) mod m) over its bytes
// beta_b (Sec. 5.3's digit table, at byte granularity): one dp4a multiplies
// four bytes of a word by four packed table bytes and accumulates in 32 bits.
// Two-limb moduli use two byte tables (the low and high byte of
// 2^(8 b) mod m < 2^14).  The table is read once for all EPT elements, and
// each plane gets one vector store.  Block: 32 x 8 threads = 32 EPT columns x
// 8 rows of elements.
template <int W16>
__global__ void __launch_bounds__(256) k_residue(DevTables T, const int4* __restrict__ blk) {
  constexpr int W32 = W16 / 2;
  constexpr int EPT = residue_ept(W32);
  constexpr int RS = 2 * W32;                          // table row stride (words)
  extern __shared__ __align__(16) uint32_t s_t8[];     // [L][RS] packed bytes, then [L] x {m, mu, 1/m, m/2}
  const int4 b = blk[blockIdx.x];
  const ProbDev& P = T.probs[b.x];
  const int side = b.y;
  const int L = P.L, L1 = P.L1;
  uint4* s_mc = reinterpret_cast<uint4*>(s_t8 + L * RS);
  for (int i = threadIdx.y * 32 + threadIdx.x; i < L * RS; i += 256) {
    const int l = i / RS, d = i - l * RS;         // low bytes [0, W32), high bytes [W32, 2 W32)
    const int src = d < W32 ? d : (T.w16max >> 1) + (d - W32);
    s_t8[i] = T.t16[(int64_t)l * T.w16max + src];
  }
  for (int l = threadIdx.y * 32 + threadIdx.x; l < L; l += 256) {
    const ModConst mc = T.mods[l];
    s_mc[l] = make_uint4(mc.m, mc.mu, __float_as_uint(mc.rcp), __float_as_uint(0.5f * (float)mc.m));
  }
  __syncthreads();
  const int R = side ? P.N : P.M;
  const int r = b.z + threadIdx.y;
  const int k = b.w + EPT * threadIdx.x;
  if (r >= R || k >= P.K) return;
  const int nk = min(EPT, P.K - k);

  const uint64_t* limbs = side ? P.b_limbs : P.a_limbs;
  const int64_t ps = side ? P.b_ps : P.a_ps;
  const int64_t stride_k = side ? P.b_ld : 1;
  const int64_t off0 = side ? ((int64_t)k * P.b_ld + r) : ((int64_t)r * P.a_ld + k);
  const int32_t* exps = side ? P.b_exp : P.a_exp;
  const int8_t* signs = side ? P.b_sign : P.a_sign;
  const int nl = P.nl;
  const int e_line = side ? P.f[r] : P.e[r];

  uint32_t w[EPT][W32];
  bool ng[EPT];
#pragma unroll
  for (int e = 0; e < EPT; ++e) {
    const int64_t off = off0 + e * stride_k;
    ng[e] = false;
    if (e < nk && __ldg(limbs + (int64_t)(nl - 1) * ps + off) != 0ull) {
      element_words<W32>(limbs, ps, off, nl, __ldg(exps + off), e_line, P.t, w[e]);
      ng[e] = __ldg(signs + off) != 0;
    } else {
#pragma unroll
      for (int q = 0; q < W32; ++q) w[e][q] = 0u;
    }
  }

  uint16_t* planes = side ? P.pb : P.pa;
  const int64_t plane_stride = (int64_t)R * P.Kp;
  uint16_t* dst = planes + (int64_t)r * P.Kp + k;      // k a multiple of EPT, Kp of 8: aligned vectors
  // |a_hat| <= 2^t has ceil(W16 / 2) nonzero words; the class may hold one more
  if ((P.W16 + 1) / 2 <= W32 - 1)
    residue_planes<W32 - 1, W32, EPT>(w, ng, s_t8, s_mc, L, L1, dst, plane_stride, nk);
  else
    residue_planes<W32, W32, EPT>(w, ng, s_t8, s_mc, L, L1, dst, plane_stride, nk);
}

// ---------------------------------------------------------------------------
// Residues on the tensor cores.  With the bytes beta_b of |a_hat| (with the
// rounding increment) and the centered table T[j][b] = cen(2^(8 b) mod m_l)
// (one-limb moduli; |T| <= 127) or its balanced base-128 halves
// (two-limb moduli: T = T0 + 128 T1, |T0| <= 64, |T1| <= 63),
//   Y[e][j] = sum_b beta_b T[j][b]   ==  |a_hat| (mod m_l)  (or its halves),
// one GEMM per tile of 128 elements with K = bytes of a (t+1)-bit integer.
// Products are below 2^15 and sums below 2^15 * K < 2^24 for K < 512 bytes,
// so f16 operands (bytes and table entries are integers below 2^11) and the
// fp32 TMEM accumulator are exact; f16 rather than bf16 because a byte
// becomes an f16 with one byte permute and one packed subtraction per two.
// The epilogue
// reduces each column mod m (fp32 reciprocal + fma, exact), applies the sign,
// centers, splits two-limb residues and writes the bf16 planes.
//
// Persistent CTAs, 8 warps, every warp in every phase: warps 0-3 build the
// bytes of tile k (one element per thread), thread 0 issues its MMA into TMEM
// slot k & 1, then all warps run the epilogue of tile k - 1 (the two warps of
// a TMEM lane quadrant take the two halves of the columns).
// Tile: 4 lines x 32 consecutive k (lines = rows of A or columns of B); entry
// {problem, side, first line, first k}, tiles of one problem contiguous.
// ---------------------------------------------------------------------------
constexpr int kRtThreads = 256;

struct RtLayout {
  uint32_t b_bytes, a_region, small_off, total;
  __host__ __device__ RtLayout(int kpad, int npad, int lmax) {
    b_bytes = (uint32_t)npad * kpad * 2;
    a_region = ((uint32_t)128 * kpad * 2 + 1023u) & ~1023u;
    small_off = b_bytes + 2 * a_region;
    // small: s_mc [lmax] float4 {m, 1/m, kind, 0}, s_neg [2][128] u8, 4 barriers, tmem slot
    total = 1024 + small_off + (uint32_t)lmax * 16 + 256 + 4 * 8 + 16;
  }
};

__host__ __device__ inline int rt_tmem_cols(int npad) {
  int c = 32;
  while (c < npad) c <<= 1;
  return c;
}

// fp32 exact integer y (|y| < 2^24) -> y mod m in [0, m), as a float
__device__ __forceinline__ float fmodf_exact(float y, float mf, float rcp) {
  const float q = rintf(y * rcp);
  float r = fmaf(-q, mf, y);
  return r < 0.f ? r + mf : r;
}

__global__ void __launch_bounds__(kRtThreads, 2)
    k_residue_tc(const __grid_constant__ DevTables T, const int4* __restrict__ tiles, int ntiles, int kpad_max,
                 int npad_max, int lmax) {
  using namespace tc;
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  uint8_t* sm = smem_raw + (base - raw);
  const RtLayout lay(kpad_max, npad_max, lmax);
  const uint32_t sB = base;
  const uint32_t sA0 = base + lay.b_bytes;
  uint8_t* small = sm + lay.small_off;
  float4* s_mc = reinterpret_cast<float4*>(small);                       // [lmax]
  uint8_t* s_neg = small + lmax * 16;                                    // [2][128]: 1 negative, 2 zero
  uint64_t* bars = reinterpret_cast<uint64_t*>(s_neg + 256);
  uint64_t* b_bar = bars;
  uint64_t* m_bar = bars + 1;        // [2]
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 3);

  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const int tcols = rt_tmem_cols(npad_max);
  if (t == 0) {
    for (int i = 0; i < 3; ++i) mbar_init(bars + i, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(2 * tcols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  volatile int abort_flag = 0;
  uint32_t bcnt = 0, mcnt[2] = {0, 0};
  bool ok = true;

  auto epilogue = [&](int4 tp, int s) {
    const ProbDev& P = T.probs[tp.x];
    if (ok) ok = mbar_wait(m_bar + s, mcnt[s] & 1u, &abort_flag, T.status, T.spin_limit);
    ++mcnt[s];
    ok = __syncthreads_and(ok);
    tc_fence_after();
    const int quad = warp & 3, hh = warp >> 2;
    const int er = quad * 32 + lane;                  // TMEM lane = element of the tile
    const int side = tp.y;
    const int R = side ? P.N : P.M;
    const int line = tp.z + quad, k = tp.w + lane;
    const int L1 = P.L1, L = P.L;
    const int ncols = L1 + 2 * (L - L1);
    const int cmid = ((ncols + 63) / 64) * 32;        // never splits a two-limb column pair
    const int c0 = hh * cmid, c1 = min(ncols, c0 + cmid);
    const bool valid = ok && line < R && k < P.K;
    const uint8_t fl = s_neg[s * 128 + er];
    const bool neg = (fl & 1) != 0;
    uint16_t* planes = side ? P.pb : P.pa;
    const int64_t pstride = (int64_t)R * P.Kp;
    uint16_t* dst = planes + (int64_t)line * P.Kp + k;
    const uint32_t trow = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(s * tcols);
    auto centered_bits = [&](float rf, float mf) -> float {
      float x = (2.f * rf > mf) ? rf - mf : rf;      // (-m/2, m/2] of |a_hat| mod m
      if (neg && x != 0.f) x = -x;                   // no -0: planes as the CUDA-core kernel
      if (2.f * x == -mf) x = -x;                    // tie of the even modulus stays +m/2
      return x;
    };
    if (ok) {
      for (int c = c0; c < c1; c += 32) {
        uint32_t v[32];
        tmem_ld32(trow + (uint32_t)c, v);
        if (!valid) continue;
#pragma unroll
        for (int q = 0; q < 32; ++q) {
          const int col = c + q;
          if (col < c1) {
            if (col < L1) {
              const float4 mc = s_mc[col];
              const float x = centered_bits(fmodf_exact(__uint_as_float(v[q]), mc.x, mc.y), mc.x);
              dst[(int64_t)col * pstride] = (uint16_t)(__float_as_uint(x) >> 16);
            } else if (((col - L1) & 1) == 0 && q + 1 < 32) {
              const int l = L1 + ((col - L1) >> 1);
              const float4 mc = s_mc[l];
              const float r0 = fmodf_exact(__uint_as_float(v[q]), mc.x, mc.y);
              const float r1 = fmodf_exact(__uint_as_float(v[q + 1]), mc.x, mc.y);
              const float x = centered_bits(fmodf_exact(fmaf(128.f, r1, r0), mc.x, mc.y), mc.x);
              const int xi = (int)x;
              const int y0 = xi & 127;
              const int lo = y0 > 64 ? y0 - 128 : y0;  // cen(r mod 128)
              const int hi = (xi - lo) >> 7;
              const int64_t g = L1 + 3 * (l - L1);
              dst[g * pstride] = (uint16_t)(__float_as_uint((float)lo) >> 16);
              dst[(g + 1) * pstride] = (uint16_t)(__float_as_uint((float)hi) >> 16);
              dst[(g + 2) * pstride] = (uint16_t)(__float_as_uint((float)(lo + hi)) >> 16);
            }
          }
        }
      }
    }
    tc_fence_before();
    __syncthreads();
  };

  int cur = -1;
  int k = 0;
  bool pending = false;
  int4 prev = make_int4(0, 0, 0, 0);
  for (int i = blockIdx.x;; i += gridDim.x) {
    const bool have = i < ntiles;
    const int4 tl = have ? tiles[i] : make_int4(-1, 0, 0, 0);
    if (!have || tl.x != cur) {
      if (pending) {
        epilogue(prev, (k - 1) & 1);
        pending = false;
      }
      if (!have || !ok) break;
      const ProbDev& P = T.probs[tl.x];
      for (int l = t; l < P.L; l += kRtThreads) {
        const ModConst& mc = T.mods[l];
        s_mc[l] = make_float4((float)mc.m, mc.rcp, 0.f, 0.f);
      }
      __syncthreads();
      if (t == 0) {
        const int kb = P.res_kpad / 64;
        const uint32_t tb = (uint32_t)P.res_npad * 128;
        mbar_expect_tx(b_bar, tb * kb);
        for (int q = 0; q < kb; ++q)
          tma_load_2d(sB + q * tb, T.tmaps + 4 * T.count + tl.x, smem_u32(b_bar), q * 64, 0);
      }
      ok = mbar_wait(b_bar, bcnt & 1u, &abort_flag, T.status, T.spin_limit);
      ok = __syncthreads_and(ok);
      ++bcnt;
      cur = tl.x;
      if (!ok) break;
    }
    const ProbDev& P = T.probs[tl.x];
    const int b = k & 1;
    // ---- bytes of |a_hat| for the 128 elements of this tile (warps 0-3)
    if (t < 128) {
      const int side = tl.y;
      const int R = side ? P.N : P.M;
      const int line = tl.z + (t >> 5), kk = tl.w + (t & 31);
      uint8_t* gA = sm + lay.b_bytes + b * lay.a_region;
      const int nw = P.res_kpad >> 2;                  // 32-bit words covering the K positions
      uint8_t flag = 2;
      uint32_t carry = 0;
      int ws = 0, bs = 0, nl = P.nl;
      const uint32_t* limbs32 = nullptr;
      int64_t ps = 0, off = 0;
      bool nz = false;
      if (line < R && kk < P.K) {
        const uint64_t* limbs = side ? P.b_limbs : P.a_limbs;
        ps = side ? P.b_ps : P.a_ps;
        off = side ? ((int64_t)kk * P.b_ld + line) : ((int64_t)line * P.a_ld + kk);
        nz = __ldg(limbs + (int64_t)(nl - 1) * ps + off) != 0ull;
        if (nz) {
          const int e_line = side ? P.f[line] : P.e[line];
          const int ex = __ldg((side ? P.b_exp : P.a_exp) + off);
          const int sh = ex - e_line + P.t - 64 * nl;
          const int Bb = 64 - sh;                      // bit of sig * 2^64 that is bit 0 of the magnitude
          limbs32 = reinterpret_cast<const uint32_t*>(limbs);
          if (Bb - 1 >= 64 * nl + 64) {
            nz = false;                                // rounds to zero
          } else {
            ws = Bb >> 5;
            bs = Bb & 31;
            const int rbpos = Bb - 1;
            const uint32_t rw = sig_word(limbs32, ps, off, nl, (rbpos >> 5) - 2);
            const uint32_t rb = (rw >> (rbpos & 31)) & 1u;
            uint32_t sticky = rw & ((1u << (rbpos & 31)) - 1u);
            for (int j = (rbpos >> 5) - 3; j >= 0 && !sticky; --j) sticky |= sig_word(limbs32, ps, off, nl, j);
            const uint32_t w0 = __funnelshift_r(sig_word(limbs32, ps, off, nl, ws - 2),
                                                sig_word(limbs32, ps, off, nl, ws - 1), bs);
            carry = rb & ((sticky != 0u) | (w0 & 1u));
            flag = __ldg((side ? P.b_sign : P.a_sign) + off) ? 1 : 0;
          }
        }
      }
      for (int w = 0; w < nw; ++w) {
        uint32_t x = 0u;
        if (nz) {
          const uint64_t y = (uint64_t)__funnelshift_r(sig_word(limbs32, ps, off, nl, ws + w - 2),
                                                       sig_word(limbs32, ps, off, nl, ws + w - 1), bs) + carry;
          x = (uint32_t)y;
          carry = (uint32_t)(y >> 32);
        }
        *reinterpret_cast<uint32_t*>(gA + tc::sw128_offset(t, 4 * w, 128)) = f16_byte_pair(x, 0x5140u);
        *reinterpret_cast<uint32_t*>(gA + tc::sw128_offset(t, 4 * w + 2, 128)) = f16_byte_pair(x, 0x7362u);
      }
      s_neg[b * 128 + t] = nz ? flag : 2;
    }
    fence_proxy_async_smem();
    __syncthreads();
    if (t == 0) {
      tc_fence_after();
      const uint32_t idesc = idesc_f16(128, P.res_npad);      // f16 bytes and f16 table
      const uint32_t tb = (uint32_t)P.res_npad * 128;
      const uint32_t d = tmem + (uint32_t)(b * tcols);
      for (int q = 0; q < P.res_kpad / 64; ++q) {
        const uint64_t da = desc_sw128(sA0 + b * lay.a_region + q * 128 * 128);
        const uint64_t db = desc_sw128(sB + q * tb);
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) umma_bf16(d, da + 2 * kk, db + 2 * kk, idesc, (q | kk) ? 1u : 0u);
      }
      umma_commit(m_bar + b);
    }
    if (pending) epilogue(prev, (k - 1) & 1);
    pending = true;
    prev = tl;
    ++k;
  }
  if (pending && ok) epilogue(prev, (k - 1) & 1);
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * tcols) : "memory");
  }
}

// ---------------------------------------------------------------------------
// Residues on the tensor cores, warp-specialised (res_mode 2).  The same byte
// GEMM as k_residue_tc: with the bytes beta_b of |a_hat| (rounding increment
// included) and the centered table T[c][b] = cen(2^(8 b) mod m_l) (one-limb
// column c = l) or its balanced base-128 halves (two-limb modulus l: columns
// L1 + 2 (l - L1) + {0, 1}),
//   Y[e][c] = sum_b beta_b T[c][b]  ==  |a_hat| (mod m_l)  (or its halves),
// exact in fp32: |beta T| <= 255 * 127 < 2^15 and at most 512 bytes keep
// every sum below 2^24.  Per tile of 4 lines x 32 consecutive k (128
// elements; TMEM lane e is line e / 32, k e % 32: 32-byte runs on both sides
// for the limb reads and the plane writes) the bytes live in tensor memory as
// the A operand (two f16 bytes per 32-bit column, two or four buffers), the table
// streams through a shared-memory ring as B in blocks of 64 bytes x cw
// columns, and Y runs in chunks of cw columns through two accumulator slots:
//   [A0 .. A(nabuf-1): kpad/2 each][slot 0: cw][slot 1: cw]  <= 512 TMEM columns
// with nabuf = 2 or 4 byte buffers (uniform within a launch).
//   warp 0      TMA producer of the table blocks
//   warp 1      MMA issuer: tile t reads A buffer t mod nabuf; chunk c into
//               slot c & 1; commits per ring stage, per chunk and per tile
//   warps 2-9   two builder groups of one warp per TMEM lane quadrant, group
//               t & 1 for tile t: integerize the tile's elements and write
//               their bytes into A buffer t mod nabuf once the MMAs of tile
//               t - nabuf are done, so that two tiles are built at once
//   warps 10-21 three per lane quadrant (sub-groups s = 0..2): the tile's
//               32-column groups in turn (rotated per tile); a group is all
//               one-limb, all two-limb pairs (L1 is even) or the one mixed
//               group: reduce mod m_l (round-to-nearest quotient in fp32, the
//               sign applied first), split two-limb residues, store the bf16
//               planes through incremental plane pointers.
// Tile list entry: {problem, side, first line, first k}.
// ---------------------------------------------------------------------------
constexpr int kRmBuilders = 256;                  // two groups of four warps
constexpr int kRmEpi = 384;                       // three warps per lane quadrant
constexpr int kRmThreads = 64 + kRmBuilders + kRmEpi;
constexpr int kRmMaxStages = 16;

struct RmLayout {
  uint32_t mc_off, bar_off, total;
  __host__ __device__ RmLayout(uint32_t stage_bytes, int stages, int lmax) {
    mc_off = (uint32_t)stages * stage_bytes;                 // {m, 1/m, m/2, 0} as floats [lmax]
    bar_off = mc_off + (uint32_t)lmax * 16;
    // barriers: full, empty [kRmMaxStages], acc_full, acc_free [2], a_full, a_free [4],
    // drain; then the abort flag and the TMEM slot
    total = 1024 + bar_off + (2 * kRmMaxStages + 13) * 8 + 16;
    if (total < 116u * 1024u) total = 116u * 1024u;          // one CTA per SM: all 512 TMEM columns
  }
};

// The four bytes b_i of x times the element's sign s as f16 pairs
// {s b0, s b1}, {s b2, s b3} (low half first): the byte permute makes the
// pair {1024 + b0, 1024 + b1} (each byte under the f16 exponent bits of 2^10,
// where the mantissa's unit is 1), and one packed fma with s2 = {s, s} and
// c2 = {-1024 s, -1024 s} leaves s b_i exactly (every value involved is an
// integer below 2^11; +0 for b_i = 0).
__device__ __forceinline__ void signed_f16_bytes(uint32_t x, uint32_t s2, uint32_t c2, uint32_t& c01, uint32_t& c23) {
  asm("fma.rn.f16x2 %0, %1, %2, %3;" : "=r"(c01) : "r"(__byte_perm(x, 0x64646464u, 0x5140)), "r"(s2), "r"(c2));
  asm("fma.rn.f16x2 %0, %1, %2, %3;" : "=r"(c23) : "r"(__byte_perm(x, 0x64646464u, 0x7362)), "r"(s2), "r"(c2));
}

// Centered residue of an exact fp32 integer y (|y| < 2^24): y - q m with q the
// round-to-nearest of y / m (the 1.5 2^23 addend rounds; q may be off by one
// because 1/m is rounded), then one step each way into (-m/2, m/2]; exact.
__device__ __forceinline__ float cmod_f32(float y, float mf, float rcp, float hm) {
  const float q = fmaf(y, rcp, 12582912.0f) - 12582912.0f;
  float r = fmaf(-q, mf, y);
  r = r > hm ? r - mf : r;
  r = r <= -hm ? r + mf : r;
  return r;
}

// Centered residue of y0 + 128 y1 (mod m) for the two byte sums of a
// two-limb modulus: m is an odd prime below 2^14, the table halves satisfy
// |T0| <= 64 and |T1| <= 63, and an integer has at most 265 bytes (t <=
// 2112), so |y0|, |y1| <= 265 255 64 < 2^23.
// For an exact fp32 integer |y| < 2^23 and rcp = RN(1/m): |y rcp - y/m| <=
// |y|/m 2^-24 < 1/(2m), while an odd m keeps y/m at least 1/(2m) away from
// every half-integer, so q = RN(y rcp) (one fma with the 1.5 2^23 addend) is
// the nearest integer to y/m and y - q m is the centered residue in
// [-(m - 1)/2, (m - 1)/2], with no correction step.  That gives r1 for y1,
// then x = y0 + 128 r1 (|x| < 4.4e6 + 1.1e6 < 2^23, exact) and r for x.
// The + 0.0f turns a -0 (all bytes of a zero element carry the sign) into +0.
__device__ __forceinline__ float cmod2_f32(uint32_t y0bits, uint32_t y1bits, float mf, float rcp) {
  const float y1 = __uint_as_float(y1bits);
  const float q1 = fmaf(y1, rcp, 12582912.0f) - 12582912.0f;
  const float x = fmaf(128.f, fmaf(-q1, mf, y1), __uint_as_float(y0bits));
  const float q = fmaf(x, rcp, 12582912.0f) - 12582912.0f;
  return fmaf(-q, mf, x) + 0.0f;
}

// Balanced base-128 split of an integer |r| < 2^13: r = lo + 128 hi with lo
// in (-64, 64].  hi = RN((r - 0.5) / 128): r - 0.5 and its scaling are exact,
// (r - 0.5) / 128 is never a half-integer, and |r - 0.5 - 128 hi| < 64 gives
// lo = r - 128 hi in [-63, 64].
__device__ __forceinline__ void split128(float r, float& lo, float& hi) {
  hi = fmaf(r - 0.5f, 0.0078125f, 12582912.0f) - 12582912.0f;
  lo = fmaf(-128.f, hi, r);
}

__global__ void __launch_bounds__(kRmThreads, 1)
    k_residue_mm(const __grid_constant__ DevTables T, const int4* __restrict__ tiles, int ntiles,
                 uint32_t stage_bytes, int stages) {
  using namespace tc;
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  uint8_t* sm = smem_raw + (base - raw);
  const RmLayout lay(stage_bytes, stages, T.lmax);
  const uint32_t sRing = base;                                // table ring [stages][cw rows][128 B]
  const float4* s_mc = reinterpret_cast<const float4*>(sm + lay.mc_off);
  uint64_t* bars = reinterpret_cast<uint64_t*>(sm + lay.bar_off);
  uint64_t* full = bars;                                      // [kRmMaxStages]
  uint64_t* empty = bars + kRmMaxStages;                      // [kRmMaxStages]
  uint64_t* acc_full = bars + 2 * kRmMaxStages;               // [2]
  uint64_t* acc_free = acc_full + 2;                          // [2] (kRmEpi arrivals)
  uint64_t* a_full = acc_full + 4;                            // [4] (one builder group's arrivals)
  uint64_t* a_free = acc_full + 8;                            // [4] MMAs of the buffer's tile done
  uint64_t* drain = acc_full + 12;
  volatile int* abort_flag = reinterpret_cast<volatile int*>(acc_full + 13);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(acc_full + 13) + 1;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  {
    float4* w_mc = reinterpret_cast<float4*>(sm + lay.mc_off);
    for (int l = threadIdx.x; l < T.lmax; l += kRmThreads) {
      const float mf = (float)__ldg(&T.mods[l].m);
      w_mc[l] = make_float4(mf, __ldg(&T.mods[l].rcp), 0.5f * mf, 0.f);
    }
  }
  if (threadIdx.x == 0) {
    for (int i = 0; i < kRmMaxStages; ++i) {
      mbar_init(full + i, 1);
      mbar_init(empty + i, 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(acc_full + i, 1);
      mbar_init(acc_free + i, kRmEpi);
    }
    for (int i = 0; i < 4; ++i) {
      mbar_init(a_full + i, kRmBuilders / 2);
      mbar_init(a_free + i, 1);
    }
    mbar_init(drain, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(smem_u32(tmem_slot))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    // ------------------------------------------------------------ table producer
    if (lane == 0) {
      int st = 0;
      uint32_t ph = 0;
      int issued_phase[kRmMaxStages];
      for (int i = 0; i < kRmMaxStages; ++i) issued_phase[i] = -1;
      bool ok = true;
      for (int i = blockIdx.x; ok && i < ntiles; i += gridDim.x) {
        const int4 tl = tiles[i];
        const ProbDev& P = T.probs[tl.x];
        const CUtensorMap* mt = T.tmaps + 4 * T.count + tl.x;
        const int nkb = P.res_kpad / 64, cw = P.res_cw, nchunk = P.res_nchunk;
        for (int c = 0; ok && c < nchunk; ++c) {
          for (int q = 0; q < nkb; ++q) {
            if (!mbar_wait(empty + st, ph ^ 1u, abort_flag, T.status, T.spin_limit)) { ok = false; break; }
            mbar_expect_tx(full + st, (uint32_t)cw * 128u);
            tma_load_2d(sRing + st * stage_bytes, mt, smem_u32(full + st), q * 64, c * cw);
            issued_phase[st] = (int)ph;
            if (++st == stages) { st = 0; ph ^= 1u; }
          }
        }
      }
      if (!ok) {
        for (int i = 0; i < stages; ++i)
          if (issued_phase[i] >= 0)
            for (uint32_t t = 0; t < kSpinLimit && !mbar_try_wait(full + i, (uint32_t)issued_phase[i]); ++t) {}
      }
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      int st = 0;
      uint32_t ph = 0;
      int ck = 0, tcount = 0;
      bool ok = true, any = false;
      for (int i = blockIdx.x; ok && i < ntiles; i += gridDim.x, ++tcount) {
        const int4 tl = tiles[i];
        const ProbDev& P = T.probs[tl.x];
        const int nkb = P.res_kpad / 64, cw = P.res_cw, nchunk = P.res_nchunk, npad = P.res_npad;
        const uint32_t acols = (uint32_t)P.res_kpad / 2;
        const int nabuf = P.res_nabuf;
        const int ab = tcount % nabuf, ause = tcount / nabuf;
        if (!mbar_wait(a_full + ab, (uint32_t)(ause & 1), abort_flag, T.status, T.spin_limit)) { ok = false; break; }
        tc_fence_after();
        const uint32_t abase = tmem + (uint32_t)ab * acols;
        for (int c = 0; ok && c < nchunk; ++c, ++ck) {
          const int s = ck & 1, use = ck >> 1;
          if (use > 0 && !mbar_wait(acc_free + s, (uint32_t)((use - 1) & 1), abort_flag, T.status, T.spin_limit)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const int ncol = min(cw, npad - c * cw);             // a multiple of 16
          const uint32_t idesc = idesc_f16(128, ncol);             // f16 bytes and f16 table
          const uint32_t d = tmem + (uint32_t)nabuf * acols + (uint32_t)(s * cw);
          for (int q = 0; q < nkb; ++q) {
            if (!mbar_wait(full + st, ph, abort_flag, T.status, T.spin_limit)) { ok = false; break; }
            tc_fence_after();
            const uint64_t db = desc_sw128(sRing + st * stage_bytes);
#pragma unroll
            for (int kk = 0; kk < 4; ++kk)
              umma_bf16_ta(d, abase + (uint32_t)(32 * q + 8 * kk), db + 2 * kk, idesc, (q | kk) ? 1u : 0u);
            umma_commit(empty + st);
            any = true;
            if (++st == stages) { st = 0; ph ^= 1u; }
          }
          if (ok) umma_commit(acc_full + s);
        }
        if (!ok) break;
        umma_commit(a_free + ab);
      }
      if (!ok && any) {
        umma_commit(drain);
        for (uint32_t t = 0; t < kSpinLimit && !mbar_try_wait(drain, 0u); ++t) {}
      }
    }
  } else if (warp < 10) {
    // ------------------------------------------------------------ byte builders
    // Per element: S = sig 2^64 as 64-bit limbs S[j] (S[0] = 0, S[j] = limb
    // j - 1), |a_hat| = bits Bb.. of S plus the round-half-even increment.
    // Every limb read is unconditional at a clamped address (masked to zero
    // outside the significand), so the reads of a step are all in flight at
    // once: the exponents first, then one batch with the limbs of the first
    // 32 columns and the two below them (the round bit and the first sticky
    // limbs), before the wait for the buffer.  The element's sign goes onto the
    // f16 bytes (a zero byte stays +0; a sum can still be -0, which the
    // epilogue's + 0.0f turns into +0).  Group bg takes the tiles t with
    // t & 1 == bg.
    const int bg = (warp - 2) >> 2;
    const int quad = warp & 3;
    const int row = quad * 32 + lane;
    const uint32_t tlane = tmem + ((uint32_t)(quad * 32) << 16);
    bool ok = true;
    int tcount = 0;
    for (int i = blockIdx.x; i < ntiles; i += gridDim.x, ++tcount) {
      if ((tcount & 1) != bg) continue;
      const int4 tl = tiles[i];
      const ProbDev& P = T.probs[tl.x];
      const int nabuf = P.res_nabuf;
      const int ab = tcount % nabuf, ause = tcount / nabuf;
      const int side = tl.y;
      const int R = side ? P.N : P.M;
      const int line = tl.z + (row >> 5), k = tl.w + (row & 31);
      const bool valid = line < R && k < P.K;
      const uint32_t acols = (uint32_t)P.res_kpad / 2;
      const int nl = P.nl;
      const int64_t ps = side ? P.b_ps : P.a_ps;
      const int64_t off = valid ? (side ? ((int64_t)k * P.b_ld + line) : ((int64_t)line * P.a_ld + k)) : 0;
      const uint64_t* el = (side ? P.b_limbs : P.a_limbs) + off;
      auto S = [&](int j) -> uint64_t {            // limb j of sig 2^64, 0 outside
        const bool in = (unsigned)(j - 1) < (unsigned)nl;
        const uint64_t v = __ldg(el + (int64_t)(in ? j - 1 : 0) * ps);
        return in ? v : 0ull;
      };
      const uint64_t top = __ldg(el + (int64_t)(nl - 1) * ps);
      const int ex = __ldg((side ? P.b_exp : P.a_exp) + off);
      const int e_line = __ldg((side ? P.f : P.e) + (valid ? line : 0));
      const bool neg = __ldg((side ? P.b_sign : P.a_sign) + off) != 0;
      int Bb = 64 - (ex - e_line + P.t - 64 * nl);  // bit of S that is bit 0 of |a_hat|
      const bool nz = valid && top != 0ull && Bb - 1 < 64 * nl + 64;
      Bb = nz ? Bb : 64;
      const int ws = Bb >> 5, bs = Bb & 31, lq = ws >> 1;
      const bool odd = ws & 1;
      // limbs lq - 2 .. lq + 8: the round bit (bit Bb - 1, in limb lq or
      // lq - 1), the first sticky limbs and the first 32 columns' window
      uint64_t lm0[11];
#pragma unroll
      for (int q = 0; q < 11; ++q) lm0[q] = S(lq - 2 + q);
      const int rbpos = Bb - 1;
      const bool rb_hi = (rbpos >> 6) == lq;       // round bit in limb lq (else lq - 1)
      const uint64_t srb = rb_hi ? lm0[2] : lm0[1];
      const uint32_t rb = (uint32_t)(srb >> (rbpos & 63)) & 1u;
      uint64_t sticky = (srb & ((1ull << (rbpos & 63)) - 1ull)) | (rb_hi ? lm0[1] : 0ull) | lm0[0];
      for (int j = lq - 3; j >= 1 && !sticky; --j) sticky |= S(j);
      uint32_t carry = nz ? (rb & ((sticky != 0ull) | ((uint32_t)(lm0[2] >> (Bb & 63)) & 1u))) : 0u;
      const uint32_t s2 = neg ? 0xBC00BC00u : 0x3C003C00u;   // {s, s} in f16
      const uint32_t c2 = neg ? 0x64006400u : 0xE400E400u;   // {-1024 s, -1024 s}
      if (ause > 0 && ok) ok = mbar_wait(a_free + ab, (uint32_t)((ause - 1) & 1), abort_flag, T.status, T.spin_limit);
      ok = __all_sync(0xffffffffu, ok);
      if (!ok) break;
      tc_fence_after();
      const uint32_t abase = tlane + (uint32_t)ab * acols;
      for (uint32_t c0 = 0; c0 < acols; c0 += 32) {  // 16 words = 64 bytes = 32 columns
        // 32-bit words ws + 16 it .. ws + 16 it + 16 of S come from limbs lq + 8 it .. + 8
        uint64_t lm[9];
        if (c0 == 0) {
#pragma unroll
          for (int q = 0; q < 9; ++q) lm[q] = lm0[2 + q];
        } else {
          const int j0 = lq + (int)(c0 >> 2);
#pragma unroll
          for (int q = 0; q < 9; ++q) lm[q] = S(j0 + q);
        }
        auto word = [&](int x) -> uint32_t {        // word x of the window (x + odd of the limbs)
          const uint32_t a = (x & 1) ? (uint32_t)(lm[x >> 1] >> 32) : (uint32_t)lm[x >> 1];
          const uint32_t b = (x & 1) ? (uint32_t)lm[(x + 1) >> 1] : (uint32_t)(lm[x >> 1] >> 32);
          return odd ? b : a;
        };
        uint32_t col[32];
#pragma unroll
        for (int w = 0; w < 16; ++w) {
          const uint64_t y = (uint64_t)__funnelshift_r(word(w), word(w + 1), bs) + carry;
          const uint32_t x = nz ? (uint32_t)y : 0u;
          carry = (uint32_t)(y >> 32);
          signed_f16_bytes(x, s2, c2, col[2 * w], col[2 * w + 1]);
        }
        tmem_st32(abase + c0, col);
      }
      tmem_wait_st();
      tc_fence_before();
      mbar_arrive(a_full + ab);
    }
    if (!ok) *abort_flag = 1;
  } else {
    // ------------------------------------------------------------ epilogues
    const int ew = warp - 10;
    const int sub = ew >> 2;                          // column sub-group 0..2
    const int quad = warp & 3;
    const int row = quad * 32 + lane;
    const uint32_t tlane = tmem + ((uint32_t)(quad * 32) << 16);
    int ck = 0, tcount = 0;
    bool ok = true;
    for (int i = blockIdx.x; i < ntiles; i += gridDim.x, ++tcount) {
      const int4 tl = tiles[i];
      const ProbDev& P = T.probs[tl.x];
      const int side = tl.y;
      const int R = side ? P.N : P.M;
      const int line = tl.z + (row >> 5), k = tl.w + (row & 31);
      const bool valid = line < R && k < P.K;
      const uint32_t acols = (uint32_t)P.res_kpad / 2;
      const int L1 = P.L1, ncols = P.L1 + 2 * (P.L - P.L1), cw = P.res_cw;
      const int nchunk = P.res_nchunk, npad = P.res_npad, nabuf = P.res_nabuf;
      uint16_t* planes = side ? P.pb : P.pa;
      const int64_t pstride = (int64_t)R * P.Kp;
      uint16_t* dst0 = planes + (int64_t)(valid ? line : 0) * P.Kp + (valid ? k : 0);
      for (int c = 0; c < nchunk; ++c, ++ck) {
        const int s = ck & 1, use = ck >> 1;
        if (ok) ok = mbar_wait(acc_full + s, (uint32_t)(use & 1), abort_flag, T.status, T.spin_limit);
        ok = __all_sync(0xffffffffu, ok);
        if (!ok) break;
        tc_fence_after();
        const uint32_t trow = tlane + (uint32_t)nabuf * acols + (uint32_t)(s * cw);
        const int j0 = c * cw;
        const int ncolp = min(cw, npad - j0);          // columns written by the MMAs
        // the tile's 32-column groups go round the three sub-groups (rotated
        // per tile), whatever the chunk width
        const int gfirst = ((sub - c * (cw >> 5) - tcount) % 3 + 3) % 3;
        for (int g = 32 * gfirst; g < ncolp; g += 96) {
          // 16 columns per TMEM load, reduced as two pieces of 8 (a rolled
          // loop: the epilogue's code stays small next to the builders' in
          // the instruction cache); pieces hold whole pairs (L1 and every
          // piece start are even)
          const int gcols = min(32, ncolp - g);           // 32 or 16
#pragma unroll 1
          for (int pc2 = 0; pc2 < gcols; pc2 += 16) {
            uint32_t y16[16];
            tmem_ld16(trow + (uint32_t)(g + pc2), y16);
            if (!valid) continue;
#pragma unroll
            for (int hh = 0; hh < 2; ++hh) {
              const int pc = pc2 + 8 * hh;
              uint32_t y[8];
#pragma unroll
              for (int q = 0; q < 8; ++q) y[q] = y16[8 * hh + q];
              const int c0 = j0 + g + pc;
              if (c0 + 8 <= L1) {
                // 8 one-limb moduli: planes c0 .. c0 + 7
                uint16_t* dp = dst0 + (int64_t)c0 * pstride;
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                  const float4 mc = s_mc[c0 + q];
                  const float r = cmod_f32(__uint_as_float(y[q]), mc.x, mc.y, mc.z) + 0.0f;
                  *dp = (uint16_t)(__float_as_uint(r) >> 16);
                  dp += pstride;
                }
              } else if (c0 >= L1) {
                // 4 two-limb pairs: moduli l = L1 + (c0 - L1) / 2 + i, planes L1 + 3 (l - L1) + {0, 1, 2}
                const int lb = L1 + ((c0 - L1) >> 1);
                uint16_t* dp = dst0 + (int64_t)(L1 + 3 * (lb - L1)) * pstride;
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                  if (c0 + 2 * i < ncols) {
                    const float4 mc = s_mc[lb + i];
                    // x is +0 for a zero residue; then lo, hi and lo + hi are never -0
                    const float x = cmod2_f32(y[2 * i], y[2 * i + 1], mc.x, mc.y);
                    float lo, hi;
                    split128(x, lo, hi);
                    dp[0] = (uint16_t)(__float_as_uint(lo) >> 16);
                    dp[pstride] = (uint16_t)(__float_as_uint(hi) >> 16);
                    dp[2 * pstride] = (uint16_t)(__float_as_uint(lo + hi) >> 16);
                  }
                  dp += 3 * pstride;
                }
              } else {
                // the piece that holds the last one-limb moduli and the first pairs
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                  const int colx = c0 + q;
                  if (colx < L1) {
                    const float4 mc = s_mc[colx];
                    const float r = cmod_f32(__uint_as_float(y[q]), mc.x, mc.y, mc.z) + 0.0f;
                    dst0[(int64_t)colx * pstride] = (uint16_t)(__float_as_uint(r) >> 16);
                  } else if ((q & 1) == 0 && colx < ncols) {   // a pair starts at an even column
                    const int l = L1 + ((colx - L1) >> 1);
                    const float4 mc = s_mc[l];
                    const float x = cmod2_f32(y[q], y[q + 1], mc.x, mc.y);
                    float lo, hi;
                    split128(x, lo, hi);
                    uint16_t* dp = dst0 + (int64_t)(L1 + 3 * (l - L1)) * pstride;
                    dp[0] = (uint16_t)(__float_as_uint(lo) >> 16);
                    dp[pstride] = (uint16_t)(__float_as_uint(hi) >> 16);
                    dp[2 * pstride] = (uint16_t)(__float_as_uint(lo + hi) >> 16);
                  }
                }
              }
            }
          }
        }
        tc_fence_before();
        mbar_arrive(acc_free + s);
      }
      if (!ok) break;
    }
    if (!ok) *abort_flag = 1;
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem) : "memory");
  }
}

// Chunk width of the warp-specialised tensor-core residues: nabuf byte
// buffers (kpad / 2 columns each) and two accumulator slots of cw columns (a
// multiple of 32) within the 512 TMEM columns; four buffers (two tiles built
// at once, two in the MMAs) where that takes no more chunks than two.
void residue_mm_geometry(int kpad, int npad, int* cw_out, int* nabuf_out) {
  const int need = (npad + 31) & ~31;
  auto width = [&](int nab) {
    int cw = (512 - nab * (kpad / 2)) / 2;
    cw = cw > 256 ? 256 : cw;
    cw &= ~31;
    return cw < need ? cw : need;
  };
  const int cw2 = width(2), cw4 = width(4);
  if (cw4 >= 32 && (npad + cw4 - 1) / cw4 <= (npad + cw2 - 1) / cw2) {
    *cw_out = cw4;
    *nabuf_out = 4;
  } else {
    *cw_out = cw2;
    *nabuf_out = 2;
  }
}

int residue_mm_smem_bytes(int cw_max, int lmax, int /*tcols*/, int* stages) {
  const uint32_t sb = (uint32_t)cw_max * 128u;
  for (int st = kRmMaxStages; st >= 2; --st) {
    const int bytes = (int)RmLayout(sb, st, lmax).total;
    if (bytes <= 227 * 1024) {
      if (stages) *stages = st;
      return bytes;
    }
  }
  if (stages) *stages = 0;
  return -1;
}

cudaError_t launch_residues_mm(const DevTables& t, const int32_t* tiles, int ntiles, int cw_max, int /*tcols*/,
                               int sms, cudaStream_t s) {
  if (ntiles == 0) return cudaSuccess;
  int stages = 0;
  const int smem = residue_mm_smem_bytes(cw_max, t.lmax, 512, &stages);
  if (smem < 0) return cudaErrorInvalidValue;
  const int grid = std::min(ntiles, sms);
  k_residue_mm<<<grid, kRmThreads, smem, s>>>(t, reinterpret_cast<const int4*>(tiles), ntiles,
                                              (uint32_t)cw_max * 128u, stages);
  return cudaGetLastError();
}

int residue_tc_smem_bytes(int kpad, int npad, int lmax) { return (int)RtLayout(kpad, npad, lmax).total; }

cudaError_t launch_residues_tc(const DevTables& t, const int32_t* tiles, int ntiles, int kpad_max, int npad_max,
                               int lmax, int sms, cudaStream_t s) {
  if (ntiles == 0) return cudaSuccess;
  const int smem = residue_tc_smem_bytes(kpad_max, npad_max, lmax);
  // several persistent CTAs per SM hide each other's load latency; TMEM caps them
  int per_sm = 1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_residue_tc, kRtThreads, smem) != cudaSuccess)
    per_sm = 1;
  per_sm = std::max(1, std::min(per_sm, 512 / (2 * rt_tmem_cols(npad_max))));
  const int grid = std::min(ntiles, sms * per_sm);
  k_residue_tc<<<grid, kRtThreads, smem, s>>>(t, reinterpret_cast<const int4*>(tiles), ntiles, kpad_max, npad_max,
                                              lmax);
  return cudaGetLastError();
}

static const int kResidueW16[] = {8, 12, 20, 36, 68, 132};
static const int kNumResidueClasses = 6;

int residue_class_for(int w16) {
  for (int i = 0; i < kNumResidueClasses; ++i)
    if (w16 <= kResidueW16[i]) return i;
  return -1;
}
int residue_class_w16(int cls) { return kResidueW16[cls]; }
int residue_class_ept(int cls) { return residue_ept(kResidueW16[cls] / 2); }

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
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_residue_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_residue_mm, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
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
