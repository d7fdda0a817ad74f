// Stage 5 of the Ozaki-II flow (Sec. 4.1): direct CRT reconstruction
// (Sec. 4.4) and the final rescale and round-to-nearest-even to p bits.
//
// Warp-cooperative: a group of GL lanes owns one output element; its
// 32-bit digits are spread across the group (digit d lives in lane d % GL,
// row d / GL).  For each element
//   v_l   = u_l (M_l^{-1} mod m_l) mod m_l
//   alpha~= floor(sum_l v_l floor(2^32/m_l) / 2^32)        in {alpha-1, alpha}
//   R     = S - alpha~ P = sum_l v_l M_l + alpha~ (2^(32 D) - P)  mod 2^(32 D)
//   x0    = R - P if R >= P else R                          (R in [0, 2P))
//   c_hat = x0 if x0 <= floor(P/2) else x0 - P
// where alpha = floor(sum v_l / m_l) is the exact quotient S div P (Sec. 4.4).
// The paper evaluates alpha in binary64 and corrects with up to two
// subtractions; the fixed-point estimate above has error below
// L 2^14 / 2^32 < 1, so one conditional subtraction suffices and no FP64 is
// needed.  Every digit sum is carried exactly: each lane accumulates 64-bit
// column sums, the high halves move one digit up with a shuffle, and the
// remaining 0/1 carries are resolved for a whole row at once with a
// generate/propagate ballot and one integer addition (carry lookahead).
#include <climits>

#include "oz2_internal.h"

namespace oz2 {

namespace {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ uint32_t barrett32(uint32_t x, uint32_t m, uint32_t mu) {
  uint32_t q = __umulhi(x, mu);
  uint32_t r = x - q * m;
  return r >= m ? r - m : r;
}

template <int GL>
__device__ __forceinline__ uint32_t gmask() {
  return GL == 32 ? 0xffffffffu : ((1u << GL) - 1u);
}

// All DPL rows of lane `src` of this lane's group.
template <int GL, int DPL>
__device__ __forceinline__ void fetch_rows(const uint32_t (&dig)[DPL], int src, uint32_t (&out)[DPL]) {
#pragma unroll
  for (int r = 0; r < DPL; ++r) out[r] = __shfl_sync(kFull, dig[r], src, GL);
}

// Digit d (per lane, may differ across lanes) of the group's number; 0 when
// d is outside [0, GL*DPL).
template <int GL, int DPL>
__device__ __forceinline__ uint32_t fetch(const uint32_t (&dig)[DPL], int d) {
  const int src = ((d % GL) + GL) % GL;
  const int row = (d - src) / GL;
  uint32_t out = 0u;
#pragma unroll
  for (int r = 0; r < DPL; ++r) {
    const uint32_t t = __shfl_sync(kFull, dig[r], src, GL);
    if (r == row) out = t;
  }
  return out;
}

// Normalise 64-bit column sums (each < 2^63) into 32-bit digits plus `cin`
// at digit 0, modulo 2^(32 GL DPL).  Returns digit `dcut` of the result and
// clears digits >= dcut.  Must be called by all 32 lanes of the warp.
template <int GL, int DPL>
__device__ __forceinline__ uint32_t normalize(const uint64_t (&acc)[DPL], uint32_t (&dig)[DPL],
                                              uint32_t cin, int dcut, int lam, int gbase) {
  uint32_t rot[DPL];
#pragma unroll
  for (int i = 0; i < DPL; ++i)
    rot[i] = __shfl_sync(kFull, (uint32_t)(acc[i] >> 32), (lam + GL - 1) & (GL - 1), GL);
  uint32_t c = cin;
#pragma unroll
  for (int i = 0; i < DPL; ++i) {
    const uint32_t hin = (lam == 0) ? (i > 0 ? rot[i - 1] : 0u) : rot[i];
    const uint64_t x = (uint64_t)(uint32_t)acc[i] + hin;          // < 2^32 + 2^31
    const bool gen = (x >> 32) != 0;
    const bool prop = (uint32_t)x == 0xffffffffu;
    const uint32_t G = (__ballot_sync(kFull, gen) >> gbase) & gmask<GL>();
    const uint32_t Pm = (__ballot_sync(kFull, prop) >> gbase) & gmask<GL>();
    // internal carries of (G|P) + G + c are exactly the digit carries
    const uint64_t s = (uint64_t)(G | Pm) + (uint64_t)G + c;
    const uint32_t cm = ((uint32_t)s ^ Pm) & gmask<GL>();
    c = (uint32_t)(s >> GL) & 1u;
    dig[i] = (uint32_t)x + ((cm >> lam) & 1u);
  }
  const uint32_t top = fetch<GL, DPL>(dig, dcut);
#pragma unroll
  for (int i = 0; i < DPL; ++i)
    if (lam + GL * i >= dcut) dig[i] = 0u;
  return top;
}

template <int GL, int DPL>
__global__ void __launch_bounds__(256) k_crt(DevTables T, const int4* __restrict__ blk) {
  constexpr int EPB = 256 / GL;
  constexpr int DS = GL * DPL;
  extern __shared__ uint16_t s_v[];              // [L][EPB]
  const int4 b = blk[blockIdx.x];
  const ProbDev& P = T.probs[b.x];
  const int64_t MN = (int64_t)P.M * P.N;
  const int64_t e0 = (int64_t)b.y * EPB;
  const int L = P.L;
  const CrtView cv = crt_view(T.crt_pool, P);

  for (int i = threadIdx.x; i < L * EPB; i += 256) {
    const int l = i / EPB, e = i - l * EPB;
    const int64_t idx = e0 + e;
    const uint32_t uu = idx < MN ? (uint32_t)P.u[(int64_t)l * MN + idx] : 0u;
    const ModConst& mc = T.mods[l];
    s_v[i] = (uint16_t)barrett32(uu * __ldg(cv.Minv + l), mc.m, mc.mu);
  }
  __syncthreads();

  const int g = threadIdx.x / GL;
  const int lam = threadIdx.x - g * GL;
  const int gbase = (threadIdx.x & 31) - lam;
  const int64_t idx = e0 + g;
  const bool valid = idx < MN;
  const int D = P.D32;

  // quotient estimate
  uint64_t sig = 0;
  for (int l = lam; l < L; l += GL) sig += (uint64_t)s_v[l * EPB + g] * T.mods[l].mu;
#pragma unroll
  for (int o = GL / 2; o; o >>= 1) sig += __shfl_xor_sync(kFull, sig, o, GL);
  const uint32_t alpha = (uint32_t)(sig >> 32);

  uint64_t acc[DPL];
#pragma unroll
  for (int i = 0; i < DPL; ++i) acc[i] = (uint64_t)alpha * __ldg(cv.negP + lam + GL * i);
  for (int l = 0; l < L; ++l) {
    const uint32_t v = s_v[l * EPB + g];
    const uint32_t* md = cv.Mdig + (int64_t)l * DS + lam;
#pragma unroll
    for (int i = 0; i < DPL; ++i) acc[i] += (uint64_t)v * __ldg(md + GL * i);
  }
  uint32_t R[DPL], R2[DPL];
  normalize<GL, DPL>(acc, R, 0u, D, lam, gbase);

  // R in [0, 2P): subtract P once if R >= P
#pragma unroll
  for (int i = 0; i < DPL; ++i) acc[i] = (uint64_t)R[i] + __ldg(cv.negP + lam + GL * i);
  const uint32_t ge = normalize<GL, DPL>(acc, R2, 0u, D, lam, gbase);
#pragma unroll
  for (int i = 0; i < DPL; ++i) R[i] = ge ? R2[i] : R[i];
  // consistency check: x0 < P
#pragma unroll
  for (int i = 0; i < DPL; ++i) acc[i] = (uint64_t)R[i] + __ldg(cv.negP + lam + GL * i);
  const uint32_t bad = normalize<GL, DPL>(acc, R2, 0u, D, lam, gbase);
  if (bad && valid && lam == 0) atomicOr(T.status, kStatusCrtRange);
  // sign: x0 > floor(P/2)  <=>  x0 + 2^(32D) - (floor(P/2) + 1) carries out
#pragma unroll
  for (int i = 0; i < DPL; ++i) acc[i] = (uint64_t)R[i] + __ldg(cv.negH1 + lam + GL * i);
  const uint32_t neg = normalize<GL, DPL>(acc, R2, 0u, D, lam, gbase);
  // |c_hat| = P - x0 for negative results: P + ~x0 + 1 (mod 2^(32 D))
#pragma unroll
  for (int i = 0; i < DPL; ++i) {
    const int d = lam + GL * i;
    acc[i] = (uint64_t)__ldg(cv.P + d) + (d < D ? (uint64_t)(~R[i]) : 0ull);
  }
  normalize<GL, DPL>(acc, R2, 1u, D, lam, gbase);
  uint32_t mag[DPL];
#pragma unroll
  for (int i = 0; i < DPL; ++i) mag[i] = neg ? R2[i] : R[i];

  const int64_t row = valid ? idx / P.N : 0;
  const int64_t col = valid ? idx - row * P.N : 0;
  if (P.dbg_chat != nullptr && valid) {
    uint32_t* dst = P.dbg_chat + idx * (int64_t)(D + 1);
    if (lam == 0) dst[0] = neg;
#pragma unroll
    for (int i = 0; i < DPL; ++i) {
      const int d = lam + GL * i;
      if (d < D) dst[1 + d] = mag[i];
    }
  }

  // bit length n of |c_hat|
  int top = -1;
#pragma unroll
  for (int i = 0; i < DPL; ++i) {
    const uint32_t nz = (__ballot_sync(kFull, mag[i] != 0u) >> gbase) & gmask<GL>();
    if (nz) top = GL * i + 31 - __clz(nz);
  }
  const uint32_t tdig = fetch<GL, DPL>(mag, top);
  int n = top >= 0 ? 32 * top + 32 - __clz(tdig) : 0;

  // rounding: keep the top p bits, round-half-even on the dropped ones
  const int p = P.p, nl = P.nl;
  const int sh = n - p;
  const int rpos = sh - 1;
  const uint32_t wr = fetch<GL, DPL>(mag, rpos >= 0 ? (rpos >> 5) : -1);
  const uint32_t wl = fetch<GL, DPL>(mag, sh >= 0 ? (sh >> 5) : -1);
  const uint32_t rb = rpos >= 0 ? (wr >> (rpos & 31)) & 1u : 0u;
  const uint32_t lsb = sh >= 0 ? (wl >> (sh & 31)) & 1u : 0u;
  uint32_t st_local = 0u;
#pragma unroll
  for (int i = 0; i < DPL; ++i) {
    const int lo = 32 * (lam + GL * i);
    if (rpos >= lo + 32) st_local |= mag[i];
    else if (rpos > lo) st_local |= mag[i] & ((1u << (rpos - lo)) - 1u);
  }
  const uint32_t sticky = (__ballot_sync(kFull, st_local != 0u) >> gbase) & gmask<GL>();
  const uint32_t up = rb & ((sticky != 0u) | lsb);

  // output field F = floor(|c_hat| 2^(64 nl - n)) with the 64 nl - p low bits
  // cleared, as 2 nl 32-bit words spread like the digits
  const int base = n - 64 * nl;
  const int q0 = base >> 5;              // floor
  const int bs = base & 31;
  const int lowb = 64 * nl - p;
  uint32_t ta[DPL], tb[DPL];
  const int xa = lam + q0, xb = lam + q0 + 1;
  const int sa = ((xa % GL) + GL) % GL, sb = ((xb % GL) + GL) % GL;
  const int ra = (xa - sa) / GL, rb0 = (xb - sb) / GL;
  fetch_rows<GL, DPL>(mag, sa, ta);
  fetch_rows<GL, DPL>(mag, sb, tb);
#pragma unroll
  for (int i = 0; i < DPL; ++i) {
    const int w = lam + GL * i;
    uint32_t dlo = 0u, dhi = 0u;
#pragma unroll
    for (int r = 0; r < DPL; ++r) {
      if (r == ra + i) dlo = ta[r];
      if (r == rb0 + i) dhi = tb[r];
    }
    uint32_t f = __funnelshift_r(dlo, dhi, bs);
    if (w >= 2 * nl || 32 * w + 32 <= lowb) f = 0u;
    else if (32 * w < lowb) f &= ~((1u << (lowb - 32 * w)) - 1u);
    uint32_t inc = 0u;
    if (up && w == (lowb >> 5)) inc = 1u << (lowb & 31);
    acc[i] = (uint64_t)f + inc;
  }
  uint32_t F[DPL];
  const uint32_t ovf = normalize<GL, DPL>(acc, F, 0u, 2 * nl, lam, gbase);
  if (ovf) {
#pragma unroll
    for (int i = 0; i < DPL; ++i) F[i] = (lam + GL * i == 2 * nl - 1) ? 0x80000000u : 0u;
    n += 1;
  }

  const uint32_t lo_w = fetch<GL, DPL>(F, 0);
  const uint32_t hi_w = fetch<GL, DPL>(F, 1);
  if (!valid) return;
  if (P.kind == 1) {
    // binary64 output (p = 53, one limb): assemble the double from the limb
    if (lam != 0) return;
    double out = 0.0;
    if (top >= 0) {
      const uint64_t limb = ((uint64_t)hi_w << 32) | lo_w;
      const int e = n + P.e[row] + P.f[col] - 2 * P.t;   // |x| in [2^(e-1), 2^e)
      const int bexp = e - 1 + 1023;
      const uint64_t sgn = neg ? (1ull << 63) : 0ull;
      if (bexp >= 1 && bexp <= 2046) {
        out = __longlong_as_double((long long)(sgn | ((uint64_t)bexp << 52) | ((limb >> 11) & ((1ull << 52) - 1))));
      } else {
        out = ldexp((double)(limb >> 11), e - 53);
        if (neg) out = -out;
      }
    }
    P.c_f64[row * P.c_f64_ld + col] = out;
    return;
  }
  uint32_t* limbs32 = reinterpret_cast<uint32_t*>(P.c_limbs);
  const int64_t coff = row * P.c_ld + col;
#pragma unroll
  for (int i = 0; i < DPL; ++i) {
    const int w = lam + GL * i;
    if (w < 2 * nl) limbs32[2 * ((int64_t)(w >> 1) * P.c_ps + coff) + (w & 1)] = top >= 0 ? F[i] : 0u;
  }
  if (lam == 0) {
    P.c_exp[coff] = top >= 0 ? n + P.e[row] + P.f[col] - 2 * P.t : 0;
    P.c_sign[coff] = (top >= 0 && neg) ? 1 : 0;
  }
}

// ---------------------------------------------------------------------------
// One lane per output element (CRT accumulators of up to 40 digits).  The
// warps of a block cooperate on the staging: the reduced products of 128
// consecutive outputs are read coalesced and turned into v_l, and the digit
// table M_l and the quotient constants are staged in shared memory, where
// every lane of a warp reads the same word (broadcast).  Each lane then runs
// the whole CRT and rounding of its output with the digits in registers and
// sequential exact carries.
// ---------------------------------------------------------------------------
constexpr int kEpb1 = 128;

template <int ND>
__global__ void __launch_bounds__(kEpb1) k_crt1(DevTables T, const int4* __restrict__ blk) {
  extern __shared__ __align__(16) uint32_t s1[];
  const int4 b = blk[blockIdx.x];
  const ProbDev& P = T.probs[b.x];
  const int64_t MN = (int64_t)P.M * P.N;
  const int64_t e0 = (int64_t)b.y * kEpb1;
  const int L = P.L;
  const int D = P.D32;
  const CrtView cv = crt_view(T.crt_pool, P);
  uint16_t* s_v = reinterpret_cast<uint16_t*>(s1);          // [L][kEpb1] (16-byte rows)
  uint32_t* s_M = s1 + L * (kEpb1 / 2);                       // [L][ND]
  uint32_t* s_mu = s_M + L * ND;                              // [L]
  uint32_t* s_tab = s_mu + L;                                 // [3][ND]: negP, negH1, P
  uint32_t* s_mag = s_tab + 3 * ND;                           // [ND][kEpb1]
  for (int i = threadIdx.x; i < L * ND; i += kEpb1) s_M[i] = __ldg(cv.Mdig + i);
  for (int i = threadIdx.x; i < ND; i += kEpb1) {
    s_tab[i] = __ldg(cv.negP + i);
    s_tab[ND + i] = __ldg(cv.negH1 + i);
    s_tab[2 * ND + i] = __ldg(cv.P + i);
  }
  // v_l = u_l M_l^{-1} mod m_l: 16-byte loads of 8 reduced products; a block
  // covers 16 x 8 = 128 outputs of 8 moduli per pass, independent loads first
  {
    const int lane8 = threadIdx.x & 15;                       // which 8 outputs
    const int lrow = threadIdx.x >> 4;                        // modulus within the pass
    const bool full = e0 + kEpb1 <= MN && (MN & 7) == 0;
    for (int l0 = 0; l0 < L; l0 += 8 * 4) {
      uint4 w[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int l = l0 + 8 * j + lrow;
        w[j] = make_uint4(0u, 0u, 0u, 0u);
        if (l < L) {
          const uint16_t* src = P.u + (int64_t)l * MN + e0 + 8 * lane8;
          if (full) {
            w[j] = __ldg(reinterpret_cast<const uint4*>(src));
          } else {
            uint16_t tmp[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) tmp[q] = (e0 + 8 * lane8 + q < MN) ? src[q] : (uint16_t)0;
            w[j].x = tmp[0] | ((uint32_t)tmp[1] << 16); w[j].y = tmp[2] | ((uint32_t)tmp[3] << 16);
            w[j].z = tmp[4] | ((uint32_t)tmp[5] << 16); w[j].w = tmp[6] | ((uint32_t)tmp[7] << 16);
          }
        }
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int l = l0 + 8 * j + lrow;
        if (l >= L) continue;
        const ModConst mc = T.mods[l];
        const uint32_t inv = __ldg(cv.Minv + l);
        const uint32_t in[4] = {w[j].x, w[j].y, w[j].z, w[j].w};
        uint32_t o[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const uint32_t lo = barrett32((in[q] & 0xffffu) * inv, mc.m, mc.mu);
          const uint32_t hi = barrett32((in[q] >> 16) * inv, mc.m, mc.mu);
          o[q] = lo | (hi << 16);
        }
        *reinterpret_cast<uint4*>(s_v + l * kEpb1 + 8 * lane8) = make_uint4(o[0], o[1], o[2], o[3]);
        if (lane8 == 0) s_mu[l] = mc.mu;
      }
    }
  }
  __syncthreads();
  const int e = threadIdx.x;
  const int64_t idx = e0 + e;
  if (idx >= MN) return;

  // quotient estimate alpha~ in {alpha - 1, alpha}
  uint64_t sig = 0;
  for (int l = 0; l < L; ++l) sig += (uint64_t)(uint32_t)s_v[l * kEpb1 + e] * s_mu[l];
  const uint32_t alpha = (uint32_t)(sig >> 32);

  // R = S + alpha~ (2^(32 D) - P) mod 2^(32 D)
  uint64_t acc[ND];
#pragma unroll
  for (int d = 0; d < ND; ++d) acc[d] = (uint64_t)alpha * s_tab[d];
  for (int l = 0; l < L; ++l) {
    const uint32_t v = s_v[l * kEpb1 + e];
    const uint4* mrow = reinterpret_cast<const uint4*>(s_M + l * ND);
#pragma unroll
    for (int q = 0; q < ND / 4; ++q) {
      const uint4 m4 = mrow[q];
      acc[4 * q + 0] += (uint64_t)v * m4.x;
      acc[4 * q + 1] += (uint64_t)v * m4.y;
      acc[4 * q + 2] += (uint64_t)v * m4.z;
      acc[4 * q + 3] += (uint64_t)v * m4.w;
    }
  }
  uint32_t R[ND];
  {
    uint64_t c = 0;
#pragma unroll
    for (int d = 0; d < ND; ++d) {
      const uint64_t x = acc[d] + c;            // acc < 2^63, c < 2^32
      R[d] = d < D ? (uint32_t)x : 0u;
      c = x >> 32;
    }
  }
  // carry out of digit D-1 of (R + Y) for a table Y of D digits
  auto carry_out = [&](const uint32_t* Y, uint32_t (&out)[ND], uint32_t cin) -> uint32_t {
    uint64_t c = cin;
    uint32_t co = 0;
#pragma unroll
    for (int d = 0; d < ND; ++d) {
      const uint64_t x = (uint64_t)R[d] + Y[d] + c;
      out[d] = d < D ? (uint32_t)x : 0u;
      c = x >> 32;
      if (d == D - 1) co = (uint32_t)c;
    }
    return co;
  };
  uint32_t W[ND];
  // R in [0, 2P): subtract P once if R >= P
  if (carry_out(s_tab, W, 0u)) {
#pragma unroll
    for (int d = 0; d < ND; ++d) R[d] = W[d];
  }
  if (carry_out(s_tab, W, 0u)) atomicOr(T.status, kStatusCrtRange);     // x0 < P must hold
  const bool neg = carry_out(s_tab + ND, W, 0u) != 0u;                  // x0 > floor(P/2)
  if (neg) {
    // |c_hat| = P - x0 = P + ~x0 + 1 (mod 2^(32 D))
    uint64_t c = 1;
#pragma unroll
    for (int d = 0; d < ND; ++d) {
      const uint64_t x = (uint64_t)s_tab[2 * ND + d] + (uint32_t)~R[d] + c;
      c = x >> 32;
      R[d] = d < D ? (uint32_t)x : 0u;
    }
  }
  if (P.dbg_chat != nullptr) {
    uint32_t* dst = P.dbg_chat + idx * (int64_t)(D + 1);
    dst[0] = neg;
#pragma unroll
    for (int d = 0; d < ND; ++d)
      if (d < D) dst[1 + d] = R[d];
  }
  int top = -1;
#pragma unroll
  for (int d = 0; d < ND; ++d) {
    s_mag[d * kEpb1 + e] = R[d];
    if (R[d]) top = d;
  }
  const int64_t row = idx / P.N, col = idx - row * P.N;
  auto mag_word = [&](int w) -> uint32_t {
    return (w >= 0 && w < ND) ? s_mag[w * kEpb1 + e] : 0u;
  };
  const int p = P.p, nl = P.nl;
  if (top < 0) {
    if (P.kind == 1) {
      P.c_f64[row * P.c_f64_ld + col] = 0.0;
    } else {
      const int64_t coff = row * P.c_ld + col;
      for (int q = 0; q < nl; ++q) P.c_limbs[(int64_t)q * P.c_ps + coff] = 0ull;
      P.c_exp[coff] = 0;
      P.c_sign[coff] = 0;
    }
    return;
  }
  int n = 32 * top + 32 - __clz(mag_word(top));
  const int sh = n - p, rpos = sh - 1;
  uint32_t up = 0;
  if (rpos >= 0) {
    const uint32_t rb = (mag_word(rpos >> 5) >> (rpos & 31)) & 1u;
    const uint32_t lsb = (mag_word(sh >> 5) >> (sh & 31)) & 1u;
    uint32_t sticky = mag_word(rpos >> 5) & ((1u << (rpos & 31)) - 1u);
    for (int w = (rpos >> 5) - 1; w >= 0 && !sticky; --w) sticky = mag_word(w);
    up = rb & ((sticky != 0u) | lsb);
  }
  // F = floor(|c_hat| 2^(64 nl - n)), low 64 nl - p bits cleared, plus the
  // rounding increment at bit 64 nl - p
  const int base = n - 64 * nl;
  const int q0 = base >> 5, bs = base & 31;
  const int lowb = 64 * nl - p;
  uint32_t F[ND];
  uint64_t c = 0;
  bool ovf = false;
#pragma unroll
  for (int w = 0; w < ND; ++w) {
    uint32_t f = 0u;
    if (w < 2 * nl) {
      f = __funnelshift_r(mag_word(q0 + w), mag_word(q0 + w + 1), bs);
      if (32 * w + 32 <= lowb) f = 0u;
      else if (32 * w < lowb) f &= ~((1u << (lowb - 32 * w)) - 1u);
    }
    const uint64_t x = (uint64_t)f + (uint64_t)((up && w == (lowb >> 5)) ? (1u << (lowb & 31)) : 0u) + c;
    F[w] = (uint32_t)x;
    c = (w < 2 * nl) ? (x >> 32) : 0u;
    if (w == 2 * nl - 1 && c) ovf = true;    // rounded up to 2^p
  }
  if (ovf) {
#pragma unroll
    for (int w = 0; w < ND; ++w) F[w] = (w == 2 * nl - 1) ? 0x80000000u : 0u;
    n += 1;
  }
  const int eo = n + P.e[row] + P.f[col] - 2 * P.t;
  if (P.kind == 1) {
    const uint64_t limb = ((uint64_t)F[1] << 32) | F[0];
    double out;
    const int bexp = eo - 1 + 1023;
    const uint64_t sgn = neg ? (1ull << 63) : 0ull;
    if (bexp >= 1 && bexp <= 2046) {
      out = __longlong_as_double((long long)(sgn | ((uint64_t)bexp << 52) | ((limb >> 11) & ((1ull << 52) - 1))));
    } else {
      out = ldexp((double)(limb >> 11), eo - 53);
      if (neg) out = -out;
    }
    P.c_f64[row * P.c_f64_ld + col] = out;
    return;
  }
  const int64_t coff = row * P.c_ld + col;
#pragma unroll
  for (int q = 0; q < ND / 2; ++q)
    if (q < nl) P.c_limbs[(int64_t)q * P.c_ps + coff] = ((uint64_t)F[2 * q + 1] << 32) | F[2 * q];
  P.c_exp[coff] = eo;
  P.c_sign[coff] = neg ? 1 : 0;
}

// Classes 0..8: one lane per output with ND = 8, 12, ..., 40 digits;
// classes 9..11: lane groups (GL lanes x DPL digits) for larger accumulators.
struct CrtClass { int gl, dpl; };
const CrtClass kCrtClasses[] = {{1, 8},  {1, 12}, {1, 16}, {1, 20}, {1, 24}, {1, 28},
                                {1, 32}, {1, 36}, {1, 40}, {16, 4}, {16, 6}, {32, 5}};
constexpr int kNumCrtClasses = 12;

template <int GL, int DPL>
cudaError_t launch_crt_t(const DevTables& t, const int4* blk, int nblk, int smem, cudaStream_t s) {
  k_crt<GL, DPL><<<nblk, 256, smem, s>>>(t, blk);
  return cudaGetLastError();
}

template <int GL, int DPL>
cudaError_t crt_attr() {
  return cudaFuncSetAttribute(k_crt<GL, DPL>, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024);
}

template <int ND>
cudaError_t crt1_attr() {
  return cudaFuncSetAttribute(k_crt1<ND>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
}

template <int ND>
cudaError_t launch_crt1_t(const DevTables& t, const int4* blk, int nblk, int lmax, cudaStream_t s) {
  const int smem = lmax * ND * 4 + lmax * 4 + 3 * ND * 4 + ND * kEpb1 * 4 + lmax * kEpb1 * 2 + 16;
  k_crt1<ND><<<nblk, kEpb1, smem, s>>>(t, blk);
  return cudaGetLastError();
}

}  // namespace

cudaError_t init_crt_attributes() {
  cudaError_t e = crt1_attr<8>();
  if (e == cudaSuccess) e = crt1_attr<12>();
  if (e == cudaSuccess) e = crt1_attr<16>();
  if (e == cudaSuccess) e = crt1_attr<20>();
  if (e == cudaSuccess) e = crt1_attr<24>();
  if (e == cudaSuccess) e = crt1_attr<28>();
  if (e == cudaSuccess) e = crt1_attr<32>();
  if (e == cudaSuccess) e = crt1_attr<36>();
  if (e == cudaSuccess) e = crt1_attr<40>();
  if (e == cudaSuccess) e = crt_attr<16, 4>();
  if (e == cudaSuccess) e = crt_attr<16, 6>();
  if (e == cudaSuccess) e = crt_attr<32, 5>();
  return e;
}

int crt_class_for(int d32) {
  for (int i = 0; i < kNumCrtClasses; ++i) {
    const CrtClass& c = kCrtClasses[i];
    // one-lane classes hold exactly D digits; lane groups need digit D as the carry slot
    if (c.gl == 1 ? d32 <= c.dpl : d32 + 1 <= c.gl * c.dpl) return i;
  }
  return -1;
}
int crt_class_elems_per_block(int cls) {
  return kCrtClasses[cls].gl == 1 ? kEpb1 : 256 / kCrtClasses[cls].gl;
}
int crt_class_digits(int cls) { return kCrtClasses[cls].gl * kCrtClasses[cls].dpl; }

cudaError_t launch_crt(const DevTables& t, int cls, const int32_t* blk_list, int nblk, int lmax,
                       cudaStream_t s) {
  static_assert(sizeof(int4) == 16, "block list entries are int4");
  if (nblk == 0) return cudaSuccess;
  const int4* blk = reinterpret_cast<const int4*>(blk_list);
  const int smem = lmax * crt_class_elems_per_block(cls) * 2;
  switch (cls) {
    case 0: return launch_crt1_t<8>(t, blk, nblk, lmax, s);
    case 1: return launch_crt1_t<12>(t, blk, nblk, lmax, s);
    case 2: return launch_crt1_t<16>(t, blk, nblk, lmax, s);
    case 3: return launch_crt1_t<20>(t, blk, nblk, lmax, s);
    case 4: return launch_crt1_t<24>(t, blk, nblk, lmax, s);
    case 5: return launch_crt1_t<28>(t, blk, nblk, lmax, s);
    case 6: return launch_crt1_t<32>(t, blk, nblk, lmax, s);
    case 7: return launch_crt1_t<36>(t, blk, nblk, lmax, s);
    case 8: return launch_crt1_t<40>(t, blk, nblk, lmax, s);
    case 9: return launch_crt_t<16, 4>(t, blk, nblk, smem, s);
    case 10: return launch_crt_t<16, 6>(t, blk, nblk, smem, s);
    case 11: return launch_crt_t<32, 5>(t, blk, nblk, smem, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace oz2
