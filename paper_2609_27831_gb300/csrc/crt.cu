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
#include "tc_ptx.cuh"

namespace oz2 {

namespace {

constexpr unsigned kFull = 0xffffffffu;

// Row and column of output idx = row N + col: a 32-bit division while idx
// fits in 32 bits (N is a positive 32-bit count), the 64-bit one beyond.
__device__ __forceinline__ void out_row_col(const ProbDev& P, int64_t idx, int64_t& row, int64_t& col) {
  if (((uint64_t)idx >> 32) == 0u) {
    const uint32_t n = (uint32_t)P.N, r = (uint32_t)idx / n;
    row = r;
    col = (uint32_t)idx - r * n;
  } else {
    row = idx / P.N;
    col = idx - row * P.N;
  }
}

// two small non-negative integers (<= 256) as a packed bf16 pair (low, high)
__device__ __forceinline__ uint32_t bf16_pair(uint32_t lo, uint32_t hi) {
  return (__float_as_uint((float)lo) >> 16) | (__float_as_uint((float)hi) & 0xffff0000u);
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
    s_v[i] = idx < MN ? P.u[(int64_t)l * P.upitch + idx] : (uint16_t)0;   // v_l from the plane GEMM
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

  int64_t row = 0, col = 0;
  if (valid) out_row_col(P, idx, row, col);
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

// e_i + f_j of output idx (row i, column j), loaded where a kernel starts so
// that the rounding does not wait for it
__device__ __forceinline__ int crt_ef(const ProbDev& P, int64_t idx) {
  int64_t row, col;
  out_row_col(P, idx, row, col);
  return __ldg(P.e + row) + __ldg(P.f + col);
}

// Round |c_hat| times 2^(e_i + f_j - 2t) to p bits, round-half-even, and
// write output idx (limbs, exponent and sign, or a binary64 value); ef =
// e_i + f_j.  Digits wbase .. wbase + nd - 1 of |c_hat| are in column e of
// s_mag (row w - wbase for digit w), `top` is the highest nonzero digit (-1
// for zero, else within the window), and sticky_below is nonzero iff a digit
// below wbase is (the window covers every digit the rounding reads but the
// sticky ones).
__device__ __forceinline__ void crt_round_write(const ProbDev& P, const uint32_t* s_mag, int ldm, int e, int nd,
                                             int top, bool neg, int64_t idx, int ef, int wbase = 0,
                                             uint32_t sticky_below = 0u) {
  int64_t row, col;
  out_row_col(P, idx, row, col);
  auto mag_word = [&](int w) -> uint32_t {
    return (w >= wbase && w < wbase + nd) ? s_mag[(w - wbase) * ldm + e] : 0u;
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
    uint32_t sticky = (mag_word(rpos >> 5) & ((1u << (rpos & 31)) - 1u)) | sticky_below;
    for (int w = (rpos >> 5) - 1; w >= wbase && !sticky; --w) sticky = mag_word(w);
    up = rb & ((sticky != 0u) | lsb);
  }
  // the 2 nl output words: F = floor(|c_hat| 2^(64 nl - n)) with the low
  // 64 nl - p bits cleared, plus the rounding increment at bit 64 nl - p
  const int base = n - 64 * nl;
  const int q0 = base >> 5, bs = base & 31;
  const int lowb = 64 * nl - p;
  const bool kind1 = P.kind == 1;
  const int64_t coff = row * P.c_ld + col;
  uint64_t c = 0;
  uint32_t prev = 0;
  uint64_t limb0 = 0;
  for (int w = 0; w < 2 * nl; ++w) {
    uint32_t f = __funnelshift_r(mag_word(q0 + w), mag_word(q0 + w + 1), bs);
    if (32 * w + 32 <= lowb) f = 0u;
    else if (32 * w < lowb) f &= ~((1u << (lowb - 32 * w)) - 1u);
    const uint64_t x = (uint64_t)f + (uint64_t)((up && w == (lowb >> 5)) ? (1u << (lowb & 31)) : 0u) + c;
    const uint32_t fw = (uint32_t)x;
    c = x >> 32;
    if (w & 1) {
      const uint64_t limb = ((uint64_t)fw << 32) | prev;
      if (kind1) limb0 = limb;
      else P.c_limbs[(int64_t)(w >> 1) * P.c_ps + coff] = limb;
    }
    prev = fw;
  }
  if (c) {                                        // rounded up to 2^p: renormalise
    n += 1;
    if (!kind1) {
      for (int q = 0; q < nl - 1; ++q) P.c_limbs[(int64_t)q * P.c_ps + coff] = 0ull;
      P.c_limbs[(int64_t)(nl - 1) * P.c_ps + coff] = 1ull << 63;
    }
    limb0 = 1ull << 63;
  }
  const int eo = n + ef - 2 * P.t;
  if (kind1) {
    double out;
    const int bexp = eo - 1 + 1023;
    const uint64_t sgn = neg ? (1ull << 63) : 0ull;
    if (bexp >= 1 && bexp <= 2046) {
      out = __longlong_as_double((long long)(sgn | ((uint64_t)bexp << 52) | ((limb0 >> 11) & ((1ull << 52) - 1))));
    } else {
      out = ldexp((double)(limb0 >> 11), eo - 53);
      if (neg) out = -out;
    }
    P.c_f64[row * P.c_f64_ld + col] = out;
    return;
  }
  P.c_exp[coff] = eo;
  P.c_sign[coff] = neg ? 1 : 0;
}

// Multi-digit arithmetic on ND little-endian 32-bit digits, one PTX carry
// chain each (add.cc / addc.cc / addc: one integer add per digit).  The
// compiler emits no carry-flag instructions of its own, so the chain's
// statements may be separated by its loads and moves.
template <int ND>
__device__ __forceinline__ uint32_t add_digits(const uint32_t (&a)[ND], const uint32_t (&b)[ND], uint32_t (&s)[ND]) {
  uint32_t c;
  asm volatile("add.cc.u32 %0, %1, %2;" : "=r"(s[0]) : "r"(a[0]), "r"(b[0]));
#pragma unroll
  for (int d = 1; d < ND; ++d) asm volatile("addc.cc.u32 %0, %1, %2;" : "=r"(s[d]) : "r"(a[d]), "r"(b[d]));
  asm volatile("addc.u32 %0, 0, 0;" : "=r"(c));
  return c;
}
// carry out of a + b only
template <int ND>
__device__ __forceinline__ uint32_t carry_digits(const uint32_t (&a)[ND], const uint32_t (&b)[ND]) {
  uint32_t c, t;
  asm volatile("add.cc.u32 %0, %1, %2;" : "=r"(t) : "r"(a[0]), "r"(b[0]));
#pragma unroll
  for (int d = 1; d < ND; ++d) asm volatile("addc.cc.u32 %0, %1, %2;" : "=r"(t) : "r"(a[d]), "r"(b[d]));
  asm volatile("addc.u32 %0, 0, 0;" : "=r"(c));
  return c;
}
// s = a - b mod 2^(32 ND)
template <int ND>
__device__ __forceinline__ void sub_digits(const uint32_t (&a)[ND], const uint32_t (&b)[ND], uint32_t (&s)[ND]) {
  asm volatile("sub.cc.u32 %0, %1, %2;" : "=r"(s[0]) : "r"(a[0]), "r"(b[0]));
#pragma unroll
  for (int d = 1; d < ND - 1; ++d) asm volatile("subc.cc.u32 %0, %1, %2;" : "=r"(s[d]) : "r"(a[d]), "r"(b[d]));
  asm volatile("subc.u32 %0, %1, %2;" : "=r"(s[ND - 1]) : "r"(a[ND - 1]), "r"(b[ND - 1]));
}

// The CRT and rounding of one output from R = (S + alpha~ (2^(32 D) - P)) mod
// 2^(32 D), i.e. R in [0, 2P) (Sec. 4.4): subtract P once if R >= P, take the
// signed representative, round |c_hat| 2^(e_i + f_j - 2t) to p bits and write
// the output.  R holds zeros in digits D .. ND - 1.  tab: [3][ND] digits of
// 2^(32 ND) - P and 2^(32 ND) - (floor(P/2) + 1) (all ones from digit D on,
// so that every comparison is one carry chain over ND digits) and of P (zero
// from digit D on).  s_mag: scratch column e of a [ND][ldm] digit array.
//   T1 = R + 2^(32 ND) - P carries out iff R >= P (then x0 = T1 = R - P,
//        else x0 = R);
//   x0 + 2^(32 ND) - floor(P/2) - 1 carries out iff x0 > floor(P/2): c_hat
//        = x0 - P is negative, |c_hat| = P - x0;
//   x0 + 2^(32 ND) - P must not carry out (x0 < P), else the tables or the
//        sums are inconsistent and the status word records it.
template <int ND>
__device__ __forceinline__ void crt_finish(const ProbDev& P, uint32_t (&R)[ND], const uint32_t* s_tab,
                                           uint32_t* s_mag, int ldm, int e, int64_t idx, int ef, int32_t* status) {
  const int D = P.D32;
  uint32_t tab[ND], x0[ND];
#pragma unroll
  for (int d = 0; d < ND; ++d) tab[d] = s_tab[d];                   // 2^(32 ND) - P
  const bool ge = add_digits<ND>(R, tab, x0) != 0u;
#pragma unroll
  for (int d = 0; d < ND; ++d) x0[d] = ge ? x0[d] : R[d];
  const bool bad = carry_digits<ND>(x0, tab) != 0u;
#pragma unroll
  for (int d = 0; d < ND; ++d) tab[d] = s_tab[ND + d];              // 2^(32 ND) - floor(P/2) - 1
  const bool neg = carry_digits<ND>(x0, tab) != 0u;
#pragma unroll
  for (int d = 0; d < ND; ++d) tab[d] = s_tab[2 * ND + d];          // P
  sub_digits<ND>(tab, x0, R);                                       // P - x0
  if (bad) atomicOr(status, kStatusCrtRange);
  int top = -1;
#pragma unroll
  for (int d = 0; d < ND; ++d) {
    const uint32_t m = neg ? R[d] : x0[d];
    R[d] = m;
    s_mag[d * ldm + e] = m;
    if (m != 0u) top = d;
  }
  if (P.dbg_chat != nullptr) {
    uint32_t* dst = P.dbg_chat + idx * (int64_t)(D + 1);
    dst[0] = neg;
#pragma unroll
    for (int d = 0; d < ND; ++d)
      if (d < D) dst[1 + d] = R[d];
  }
  crt_round_write(P, s_mag, ldm, e, ND, top, neg, idx, ef);
}

// ---------------------------------------------------------------------------
// One lane per output element (CRT accumulators of up to 40 digits).  The
// warps of a block cooperate on the staging: the values v_l of 128
// consecutive outputs (as the plane GEMM stored them) are read coalesced, and
// the digit table M_l and the quotient constants are staged in shared memory, where
// every lane of a warp reads the same word (broadcast).  Each lane then runs
// the whole CRT and rounding of its output with the digits in registers and
// sequential exact carries.
// ---------------------------------------------------------------------------
constexpr int kEpb1 = 128;

// acc[d] += sum_l v_l M_l[d] for the first NM digits (the rest of M_l is zero)
template <int ND, int NM>
__device__ __forceinline__ void crt1_sum(uint64_t (&acc)[ND], const uint16_t* s_v, const uint32_t* s_M,
                                         int L, int e) {
  static_assert(NM % 4 == 0 && NM <= ND, "digit columns in groups of four");
  for (int l = 0; l < L; ++l) {
    const uint32_t v = s_v[l * kEpb1 + e];
    const uint4* mrow = reinterpret_cast<const uint4*>(s_M + l * ND);
#pragma unroll
    for (int q = 0; q < NM / 4; ++q) {
      const uint4 m4 = mrow[q];
      acc[4 * q + 0] += (uint64_t)v * m4.x;
      acc[4 * q + 1] += (uint64_t)v * m4.y;
      acc[4 * q + 2] += (uint64_t)v * m4.z;
      acc[4 * q + 3] += (uint64_t)v * m4.w;
    }
  }
}

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
  const int e = threadIdx.x;
  const int64_t idx = e0 + e;
  const int ef = idx < MN ? crt_ef(P, idx) : 0;               // early: used by the rounding
  uint16_t* s_v = reinterpret_cast<uint16_t*>(s1);          // [L][kEpb1] (16-byte rows)
  uint32_t* s_M = s1 + L * (kEpb1 / 2);                       // [L][ND]
  uint32_t* s_mu = s_M + L * ND;                              // [L]
  uint32_t* s_tab = s_mu + L;                                 // [3][ND]: negP, negH1, P
  uint32_t* s_mag = s_tab + 3 * ND;                           // [ND][kEpb1]
  for (int i = threadIdx.x; i < L * ND; i += kEpb1) s_M[i] = __ldg(cv.Mdig + i);
  for (int i = threadIdx.x; i < ND; i += kEpb1) {
    s_tab[i] = i < D ? __ldg(cv.negP + i) : ~0u;           // widened to ND digits (crt_finish)
    s_tab[ND + i] = i < D ? __ldg(cv.negH1 + i) : ~0u;
    s_tab[2 * ND + i] = i < D ? __ldg(cv.P + i) : 0u;
  }
  // v_l = (c mod m_l) M_l^{-1} mod m_l as the plane GEMM stored it: 16-byte
  // loads of 8 values; a block covers 16 x 8 = 128 outputs of 8 moduli per
  // pass, independent loads first
  {
    const int lane8 = threadIdx.x & 15;                       // which 8 outputs
    const int lrow = threadIdx.x >> 4;                        // modulus within the pass
    const bool full = e0 + kEpb1 <= MN;
    for (int l0 = 0; l0 < L; l0 += 8 * 4) {
      uint4 w[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int l = l0 + 8 * j + lrow;
        w[j] = make_uint4(0u, 0u, 0u, 0u);
        if (l < L) {
          const uint16_t* src = P.u + (int64_t)l * P.upitch + e0 + 8 * lane8;
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
        *reinterpret_cast<uint4*>(s_v + l * kEpb1 + 8 * lane8) = w[j];
        if (lane8 == 0) s_mu[l] = T.mods[l].mu;
      }
    }
  }
  __syncthreads();
  if (idx >= MN) return;

  // quotient estimate alpha~ in {alpha - 1, alpha}
  uint64_t sig = 0;
  for (int l = 0; l < L; ++l) sig += (uint64_t)(uint32_t)s_v[l * kEpb1 + e] * s_mu[l];
  const uint32_t alpha = (uint32_t)(sig >> 32);

  // R = S + alpha~ (2^(32 D) - P) mod 2^(32 D)
  uint64_t acc[ND];
#pragma unroll
  for (int d = 0; d < ND; ++d) acc[d] = (uint64_t)alpha * s_tab[d];
  // M_l < P < 2^(32 (D - 2)): digits D - 2 and up of every M_l are zero
  if (D - 2 <= ND - 4) crt1_sum<ND, ND - 4>(acc, s_v, s_M, L, e);
  else crt1_sum<ND, ND>(acc, s_v, s_M, L, e);
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
  crt_finish<ND>(P, R, s_tab, s_mag, kEpb1, e, idx, ef, T.status);
}


// ---------------------------------------------------------------------------
// CRT column sums on the tensor cores.  With v_l = v0 + 128 v1 (7-bit halves)
// and M_l = sum_j M_l[j] 128^j (7-bit pieces),
//   S = sum_l v_l M_l = sum_j 128^j Y_j,   Y_j = sum_l (v0_l M_l[j] + v1_l M_l[j-1]),
// which is one GEMM Y = V B with K = 2L (columns 2l, 2l+1 of V hold v0_l, v1_l)
// and N = the number of 7-bit pieces of S.  Every product is below 2^14 and
// every partial sum below 2L 2^14 < 2^23, so bf16 operands and the fp32 TMEM
// accumulator are exact.
//
// One CTA per tile of 128 consecutive outputs, 8 warps, sized for two CTAs
// per SM.  Thread 0 loads the piece table B and the tile's values v_l with
// TMA; all threads build V (two threads per output, half of the moduli
// each) together with the quotient estimate; thread 0 issues the MMAs; the
// epilogue splits the columns of Y between the two warps of each TMEM lane
// quadrant, carries sum_j 128^j Y_j into 32-bit digits, merges the halves and
// finishes the CRT and rounding of each output (crt_finish).
// Tile list entry: {problem, tile index, 0, 0}.
// ---------------------------------------------------------------------------
constexpr int kCtThreads = 256;

__host__ __device__ inline int crt_tc_tmem_cols(int npad) {
  int c = 32;
  while (c < npad) c <<= 1;
  return c;
}

// Shared-memory layout of the tensor-core CRT (launch-wide maxima).
struct CtLayout {
  uint32_t b_bytes, a_region, u_region, small_off, total;
  __host__ __device__ CtLayout(int ND, int kpad, int npad, int lmax) {
    b_bytes = (uint32_t)npad * kpad * 2;
    uint32_t a = (uint32_t)128 * kpad * 2;
    if (a < (uint32_t)(2 * ND * 128 * 4)) a = (uint32_t)(2 * ND * 128 * 4);   // digit arrays reuse a V buffer
    a_region = (a + 1023u) & ~1023u;
    u_region = ((uint32_t)lmax * 128 * 2 + 1023u) & ~1023u;
    small_off = b_bytes + 2 * a_region + 2 * u_region;
    // small: s_sig [2][2][128] u64, s_pc [lmax] uint4, s_tab [3][ND], 8 barriers, tmem slot
    total = 1024 + small_off + 4096 + (uint32_t)lmax * 16 + 3 * ND * 4 + 16 + 8 * 8 + 16;
  }
};

template <int ND>
__global__ void __launch_bounds__(kCtThreads, (ND <= 24 ? 2 : 1))
    k_crt_tc(const __grid_constant__ DevTables T, const int4* __restrict__ tiles, int ntiles, int kpad_max,
             int npad_max, int lmax) {
  using namespace tc;
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  uint8_t* sm = smem_raw + (base - raw);
  const CtLayout lay(ND, kpad_max, npad_max, lmax);
  const uint32_t sB = base;                                       // table [kb][npad][128 B]
  const uint32_t sA0 = base + lay.b_bytes;                        // V buffers [2]
  const uint32_t sU0 = sA0 + 2 * lay.a_region;                    // u tiles [2][L][128]
  uint8_t* small = sm + lay.small_off;
  uint64_t* s_sig = reinterpret_cast<uint64_t*>(small);            // [slot][half][128]
  uint4* s_pc = reinterpret_cast<uint4*>(small + 4096);            // [lmax]
  uint32_t* s_tab = reinterpret_cast<uint32_t*>(s_pc + lmax);      // [3][ND]
  uint64_t* bars = reinterpret_cast<uint64_t*>(s_tab + 3 * ND + 4);
  uint64_t* b_bar = bars;             // table loaded
  uint64_t* u_bar = bars + 1;         // [2] u tile landed
  uint64_t* m_bar = bars + 3;         // [2] MMA into slot done
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 8);

  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const int tcols = crt_tc_tmem_cols(npad_max);
  if (t == 0) {
    for (int i = 0; i < 5; ++i) mbar_init(bars + i, 1);
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
  uint32_t bcnt = 0, ucnt[2] = {0, 0}, mcnt[2] = {0, 0};
  bool ok = true;

  // u tile of tile list entry gi (problem `pr`) into buffer b (thread 0)
  auto issue_u = [&](int gi, int b) {
    const int4 t2 = tiles[gi];
    const ProbDev& Q = T.probs[t2.x];
    mbar_expect_tx(u_bar + b, (uint32_t)Q.L * 128 * 2);
    tma_load_2d(sU0 + b * lay.u_region, T.tmaps + 3 * T.count + t2.x, smem_u32(u_bar + b), t2.y * 128, 0);
  };

  // epilogue of tile `tp` held in TMEM slot `s`; digit arrays in V buffer `s`
  auto epilogue = [&](int4 tp, int s) {
    const ProbDev& P = T.probs[tp.x];
    const int D = P.D32, np = P.crt_np;
    if (ok) ok = mbar_wait(m_bar + s, mcnt[s] & 1u, &abort_flag, T.status, T.spin_limit);
    ++mcnt[s];
    ok = __syncthreads_and(ok);                   // keep every thread on the same path
    tc_fence_after();
    uint32_t* s_dig = reinterpret_cast<uint32_t*>(sm + lay.b_bytes + s * lay.a_region);   // [ND][128]
    uint32_t* s_part = s_dig + ND * 128;
    const int quad = warp & 3, hh = warp >> 2;
    const int er = quad * 32 + lane;
    const int half = ((np + 63) / 64) * 32;
    const int j0 = hh * half, j1 = min(np, j0 + half);
    uint32_t* dst = hh ? s_part : s_dig;
    if (ok) {
      for (int dd = 0; dd < ND; ++dd) dst[dd * 128 + er] = 0u;
      uint64_t win = 0;
      int d = (7 * j0) >> 5;
      const uint32_t trow = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(s * tcols);
      for (int c = j0; c < j1; c += 32) {
        uint32_t v[32];
        tmem_ld32(trow + (uint32_t)c, v);
#pragma unroll
        for (int q = 0; q < 32; ++q) {
          const int j = c + q;
          if (j < j1) {
            int sh = 7 * j - 32 * d;
            if (sh >= 32) {
              if (d < ND) dst[d * 128 + er] = (uint32_t)win;
              win >>= 32;
              ++d;
              sh -= 32;
            }
            // exact integer y < 2^23 held in fp32
            const uint32_t y = __float_as_uint(__uint_as_float(v[q]) + 8388608.0f) - 0x4B000000u;
            win += (uint64_t)y << sh;
          }
        }
      }
      for (; d < ND; ++d) {
        dst[d * 128 + er] = (uint32_t)win;
        win >>= 32;
      }
    }
    tc_fence_before();
    __syncthreads();
    if (hh == 0 && ok) {
      const uint32_t alpha =
          (uint32_t)((s_sig[(s * 2 + 0) * 128 + er] + s_sig[(s * 2 + 1) * 128 + er]) >> 32);
      uint32_t R[ND];
      uint64_t cr = 0;
#pragma unroll
      for (int q = 0; q < ND; ++q) {
        const uint64_t x = (uint64_t)s_dig[q * 128 + er] + s_part[q * 128 + er] + (uint64_t)alpha * s_tab[q] + cr;
        R[q] = q < D ? (uint32_t)x : 0u;
        cr = x >> 32;
      }
      const int64_t idx = (int64_t)tp.y * 128 + er;
      if (idx < (int64_t)P.M * P.N) crt_finish<ND>(P, R, s_tab, s_dig, 128, er, idx, crt_ef(P, idx), T.status);
    }
    __syncthreads();
  };

  int cur = -1;
  int k = 0;
  bool pending = false;
  int4 prev = make_int4(0, 0, 0, 0);
  for (int i = blockIdx.x;; i += gridDim.x) {
    const bool have = i < ntiles;
    int4 tl = have ? tiles[i] : make_int4(-1, 0, 0, 0);
    if (!have || tl.x != cur) {
      if (pending) {                                  // drain the previous problem
        epilogue(prev, (k - 1) & 1);
        pending = false;
      }
      if (!have || !ok) break;
      const ProbDev& P = T.probs[tl.x];
      const CrtView cv = crt_view(T.crt_pool, P);
      for (int l = t; l < P.L; l += kCtThreads) {
        const ModConst& mc = T.mods[l];
        s_pc[l] = make_uint4(mc.m, mc.mu, 0u, 0u);
      }
      for (int d = t; d < ND; d += kCtThreads) {
        s_tab[d] = d < P.D32 ? __ldg(cv.negP + d) : ~0u;   // widened to ND digits (crt_finish)
        s_tab[ND + d] = d < P.D32 ? __ldg(cv.negH1 + d) : ~0u;
        s_tab[2 * ND + d] = d < P.D32 ? __ldg(cv.P + d) : 0u;
      }
      __syncthreads();
      if (t == 0) {
        const int kb = P.crt_kpad / 64;
        const uint32_t tb = (uint32_t)P.crt_npad * 128;
        mbar_expect_tx(b_bar, tb * kb);
        for (int q = 0; q < kb; ++q)
          tma_load_2d(sB + q * tb, T.tmaps + 2 * T.count + tl.x, smem_u32(b_bar), q * 64, 0);
        issue_u(i, k & 1);
        const int i2 = i + gridDim.x;
        if (i2 < ntiles && tiles[i2].x == tl.x) issue_u(i2, (k + 1) & 1);
      }
      ok = mbar_wait(b_bar, bcnt & 1u, &abort_flag, T.status, T.spin_limit);
      ok = __syncthreads_and(ok);
      ++bcnt;
      cur = tl.x;
    }
    const ProbDev& P = T.probs[tl.x];
    const int L = P.L;
    const int b = k & 1;
    // ---- V for this tile (two threads per output, half of the moduli each)
    if (ok) ok = mbar_wait(u_bar + b, ucnt[b] & 1u, &abort_flag, T.status, T.spin_limit);
    ++ucnt[b];
    ok = __syncthreads_and(ok);
    if (!ok) break;
    {
      const int e = t & 127, h = t >> 7;
      const int lh = (L + 1) >> 1;
      const int l0 = h * lh, l1 = min(L, l0 + lh);
      const uint16_t* s_u = reinterpret_cast<const uint16_t*>(sm + lay.b_bytes + 2 * lay.a_region + b * lay.u_region);
      uint8_t* gA = sm + lay.b_bytes + b * lay.a_region;
      uint64_t sig = 0;
#pragma unroll 4
      for (int l = l0; l < l1; ++l) {
        const uint32_t v = s_u[l * 128 + e];          // v_l from the plane GEMM
        const uint4 pc = s_pc[l];
        sig += (uint64_t)v * pc.y;
        *reinterpret_cast<uint32_t*>(gA + tc::sw128_offset(e, 2 * l, 128)) = bf16_pair(v & 127u, v >> 7);
      }
      if (h == 1)
        for (int kk = 2 * L; kk < P.crt_kpad; kk += 2)
          *reinterpret_cast<uint32_t*>(gA + tc::sw128_offset(e, kk, 128)) = 0u;
      s_sig[(b * 2 + h) * 128 + e] = sig;
    }
    fence_proxy_async_smem();
    __syncthreads();
    if (t == 0) {
      tc_fence_after();
      const uint32_t idesc = idesc_bf16(128, P.crt_npad);
      const uint32_t tb = (uint32_t)P.crt_npad * 128;
      const uint32_t d = tmem + (uint32_t)(b * tcols);
      for (int q = 0; q < P.crt_kpad / 64; ++q) {
        const uint64_t da = desc_sw128(sA0 + b * lay.a_region + q * 128 * 128);
        const uint64_t db = desc_sw128(sB + q * tb);
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) umma_bf16(d, da + 2 * kk, db + 2 * kk, idesc, (q | kk) ? 1u : 0u);
      }
      umma_commit(m_bar + b);
      const int i3 = i + 2 * gridDim.x;                // u buffer b is free again
      if (i3 < ntiles && tiles[i3].x == tl.x) issue_u(i3, b);
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
// Finish of long accumulators (crt_mode 2, more than 24 digits): one thread
// per output, digit-serial, with no copy of R in shared memory.  Digit d of
//   R = (sum_g Q_g 2^(224 g) + alpha~ (2^(32 D) - P)) mod 2^(32 D)
// is rebuilt from the group words (read coalesced across the block, straight
// from global memory) each time it is needed:
//   pass 1: the carries out of R + (2^(32 D) - P) (R >= P: x0 = R - P, else
//           x0 = R) and of x + (2^(32 D) - floor(P/2) - 1) for x = R and
//           x = R - P (x0 > floor(P/2): c_hat = x0 - P is negative);
//   pass 2: the digits of |c_hat| = x0 or P - x0, the check x0 < P, the
//           highest nonzero digit, and a window of the W = 2 nl + 4 highest
//           digits D - W .. D - 1 in shared memory (the OR of the digits
//           below it kept as a sticky word);
//   the rounding reads its words from the window.  When |c_hat| is so small
//   that a word below the window is needed, a third pass writes the window
//   from the lowest needed word on.
// Both passes first run over the groups from the one below the window on
// only (the fast form, about half the group words at large D); the digits
// below that group enter only through one bounded carry, and the output
// keeps the fast result where no decision depends on that carry (else it
// runs the full form above).
// Block list entry: {problem, block of 128 outputs, 0, 0}.
// ---------------------------------------------------------------------------
constexpr int kFinThreads = 128;

// Carry chains over a group of N digits with the carry (or borrow) in and
// out as a register: cin must be 0 or 1; the chain starts by turning it into
// the carry flag (cin + 0xffffffff carries out iff cin = 1).
template <int N>
__device__ __forceinline__ uint32_t add_chain(const uint32_t (&a)[N], const uint32_t (&b)[N], uint32_t (&s)[N],
                                              uint32_t cin) {
  uint32_t t, c;
  asm volatile("add.cc.u32 %0, %1, 0xffffffff;" : "=r"(t) : "r"(cin));
#pragma unroll
  for (int d = 0; d < N; ++d) asm volatile("addc.cc.u32 %0, %1, %2;" : "=r"(s[d]) : "r"(a[d]), "r"(b[d]));
  asm volatile("addc.u32 %0, 0, 0;" : "=r"(c));
  return c;
}
template <int N>
__device__ __forceinline__ uint32_t carry_chain(const uint32_t (&a)[N], const uint32_t (&b)[N], uint32_t cin) {
  uint32_t t, c;
  asm volatile("add.cc.u32 %0, %1, 0xffffffff;" : "=r"(t) : "r"(cin));
#pragma unroll
  for (int d = 0; d < N; ++d) asm volatile("addc.cc.u32 %0, %1, %2;" : "=r"(t) : "r"(a[d]), "r"(b[d]));
  asm volatile("addc.u32 %0, 0, 0;" : "=r"(c));
  return c;
}
// s = a - b - bin, returns the borrow out (bin 0 or 1)
template <int N>
__device__ __forceinline__ uint32_t sub_chain(const uint32_t (&a)[N], const uint32_t (&b)[N], uint32_t (&s)[N],
                                              uint32_t bin) {
  uint32_t t;
  asm volatile("sub.cc.u32 %0, 0, %1;" : "=r"(t) : "r"(bin));
#pragma unroll
  for (int d = 0; d < N; ++d) asm volatile("subc.cc.u32 %0, %1, %2;" : "=r"(s[d]) : "r"(a[d]), "r"(b[d]));
  asm volatile("subc.u32 %0, 0, 0;" : "=r"(t));
  return t & 1u;
}

__global__ void __launch_bounds__(kFinThreads) k_crt_fin_long(DevTables T, const int4* __restrict__ blk) {
  extern __shared__ __align__(16) uint32_t sf[];
  const int4 b = blk[blockIdx.x];
  const ProbDev& P = T.probs[b.x];
  const int D = P.D32, ng = P.crt_ngrp, gsk = P.crt_gskip;   // group sums stored from group gsk on
  const int DG = 7 * ((D + 6) / 7);     // digits rounded up to whole groups of seven
  const int W = 2 * P.nl + 4, Wcap = W + 6;   // window digits: used, held
  const CrtView cv = crt_view(T.crt_pool, P);
  // tables over DG digits: 2^(32 DG) - P and 2^(32 DG) - floor(P/2) - 1
  // (all ones from digit D on, so that every carry chain may run over whole
  // groups: R is zero there) and P (zero from digit D on)
  uint32_t* s_negP = sf;                // [DG]
  uint32_t* s_negH1 = s_negP + DG;      // [DG]
  uint32_t* s_P = s_negH1 + DG;         // [DG]
  uint32_t* s_win = s_P + DG;           // [Wcap][128]
  for (int i = threadIdx.x; i < DG; i += kFinThreads) {
    s_P[i] = i < D ? __ldg(cv.P + i) : 0u;
    s_negP[i] = i < D ? __ldg(cv.negP + i) : ~0u;
    s_negH1[i] = i < D ? __ldg(cv.negH1 + i) : ~0u;
  }
  __syncthreads();
  const int e = threadIdx.x, lane = e & 31;
  // lanes past the last output do no output work but join the warp-wide
  // rebuild of R below
  const bool valid = (int64_t)b.y * kFinThreads + e < (int64_t)P.M * P.N;
  const int64_t idx = valid ? (int64_t)b.y * kFinThreads + e : 0;
  const int ef = valid ? crt_ef(P, idx) : 0;
  const int64_t up = P.upitch;
  const uint32_t* const qcol = P.crt_q + idx;
  const uint32_t alpha = valid ? __ldg(P.crt_alpha + idx) : 0u;
  // R seven digits at a time from group gs on, to f(g, r): word k of group g
  // is digit 7 g + k (k < 7); words 7 and 8 of group g add into digits
  // 7 g + 7 and 7 g + 8; digits from D on are zero.  The nine words of group
  // g + 1 are loaded while group g's digits are formed.  From gs > 0 the
  // carry into digit 7 gs from the digits below is left out: the digits come
  // out as those of R_up + c (R_up: R's digits from 7 gs on) with c, the
  // carry that was left out, at most alpha + 2 (every digit step adds below
  // (alpha + 2) 2^32 to a carry of at most alpha + 2).
  // Where the group sums below group gsk were not formed and an output needs
  // its full form, R comes from the plane GEMM's v_l instead, digit d of
  // sum_l v_l M_l + alpha~ (2^(32 D) - P), built by the whole warp (below)
  // into the owning thread's array (from_v).
  uint32_t Rv[kCrtSkipMaxDigits];
  bool from_v = false;
  auto for_each_group = [&](int gs, auto&& f) {
    if (from_v) {
      for (int g = gs; 7 * g < D; ++g) {
        uint32_t r[7];
#pragma unroll
        for (int k = 0; k < 7; ++k) r[k] = 7 * g + k < D ? Rv[7 * g + k] : 0u;
        f(g, r);
      }
      return;
    }
    uint32_t wc[9], wn[9];
    auto load = [&](int g, uint32_t (&w)[9]) {
#pragma unroll
      for (int k = 0; k < 9; ++k)
        w[k] = (g >= gsk && g - gsk < ng) ? __ldg(qcol + ((int64_t)(g - gsk) * 9 + k) * up) : 0u;
    };
    load(gs, wc);
    uint32_t prev7 = 0, prev8 = 0;
    if (gs > 0) {                        // gs - 1 >= gsk: that group's sum is stored
      prev7 = __ldg(qcol + ((int64_t)(gs - 1 - gsk) * 9 + 7) * up);
      prev8 = __ldg(qcol + ((int64_t)(gs - 1 - gsk) * 9 + 8) * up);
    }
    uint64_t carry = 0;
    for (int g = gs; 7 * g < D; ++g) {
      load(g + 1, wn);
      uint32_t r[7];
#pragma unroll
      for (int k = 0; k < 7; ++k) {
        const int d = 7 * g + k;
        uint64_t x = carry + (uint64_t)alpha * s_negP[d] + wc[k];
        if (k == 0) x += prev7;
        if (k == 1) x += prev8;
        carry = x >> 32;
        r[k] = d < D ? (uint32_t)x : 0u;
      }
      f(g, r);
      prev7 = wc[7];
      prev8 = wc[8];
#pragma unroll
      for (int k = 0; k < 9; ++k) wc[k] = wn[k];
    }
  };
  auto tab7 = [&](const uint32_t* t, int g, uint32_t (&v)[7]) {
#pragma unroll
    for (int k = 0; k < 7; ++k) v[k] = t[7 * g + k];
  };
  // From gs > 0 every chain below starts at digit d0 = 7 gs with no carry
  // in, and digit d0 of each of its operands is short by at most alpha + 3
  // (c, one carry or borrow of a chain below d0, one of the chain before).
  // Where the chain's digit d0 stays at least U = alpha + 5 away from both
  // ends of its range, no such shortfall moves a carry or borrow out of
  // digit d0: the chain's higher digits and carry out are exact.  `exact`
  // records that for every digit d0 the finish uses.
  const uint32_t U = alpha + 5u;
  auto safe = [&](uint32_t v) { return v >= U && v <= 0xffffffffu - U; };
  bool exact = true;
  // pass 1: R >= P (R + 2^(32 DG) - P carries out), and the sign of x0 for
  // either choice (x + 2^(32 DG) - floor(P/2) - 1 carries out iff x > floor(P/2))
  uint32_t c1 = 0, c3 = 0, c4 = 0;
  auto pass1 = [&](int gs) {
    c1 = c3 = c4 = 0;
    for_each_group(gs, [&](int g, const uint32_t (&r)[7]) {
      uint32_t np[7], nh[7], t1[7];
      tab7(s_negP, g, np);
      tab7(s_negH1, g, nh);
      c1 = add_chain<7>(r, np, t1, c1);                        // R - P
      c3 = carry_chain<7>(r, nh, c3);
      c4 = carry_chain<7>(t1, nh, c4);
      if (gs > 0 && g == gs) exact = safe(r[0]) && safe(t1[0]) && safe(r[0] + nh[0]) && safe(t1[0] + nh[0]);
    });
  };
  uint32_t* const dbg = P.dbg_chat != nullptr ? P.dbg_chat + idx * (int64_t)(D + 1) : nullptr;
  bool ge = false, neg = false;
  // pass 2 (and 3): |c_hat| = x0 or P - x0 digit by digit; digits from
  // wbase on go to the window, the ones below it into the sticky word
  // (from gs > 0: the digits above d0 only)
  int top = -1;
  uint32_t topv = 0, sticky = 0, bad = 0;
  auto magnitude = [&](int wbase, bool dump, int gs) {
    uint32_t cs = 0, cc = 0, br = 0;
    top = -1;
    sticky = 0;
    for_each_group(gs, [&](int g, const uint32_t (&r)[7]) {
      uint32_t np[7], pp[7], x0[7], pm[7];
      tab7(s_negP, g, np);
      tab7(s_P, g, pp);
      cs = add_chain<7>(r, np, x0, cs);                      // R - P
#pragma unroll
      for (int k = 0; k < 7; ++k) x0[k] = ge ? x0[k] : r[k];
      cc = carry_chain<7>(x0, np, cc);                       // carries out iff x0 >= P
      br = sub_chain<7>(pp, x0, pm, br);                     // P - x0
      if (gs > 0 && g == gs) exact = exact && safe(x0[0]) && safe(x0[0] + np[0]) && safe(pp[0] - x0[0]);
#pragma unroll
      for (int k = 0; k < 7; ++k) {
        const int d = 7 * g + k;
        if (gs > 0 && d == 7 * gs) continue;               // short by up to alpha + 3
        const uint32_t mag = neg ? pm[k] : x0[k];
        if (mag) {
          top = d;
          topv = mag;
        }
        if (d >= wbase) {
          if (d < wbase + Wcap) s_win[(d - wbase) * kFinThreads + e] = mag;
        } else {
          sticky |= mag;
        }
        if (dump && d < D) dbg[1 + d] = mag;
      }
    });
    bad = cc;
  };
  int wbase = D > W ? D - W : 0;
  // Fast form: both passes from group g0 on (d0 = 7 g0, just below the
  // window), about half the group words where D is large; its window holds
  // every digit above d0 (at most W + 6).  It stands when every digit d0 it
  // uses is safe, the round bit lies above d0 and some bit between d0 and
  // the round bit is nonzero (the sticky bit is then set whatever lies
  // below); otherwise, and with the debug dump, the output takes the full
  // form from group 0.
  const int g0 = wbase > 7 ? (wbase - 1) / 7 : 0;
  bool fast = valid && dbg == nullptr && g0 > 0 && (gsk == 0 || gsk == g0 - 1);
  if (fast) {
    pass1(g0);
    ge = c1 != 0;
    neg = ge ? c4 != 0 : c3 != 0;
    fast = exact;
    if (fast) {
      const int wf = 7 * g0 + 1;                           // the lowest exact digit
      magnitude(wf, false, g0);
      fast = exact && top >= wf;
      if (fast) {
        const int rpos = 32 * top + 32 - __clz(topv) - P.p - 1;
        fast = rpos >= 32 * wf;
        if (fast) {
          uint32_t st = s_win[((rpos >> 5) - wf) * kFinThreads + e] & ((1u << (rpos & 31)) - 1u);
          for (int w = (rpos >> 5) - 1; w >= wf && !st; --w) st = s_win[(w - wf) * kFinThreads + e];
          fast = st != 0u;
        }
      }
      if (fast) wbase = wf;
    }
  }
  // R from v_l for each lane whose fast form did not stand while the lower
  // group sums were not formed, one such lane at a time by the whole warp:
  // lane j sums the digits d = j mod 32 over every modulus (the digits of
  // M_l read coalesced across the lanes, v_l one broadcast word; each sum is
  // below L 2^46 + alpha~ 2^32 < 2^56), then every lane runs the same carry
  // chain over the digits (each fetched from its lane) and the owner keeps
  // them.
  {
    const unsigned need = __ballot_sync(0xffffffffu, valid && !fast && gsk > 0);
    const int L = P.L, DS = P.DS;
    for (unsigned m = need; m; m &= m - 1) {
      const int src = __ffs(m) - 1;
      const int64_t sidx = __shfl_sync(0xffffffffu, idx, src);
      const uint32_t salpha = __shfl_sync(0xffffffffu, alpha, src);
      constexpr int kJ = kCrtSkipMaxDigits / 32;
      uint64_t acc[kJ];
#pragma unroll
      for (int j = 0; j < kJ; ++j) {
        const int d = 32 * j + lane;
        acc[j] = d < D ? (uint64_t)salpha * s_negP[d] : 0ull;
      }
      for (int l = 0; l < L; ++l) {
        const uint64_t v = __ldg(P.u + (int64_t)l * up + sidx);
        const uint32_t* ml = cv.Mdig + (int64_t)l * DS;
#pragma unroll
        for (int j = 0; j < kJ; ++j) {
          const int d = 32 * j + lane;
          if (32 * j < D && d < D) acc[j] += v * __ldg(ml + d);
        }
      }
      uint64_t c = 0;
#pragma unroll
      for (int j = 0; j < kJ; ++j) {
        if (32 * j >= D) break;
        for (int ln = 0; ln < 32 && 32 * j + ln < D; ++ln) {
          const uint64_t x = __shfl_sync(0xffffffffu, acc[j], ln) + c;
          c = x >> 32;
          if (lane == src) Rv[32 * j + ln] = (uint32_t)x;
        }
      }
      if (lane == src) from_v = true;
    }
  }
  if (!valid) return;
  if (!fast) {
    exact = true;
    pass1(0);
    ge = c1 != 0;               // R >= P: x0 = R - P
    neg = ge ? c4 != 0 : c3 != 0;
    if (dbg) dbg[0] = neg;
    magnitude(wbase, dbg != nullptr, 0);
    if (top >= 0) {
      // lowest word the rounding reads: the one holding the round bit (or 0
      // when |c_hat| has at most p bits)
      const int n = 32 * top + 32 - __clz(topv);
      const int lo = n > P.p ? (n - P.p - 1) >> 5 : 0;
      if (lo < wbase) {
        wbase = lo;
        magnitude(wbase, false, 0);
      }
    }
  }
  if (bad) atomicOr(T.status, kStatusCrtRange);
  crt_round_write(P, s_win, kFinThreads, e, min(Wcap, D - wbase), top, neg, idx, ef, wbase, sticky);
}

// The finish of short accumulators (D <= ND digits, used up to 24) after the
// tensor-core CRT sums, R in registers: every group word and the quotient
// estimate are loaded at once (coalesced across the block), then
// R = (sum_g Q_g 2^(224 g) + alpha~ (2^(32 D) - P)) mod 2^(32 D), then the same
// unrolled steps as k_crt1 (crt_finish).  Group g holds 9 words starting at
// word 7 g, so word d collects word d - 7 g of group g = d / 7 and, for
// d mod 7 < 2, word d - 7 (g - 1) of the group before.
template <int ND>
__global__ void __launch_bounds__(kFinThreads, (ND <= 24 ? 6 : 1)) k_crt_fin_short(DevTables T, const int4* __restrict__ blk) {
  __shared__ uint32_t s_tab[3 * ND];              // 2^(32 ND) - P, 2^(32 ND) - floor(P/2) - 1, P
  __shared__ uint32_t s_mag[ND * kFinThreads];    // rounding scratch
  const int4 b = blk[blockIdx.x];
  const ProbDev& P = T.probs[b.x];
  const CrtView cv = crt_view(T.crt_pool, P);
  const int D = P.D32, ng = P.crt_ngrp;
  for (int i = threadIdx.x; i < ND; i += kFinThreads) {
    s_tab[i] = i < D ? __ldg(cv.negP + i) : ~0u;           // widened to ND digits (crt_finish)
    s_tab[ND + i] = i < D ? __ldg(cv.negH1 + i) : ~0u;
    s_tab[2 * ND + i] = i < D ? __ldg(cv.P + i) : 0u;
  }
  const int e = threadIdx.x;
  const int64_t idx = (int64_t)b.y * kFinThreads + e;
  const bool valid = idx < (int64_t)P.M * P.N;
  const int64_t up = P.upitch;
  const uint32_t* const qcol = P.crt_q + (valid ? idx : 0);

  uint32_t w0[ND], w1[ND];
#pragma unroll
  for (int d = 0; d < ND; ++d) {                   // independent loads first
    const int g = d / 7, k = d - 7 * g;
    w0[d] = (d < D && g < ng) ? __ldg(qcol + ((int64_t)g * 9 + k) * up) : 0u;
    w1[d] = (d < D && k < 2 && g >= 1 && g - 1 < ng) ? __ldg(qcol + ((int64_t)(g - 1) * 9 + k + 7) * up) : 0u;
  }
  const uint64_t alpha = __ldg(P.crt_alpha + (valid ? idx : 0));
  const int ef = valid ? crt_ef(P, idx) : 0;
  __syncthreads();
  if (!valid) return;
  uint32_t R[ND];
  uint64_t carry = 0;
#pragma unroll
  for (int d = 0; d < ND; ++d) {
    const uint64_t x = carry + alpha * s_tab[d] + w0[d] + w1[d];
    R[d] = d < D ? (uint32_t)x : 0u;
    carry = x >> 32;
  }
  crt_finish<ND>(P, R, s_tab, s_mag, kFinThreads, e, idx, ef, T.status);
}

// ---------------------------------------------------------------------------
// CRT sums of any length on the tensor cores (crt_mode 2).  As in k_crt_tc,
// S = sum_l v_l M_l = sum_j 128^j Y_j with Y = V B (K = 2L: the 7-bit halves
// of v_l; columns j: the 7-bit pieces of M_l), and every fp32 sum in TMEM is
// an exact integer below 2L 127^2 < 2^24 for L <= 520.  The plane GEMM
// already stored v_l = u_l M_l^{-1} mod m_l in place of u_l.
//
// Per tile of 128 consecutive outputs, V lives in tensor memory: TMEM lane r
// holds output r's row, column l the bf16 pair (v0_l, v1_l).  The columns of
// Y run in chunks of cw (a multiple of 32) through two TMEM accumulator slots
// after V (kpad / 2 + 2 cw <= 512), or through one slot when two would make
// the MMAs narrower than 128 columns; the B blocks (64 k x cw columns) stream
// through a shared-memory ring.  32 consecutive pieces span exactly 7 words,
// so group g of 32 columns is the integer
//   Q_g = sum_{q < 32} Y_{32 g + q} 2^(7 q),   S = sum_g Q_g 2^(224 g),
// with piece q in word 7 q / 32 at shift 7 q mod 32 (both constants); each
// Q_g is written on its own as 9 words (7 carried word sums and the carry),
// and the finish adds the groups and alpha~ (2^(32 D) - P).  With
// crt_gskip > 0 (the long finish, whose fast form reads no lower group) the
// columns start at 32 crt_gskip: the groups below are not formed, and stored
// group i is group crt_gskip + i.
//   warp 0      TMA producer of the B blocks, in (chunk, K block) order
//   warp 1      MMA issuer: chunks into the slots in turn (one slot: always
//               slot 0); commits per ring stage, per chunk and per tile
//   warp 2      TMA producer of the tile's v values, 32 moduli x 128 outputs
//               per copy, into a four-slot ring
//   warps 3-18  four threads per output (its TMEM lane), groups h = 0..3:
//               group h writes the V columns of the copies c = h mod 4 (in
//               pieces of 8 columns); then the tile's 32-column groups in
//               turn.  The last group's columns 27..31 are the sums of the
//               pieces of floor(2^28 / m_l): the quotient estimate
//               alpha~ = floor(sum_l v_l floor(2^28 / m_l) / 2^28), in
//               {alpha - 1, alpha}, written per output for the finish.
// A warp rewrites its V columns only after the commit that follows the
// previous tile's last MMA, and the next tile's MMAs wait for every warp's V
// columns (tcgen05.st waited and fenced), so V is never read and written at
// once; an accumulator slot is reused only after every worker has read it.
// Tile list entry: {problem, tile, 0, 0}.
// ---------------------------------------------------------------------------
constexpr int kCmWorkers = 512;
constexpr int kCmThreads = 96 + kCmWorkers;
constexpr int kCmMaxStages = 24;
constexpr int kCmUMods = 32;                         // moduli per v copy
constexpr int kCmUSlots = 4;
constexpr uint32_t kCmUBytes = kCmUMods * 128 * 2;   // [32][128] uint16
constexpr int kCmMinSmem = 116 * 1024;               // one CTA per SM: it holds all 512 TMEM columns

struct CmLayout {
  uint32_t ring_off, u_off, mu_off, bar_off, total;
  __host__ __device__ CmLayout(uint32_t stage_bytes, int stages, int lmax) {
    ring_off = 0;
    u_off = (uint32_t)stages * stage_bytes;
    mu_off = u_off + kCmUSlots * kCmUBytes;                 // floor(2^32 / m_l) [lmax]
    bar_off = mu_off + (((uint32_t)lmax * 4 + 15u) & ~15u);
    // barriers: full, empty [kCmMaxStages], u_full, u_free [kCmUSlots], acc_full, acc_free [2],
    // v_full, v_free [2], drain; then the abort flag and the TMEM slot
    total = 1024 + bar_off + (2 * kCmMaxStages + 2 * kCmUSlots + 9) * 8 + 16;
    if (total < (uint32_t)kCmMinSmem) total = kCmMinSmem;
  }
};

// exact integer value (< 2^24) of an fp32 holding one
__device__ __forceinline__ uint32_t f2u_exact24(uint32_t bits) {
  const float f = __uint_as_float(bits);
  return f >= 8388608.0f ? bits - 0x4A800000u : __float_as_uint(f + 8388608.0f) - 0x4B000000u;
}


// {bf16(v mod 128), bf16(floor(v / 128))} for v < 2^14 (low half, high half):
// 2^23 + x has x in its low mantissa bits; both halves are exact in bf16
__device__ __forceinline__ uint32_t bf16_halves7(uint32_t v) {
  const float f0 = __uint_as_float(0x4B000000u | (v & 127u)) - 8388608.0f;
  const float f1 = __uint_as_float(0x4B000000u | (v >> 7)) - 8388608.0f;
  uint32_t r;
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(f1), "f"(f0));
  return r;
}

// Add 32 pieces y[q] 2^(7 q) of one group into the 7 word accumulators.
template <int NQ>
__device__ __forceinline__ void crt_group(const uint32_t* y, uint64_t (&acc)[7]) {
#pragma unroll
  for (int q = 0; q < NQ; ++q) acc[(7 * q) >> 5] += (uint64_t)f2u_exact24(y[q]) << ((7 * q) & 31);
}

// sum over the pieces q < NQ in word w of 0x4B000000 2^(7 q mod 32)
template <int NQ>
__device__ __forceinline__ constexpr uint64_t crt_group_bias(int w) {
  uint64_t b = 0;
  for (int q = 0; q < NQ; ++q)
    if (((7 * q) >> 5) == w) b += 0x4B000000ull << ((7 * q) & 31);
  return b;
}

// The same for sums below 2^23 (2L 127^2 < 2^23): the bits of y + 2^23 are
// 0x4B000000 + y, one add per piece; the 0x4B000000 terms come off once per
// word (modulo 2^64, the true word sums fit).
template <int NQ>
__device__ __forceinline__ void crt_group_small(const uint32_t* y, uint64_t (&acc)[7]) {
#pragma unroll
  for (int q = 0; q < NQ; ++q)
    acc[(7 * q) >> 5] += (uint64_t)__float_as_uint(__uint_as_float(y[q]) + 8388608.0f) << ((7 * q) & 31);
#pragma unroll
  for (int w = 0; w < 7; ++w) acc[w] -= crt_group_bias<NQ>(w);
}

template <bool resident>
__global__ void __launch_bounds__(kCmThreads, 1)
    k_crt_mm(const __grid_constant__ DevTables T, const int4* __restrict__ tiles, int ntiles, uint32_t stage_bytes,
             int stages) {
  using namespace tc;
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  uint8_t* sm = smem_raw + (base - raw);
  const CmLayout lay(stage_bytes, stages, T.lmax);
  const uint32_t sRing = base + lay.ring_off;                 // B ring [stages][cw cols][128 B]
  const uint32_t sU = base + lay.u_off;                       // v ring [kCmUSlots][32][128] uint16
  uint64_t* bars = reinterpret_cast<uint64_t*>(sm + lay.bar_off);
  uint64_t* full = bars;                                      // [kCmMaxStages]
  uint64_t* empty = bars + kCmMaxStages;                      // [kCmMaxStages]
  uint64_t* u_full = bars + 2 * kCmMaxStages;                 // [kCmUSlots]
  uint64_t* u_free = u_full + kCmUSlots;                      // [kCmUSlots] (128 arrivals: one half)
  uint64_t* acc_full = u_free + kCmUSlots;                    // [2] chunk in slot done
  uint64_t* acc_free = acc_full + 2;                          // [2] slot read out (256 arrivals)
  uint64_t* v_full = acc_free + 2;                            // [2] V buffer written (every worker)
  uint64_t* v_free = v_full + 2;                              // [2] MMAs reading the buffer done
  uint64_t* drain = v_full + 4;                               // abort drain of the MMA pipe
  volatile int* abort_flag = reinterpret_cast<volatile int*>(v_full + 5);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(v_full + 5) + 1;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int i = 0; i < kCmMaxStages; ++i) {
      mbar_init(full + i, 1);
      mbar_init(empty + i, 1);
    }
    for (int i = 0; i < kCmUSlots; ++i) {
      mbar_init(u_full + i, 1);
      mbar_init(u_free + i, 128);
    }
    for (int i = 0; i < 2; ++i) mbar_init(acc_full + i, 1);
    for (int i = 0; i < 2; ++i) {
      mbar_init(v_full + i, kCmWorkers);
      mbar_init(v_free + i, 1);
    }
    for (int i = 0; i < 2; ++i) mbar_init(acc_free + i, kCmWorkers);   // every worker reads every chunk
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
    // ------------------------------------------------------------ B producer
    if (lane == 0) {
      int st = 0;
      uint32_t ph = 0;
      int issued_phase[kCmMaxStages];
      for (int i = 0; i < kCmMaxStages; ++i) issued_phase[i] = -1;
      bool ok = true;
      // resident table (one problem whose blocks all fit in the ring): each
      // block is loaded once, into stage c nkb + q, and read by every tile
      for (int i = blockIdx.x; ok && i < (resident ? min(ntiles, (int)blockIdx.x + 1) : ntiles); i += gridDim.x) {
        const int4 tl = tiles[i];
        const ProbDev& P = T.probs[tl.x];
        const CUtensorMap* mt = T.tmaps + 2 * T.count + tl.x;
        const int nkb = P.crt_kpad / 64, cw = P.crt_cw, nchunk = P.crt_nchunk, col0 = 32 * P.crt_gskip;
        for (int c = 0; ok && c < nchunk; ++c) {
          for (int q = 0; q < nkb; ++q) {
            if (!mbar_wait(empty + st, ph ^ 1u, abort_flag, T.status, T.spin_limit)) { ok = false; break; }
            mbar_expect_tx(full + st, (uint32_t)cw * 128u);
            tma_load_2d(sRing + st * stage_bytes, mt, smem_u32(full + st), q * 64, col0 + c * cw);
            issued_phase[st] = (int)ph;
            if (++st == stages) { st = 0; ph ^= 1u; }
          }
        }
      }
      if (!ok) {
        // let copies already in flight land before the CTA exits
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
      int next = 0, uses[2] = {0, 0}, vnext = 0, vuses[2] = {0, 0};
      bool ok = true, any = false;
      for (int i = blockIdx.x; ok && i < ntiles; i += gridDim.x) {
        const int4 tl = tiles[i];
        const bool first = i == (int)blockIdx.x;
        const ProbDev& P = T.probs[tl.x];
        const int nkb = P.crt_kpad / 64, cw = P.crt_cw, nchunk = P.crt_nchunk, npad = P.crt_npad - 32 * P.crt_gskip;
        const int nslot = P.crt_nslot, nvbuf = P.crt_nvbuf;
        const uint32_t vcols = (uint32_t)P.crt_kpad / 2;
        const int vb = nvbuf == 2 ? vnext : 0, vuse = vuses[vb]++;
        vnext = nvbuf == 2 ? vnext ^ 1 : 0;
        if (!mbar_wait(v_full + vb, (uint32_t)(vuse & 1), abort_flag, T.status, T.spin_limit)) { ok = false; break; }
        tc_fence_after();
        const uint32_t vbase = tmem + (uint32_t)vb * vcols;
        for (int c = 0; ok && c < nchunk; ++c) {
          const int s = nslot == 2 ? next : 0, use = uses[s]++;
          next = nslot == 2 ? next ^ 1 : 0;
          if (use > 0 && !mbar_wait(acc_free + s, (uint32_t)((use - 1) & 1), abort_flag, T.status, T.spin_limit)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const int ncol = min(cw, npad - c * cw);             // a multiple of 16
          const uint32_t idesc = idesc_bf16(128, ncol);
          const uint32_t d = tmem + (uint32_t)nvbuf * vcols + (uint32_t)(s * cw);
          for (int q = 0; q < nkb; ++q) {
            if (resident) st = c * nkb + q;
            if ((!resident || first) && !mbar_wait(full + st, resident ? 0u : ph, abort_flag, T.status, T.spin_limit)) {
              ok = false;
              break;
            }
            tc_fence_after();
            const uint64_t db = desc_sw128(sRing + st * stage_bytes);
#pragma unroll
            for (int kk = 0; kk < 4; ++kk)
              umma_bf16_ta(d, vbase + (uint32_t)(32 * q + 8 * kk), db + 2 * kk, idesc, (q | kk) ? 1u : 0u);
            any = true;
            if (!resident) {
              umma_commit(empty + st);
              if (++st == stages) { st = 0; ph ^= 1u; }
            }
          }
          if (ok) umma_commit(acc_full + s);
        }
        if (!ok) break;
        umma_commit(v_free + vb);
      }
      if (!ok && any) {
        // drain issued MMAs before TMEM is released
        umma_commit(drain);
        for (uint32_t t = 0; t < kSpinLimit && !mbar_try_wait(drain, 0u); ++t) {}
      }
    }
  } else if (warp == 2) {
    // ------------------------------------------------------------ v producer
    if (lane == 0) {
      int uc = 0;
      int issued_phase[kCmUSlots];
      for (int i = 0; i < kCmUSlots; ++i) issued_phase[i] = -1;
      bool ok = true;
      for (int i = blockIdx.x; ok && i < ntiles; i += gridDim.x) {
        const int4 tl = tiles[i];
        const ProbDev& P = T.probs[tl.x];
        const CUtensorMap* mu_ = T.tmaps + 3 * T.count + tl.x;
        const int L = P.L;
        for (int l0 = 0; l0 < L; l0 += kCmUMods, ++uc) {
          const int s = uc % kCmUSlots, use = uc / kCmUSlots;
          if (use > 0 && !mbar_wait(u_free + s, (uint32_t)((use - 1) & 1), abort_flag, T.status, T.spin_limit)) {
            ok = false;
            break;
          }
          mbar_expect_tx(u_full + s, kCmUBytes);
          tma_load_2d(sU + s * kCmUBytes, mu_, smem_u32(u_full + s), tl.y * 128, l0);
          issued_phase[s] = use & 1;
        }
      }
      if (!ok)
        for (int s = 0; s < kCmUSlots; ++s)
          if (issued_phase[s] >= 0)
            for (uint32_t t = 0; t < kSpinLimit && !mbar_try_wait(u_full + s, (uint32_t)issued_phase[s]); ++t) {}
    }
  } else {
    // ------------------------------------------------------------ V columns + chunk epilogues
    const int wk = warp - 3;
    const int half = wk >> 2;                         // worker group 0..3
    const int quad = warp & 3;
    const int row = quad * 32 + lane;
    const uint32_t tlane = tmem + ((uint32_t)(quad * 32) << 16);
    const uint16_t* s_u = reinterpret_cast<const uint16_t*>(sm + lay.u_off);
    int next = 0, uses[2] = {0, 0}, uc = 0, vnext = 0, vuses[2] = {0, 0}, ecount = 0;
    bool ok = true;
    // V of tile i into its buffer: the group's v copies (c = h mod 4) as bf16
    // 7-bit halves, and the group's part of the quotient sum
    auto build = [&](int i) {
      const int4 tl = tiles[i];
      const ProbDev& P = T.probs[tl.x];
      // the problem's fields in registers before the waits (their memory
      // clobbers would reload them from global memory after every barrier)
      const int L = P.L, nvbuf = P.crt_nvbuf;
      const uint32_t vcols = (uint32_t)P.crt_kpad / 2;
      const int vb = nvbuf == 2 ? vnext : 0, vuse = vuses[vb]++;
      vnext = nvbuf == 2 ? vnext ^ 1 : 0;
      // the buffer may be rewritten once every MMA of its previous tile is done
      if (vuse > 0 && ok) ok = mbar_wait(v_free + vb, (uint32_t)((vuse - 1) & 1), abort_flag, T.status, T.spin_limit);
      ok = __all_sync(0xffffffffu, ok);
      if (!ok) return;
      tc_fence_after();
      const uint32_t vrow = tlane + (uint32_t)vb * vcols;
      for (int l0 = 0; l0 < L; l0 += kCmUMods, ++uc) {
        if ((uc & 3) != half) continue;             // another group's copy
        const int s = uc % kCmUSlots, use = uc / kCmUSlots;
        if (ok) ok = mbar_wait(u_full + s, (uint32_t)(use & 1), abort_flag, T.status, T.spin_limit);
        ok = __all_sync(0xffffffffu, ok);
        if (!ok) return;
        const uint16_t* su = s_u + s * (kCmUMods * 128);
        // pieces of 8 moduli in a rolled loop (small code), V columns
        // l0 + 8 pc .. + 7 (zero beyond L)
#pragma unroll 1
        for (int pc = 0; pc < kCmUMods; pc += 8) {
          const int lp = l0 + pc;
          uint32_t pr[8];
          if (lp + 8 <= L) {                          // a full piece: no bounds
#pragma unroll
            for (int j = 0; j < 8; ++j) pr[j] = bf16_halves7(su[(pc + j) * 128 + row]);
          } else {
#pragma unroll
            for (int j = 0; j < 8; ++j) {
              const int l = lp + j;
              pr[j] = bf16_halves7(l < L ? (uint32_t)su[(pc + j) * 128 + row] : 0u);
            }
          }
          tmem_st8(vrow + (uint32_t)lp, pr);
        }
        mbar_arrive(u_free + s);
      }
      tmem_wait_st();
      tc_fence_before();
      mbar_arrive(v_full + vb);
    };
    // chunk epilogues of tile i: the tile's 32-column groups in turn over the
    // four groups (rotated per tile)
    auto epilogue = [&](int i) {
      const int4 tl = tiles[i];
      const ProbDev& P = T.probs[tl.x];
      // columns from 32 crt_gskip on (the groups below are not formed); the
      // group sums are stored from that group on
      const int cw = P.crt_cw, nchunk = P.crt_nchunk, npad = P.crt_npad - 32 * P.crt_gskip, nslot = P.crt_nslot;
      const uint32_t acc0 = (uint32_t)P.crt_nvbuf * ((uint32_t)P.crt_kpad / 2);
      const bool small = 2 * P.L * 127 * 127 < (1 << 23);   // every column sum below 2^23
      const int64_t idx = (int64_t)tl.y * 128 + row;
      const bool valid = idx < (int64_t)P.M * P.N;
      const int64_t up = P.upitch;
      uint32_t* const qbase = P.crt_q;
      for (int c = 0; c < nchunk; ++c) {
        const int s = nslot == 2 ? next : 0, use = uses[s]++;
        next = nslot == 2 ? next ^ 1 : 0;
        if (ok) ok = mbar_wait(acc_full + s, (uint32_t)(use & 1), abort_flag, T.status, T.spin_limit);
        ok = __all_sync(0xffffffffu, ok);
        if (!ok) return;
        tc_fence_after();
        const uint32_t trow = tlane + acc0 + (uint32_t)(s * cw);
        const int ncol = min(cw, npad - c * cw);             // columns written by the MMAs
        const int gfirst = (half - c * (cw >> 5) - ecount) & 3;
        for (int g = 32 * gfirst; g < cw; g += 128) {
          uint64_t acc[7] = {0, 0, 0, 0, 0, 0, 0};
          if (g < ncol) {
            uint32_t y[32];
            if (g + 32 <= ncol) {
              tmem_ld32(trow + (uint32_t)g, y);
            } else {                                  // 16 columns left: the rest are zero pieces
              uint32_t y16[16];
              tmem_ld16(trow + (uint32_t)g, y16);
#pragma unroll
              for (int q = 0; q < 16; ++q) y[q] = y16[q];
#pragma unroll
              for (int q = 16; q < 32; ++q) y[q] = 0u;
            }
            if (c * cw + g + 32 == npad) {
              // the last group's columns 27..31 hold sum_k 128^k Y = sum_l v_l
              // floor(2^28 / m_l): alpha~ = floor of it / 2^28, in {alpha - 1,
              // alpha} (its error is below L 2^14 / 2^28); then they are cleared
              uint64_t a = 0;
#pragma unroll
              for (int k = 4; k >= 0; --k) a = (a << 7) + f2u_exact24(y[27 + k]);
              if (valid) P.crt_alpha[idx] = (uint32_t)(a >> 28);
#pragma unroll
              for (int k = 27; k < 32; ++k) y[k] = 0u;
            }
            if (small) crt_group_small<32>(y, acc);
            else crt_group<32>(y, acc);
          }
          // group sum as 9 words: 7 word sums with carries, then the carry
          uint32_t* qcol = qbase + (int64_t)((c * cw + g) >> 5) * 9 * up + (valid ? idx : 0);
          uint64_t carry = 0;
#pragma unroll
          for (int k = 0; k < 7; ++k) {
            const uint64_t x = acc[k] + carry;
            if (valid) qcol[(int64_t)k * up] = (uint32_t)x;
            carry = x >> 32;
          }
          if (valid) {
            qcol[(int64_t)7 * up] = (uint32_t)carry;
            qcol[(int64_t)8 * up] = (uint32_t)(carry >> 32);
          }
        }
        tc_fence_before();
        mbar_arrive(acc_free + s);
      }
      ++ecount;
    };
    // With two V buffers (uniform within a launch) the next tile's V is built
    // before this tile's chunks are read, so its MMAs overlap the epilogue;
    // that order waits for the MMAs of the tile before this one only.  With
    // one buffer it would wait for this tile's MMAs, whose later chunks wait
    // for this tile's epilogue: tiles then go strictly in turn.
    const bool two = blockIdx.x < ntiles && T.probs[tiles[blockIdx.x].x].crt_nvbuf == 2;
    if (two && blockIdx.x < ntiles) build(blockIdx.x);
    for (int i = blockIdx.x; ok && i < ntiles; i += gridDim.x) {
      if (!two) build(i);
      else if (i + (int)gridDim.x < ntiles) build(i + gridDim.x);
      if (!ok) break;
      epilogue(i);
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

template <int ND>
cudaError_t crt_tc_attr() {
  return cudaFuncSetAttribute(k_crt_tc<ND>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
}

}  // namespace

int crt_tc_smem_bytes(int cls, int kpad, int npad, int lmax, int /*nbuf*/) {
  return (int)CtLayout(kCrtClasses[cls].dpl, kpad, npad, lmax).total;
}

cudaError_t launch_crt_tc(const DevTables& t, int cls, const int32_t* tiles, int ntiles, int kpad_max,
                          int npad_max, int lmax, int grid, cudaStream_t s) {
  if (ntiles == 0) return cudaSuccess;
  const int smem = crt_tc_smem_bytes(cls, kpad_max, npad_max, lmax, 2);
  const int4* tl = reinterpret_cast<const int4*>(tiles);
  const int sms = grid;
  switch (cls) {
#define OZ2_CRT_TC(i, nd)                                                                              \
  case i: {                                                                                           \
    int per_sm = 1;                                                                                   \
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_crt_tc<nd>, kCtThreads, smem) != cudaSuccess) \
      per_sm = 1;                                                                                     \
    per_sm = per_sm < 1 ? 1 : per_sm;                                                                 \
    const int cap = 512 / (2 * crt_tc_tmem_cols(npad_max));                                           \
    per_sm = per_sm > cap ? cap : per_sm;                                                             \
    const int g = ntiles < sms * per_sm ? ntiles : sms * per_sm;                                      \
    k_crt_tc<nd><<<g, kCtThreads, smem, s>>>(t, tl, ntiles, kpad_max, npad_max, lmax);                \
    break;                                                                                            \
  }
    OZ2_CRT_TC(0, 8) OZ2_CRT_TC(1, 12) OZ2_CRT_TC(2, 16) OZ2_CRT_TC(3, 20) OZ2_CRT_TC(4, 24)
    OZ2_CRT_TC(5, 28) OZ2_CRT_TC(6, 32) OZ2_CRT_TC(7, 36) OZ2_CRT_TC(8, 40)
#undef OZ2_CRT_TC
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// Chunk width of the tensor-core CRT sums: columns of Y per TMEM slot, a
// multiple of 32, with V (kpad / 2 columns) and one or two slots within 512
// columns.
int crt_mm_chunk(int kpad, int npad, int* nslot) {
  // two slots (the epilogue of one chunk overlaps the MMAs of the next)
  // unless that leaves chunks narrower than 128 columns: one slot then, for
  // MMAs of N >= 128 (narrow MMAs cost as much to issue as they compute)
  const int need = (npad + 31) & ~31;
  int cw2 = ((512 - kpad / 2) / 2) & ~31;
  cw2 = cw2 > 256 ? 256 : cw2;
  if (cw2 >= 128 || cw2 >= need) {
    if (nslot) *nslot = 2;
    return cw2 < need ? cw2 : need;
  }
  int cw1 = (512 - kpad / 2) & ~31;
  cw1 = cw1 > 256 ? 256 : cw1;
  if (nslot) *nslot = 1;
  return cw1 < need ? cw1 : need;
}

int crt_mm_smem_bytes(int cw_max, int lmax, int* stages) {
  // the deepest B ring (2 to kCmMaxStages stages of cw_max columns) that fits
  const uint32_t sb = (uint32_t)cw_max * 128u;
  for (int st = kCmMaxStages; st >= 2; --st) {
    const int bytes = (int)CmLayout(sb, st, lmax).total;
    if (bytes <= 227 * 1024) {
      if (stages) *stages = st;
      return bytes;
    }
  }
  if (stages) *stages = 0;
  return -1;
}

// blocks_one: the table blocks of a tile (K blocks x chunks) when every tile
// of the launch belongs to one problem, else 0; where they fit in the ring
// the table stays resident (loaded once per CTA).
cudaError_t launch_crt_mm(const DevTables& t, const int32_t* tiles, int ntiles, int cw_max, int grid,
                          int blocks_one, cudaStream_t s) {
  if (ntiles == 0) return cudaSuccess;
  int stages = 0;
  const int smem = crt_mm_smem_bytes(cw_max, t.lmax, &stages);
  if (smem < 0) return cudaErrorInvalidValue;
  const int g = ntiles < grid ? ntiles : grid;
  const int4* tl = reinterpret_cast<const int4*>(tiles);
  if (blocks_one > 0 && blocks_one <= stages)
    k_crt_mm<true><<<g, kCmThreads, smem, s>>>(t, tl, ntiles, (uint32_t)cw_max * 128u, stages);
  else
    k_crt_mm<false><<<g, kCmThreads, smem, s>>>(t, tl, ntiles, (uint32_t)cw_max * 128u, stages);
  return cudaGetLastError();
}

// tables (three of up to dmax + 6 digits) and the window of 2 nl + 10 digits
// per output (2 nl + 4, and six more for the fast form's window)
int crt_finish_long_smem(int dmax, int nlmax) { return 3 * (dmax + 6) * 4 + (2 * nlmax + 10) * kFinThreads * 4; }

cudaError_t launch_crt_finish_long(const DevTables& t, const int32_t* blk, int nblk, int dmax, int nlmax,
                                   cudaStream_t s) {
  if (nblk == 0) return cudaSuccess;
  const int smem = crt_finish_long_smem(dmax, nlmax);
  k_crt_fin_long<<<nblk, kFinThreads, smem, s>>>(t, reinterpret_cast<const int4*>(blk));
  return cudaGetLastError();
}

cudaError_t launch_crt_fin_short(const DevTables& t, int cls, const int32_t* blk, int nblk, cudaStream_t s) {
  if (nblk == 0) return cudaSuccess;
  const int4* bl = reinterpret_cast<const int4*>(blk);
  switch (cls) {
    case 0: k_crt_fin_short<8><<<nblk, kFinThreads, 0, s>>>(t, bl); break;
    case 1: k_crt_fin_short<12><<<nblk, kFinThreads, 0, s>>>(t, bl); break;
    case 2: k_crt_fin_short<16><<<nblk, kFinThreads, 0, s>>>(t, bl); break;
    case 3: k_crt_fin_short<20><<<nblk, kFinThreads, 0, s>>>(t, bl); break;
    case 4: k_crt_fin_short<24><<<nblk, kFinThreads, 0, s>>>(t, bl); break;
    case 5: k_crt_fin_short<28><<<nblk, kFinThreads, 0, s>>>(t, bl); break;
    case 6: k_crt_fin_short<32><<<nblk, kFinThreads, 0, s>>>(t, bl); break;
    case 7: k_crt_fin_short<36><<<nblk, kFinThreads, 0, s>>>(t, bl); break;
    case 8: k_crt_fin_short<40><<<nblk, kFinThreads, 0, s>>>(t, bl); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t init_crt_attributes() {
  cudaError_t e = cudaFuncSetAttribute(k_crt_mm<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_crt_mm<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_crt_fin_long, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  if (e == cudaSuccess) e = crt1_attr<8>();
  if (e == cudaSuccess) e = crt1_attr<12>();
  if (e == cudaSuccess) e = crt1_attr<16>();
  if (e == cudaSuccess) e = crt1_attr<20>();
  if (e == cudaSuccess) e = crt1_attr<24>();
  if (e == cudaSuccess) e = crt1_attr<28>();
  if (e == cudaSuccess) e = crt1_attr<32>();
  if (e == cudaSuccess) e = crt1_attr<36>();
  if (e == cudaSuccess) e = crt1_attr<40>();
  if (e == cudaSuccess) e = crt_tc_attr<8>();
  if (e == cudaSuccess) e = crt_tc_attr<12>();
  if (e == cudaSuccess) e = crt_tc_attr<16>();
  if (e == cudaSuccess) e = crt_tc_attr<20>();
  if (e == cudaSuccess) e = crt_tc_attr<24>();
  if (e == cudaSuccess) e = crt_tc_attr<28>();
  if (e == cudaSuccess) e = crt_tc_attr<32>();
  if (e == cudaSuccess) e = crt_tc_attr<36>();
  if (e == cudaSuccess) e = crt_tc_attr<40>();
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
