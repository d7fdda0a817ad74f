// Complex products in 3M form in the residue domain (the paper's Sec. 11
// lists complex 3M/4M products as future work).  C = (Ar + i Ai)(Br + i Bi)
// runs as a plan of three real products that share one row exponent e_i
// (over Ar and Ai) and one column exponent f_j (over Br and Bi):
//   product 0: Ar Br      (its C is Cr)
//   product 1: Ai Bi      (its C is Ci)
//   product 2: (Ar + Ai)(Br + Bi), whose residue planes are the sums of the
//              first two products' planes (k_plane_sum) and which has no CRT.
// After the plane GEMMs, k_combine_complex forms v_r = v_0 - v_1 and
// v_i = v_2 - v_0 - v_1 mod m_l (v_l = u_l M_l^{-1} mod m_l is linear in u_l)
// in products 0 and 1, whose CRT then gives Cr and Ci.  Three plane products
// per modulus instead of four.
#include "oz2_internal.h"

namespace oz2 {

namespace {

__device__ __forceinline__ int bf_int(uint32_t h) { return (int)__uint_as_float(h << 16); }
__device__ __forceinline__ uint32_t int_bf(int x) { return __float_as_uint((float)x) >> 16; }

// centered residue of a + b for centered a, b of modulus m: in (-m/2, m/2]
__device__ __forceinline__ int cen_add(int a, int b, int m) {
  int r = a + b;
  if (2 * r > m) r -= m;
  if (2 * r <= -m) r += m;
  return r;
}

// Residue planes of the sums Ar + Ai (side 0) and Br + Bi (side 1): one thread
// per (side, modulus, line, 8 consecutive k).  One-limb planes add directly;
// a two-limb residue is rebuilt from its balanced halves r0 + 128 r1 (planes
// g, g + 1), added, centered and split again into r0, r1, r0 + r1.
__global__ void __launch_bounds__(256) k_plane_sum(const __grid_constant__ DevTables T, int64_t items_a,
                                                   int64_t items_b) {
  const int64_t it = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (it >= items_a + items_b) return;
  const ProbDev& P0 = T.probs[0];
  const ProbDev& P1 = T.probs[1];
  const ProbDev& P2 = T.probs[2];
  const int side = it >= items_a;
  const int64_t local = side ? it - items_a : it;
  const int R = side ? P0.N : P0.M;
  const int kc = P0.Kp / 8;
  const int64_t per_l = (int64_t)R * kc;
  const int l = (int)(local / per_l);
  const int64_t rem = local - (int64_t)l * per_l;
  const int line = (int)(rem / kc), k8 = (int)(rem - (int64_t)line * kc);
  const int m = (int)T.mods[l].m;
  const bool two = l >= P0.L1;
  const int g = two ? P0.L1 + 3 * (l - P0.L1) : l;
  const int64_t ps = (int64_t)R * P0.Kp;
  const int64_t off = (int64_t)g * ps + (int64_t)line * P0.Kp + 8 * k8;
  const uint16_t* a = (side ? P0.pb : P0.pa) + off;
  const uint16_t* b = (side ? P1.pb : P1.pa) + off;
  uint16_t* c = (side ? P2.pb : P2.pa) + off;
  const uint4 a0 = *reinterpret_cast<const uint4*>(a);
  const uint4 b0 = *reinterpret_cast<const uint4*>(b);
  const uint32_t* aw0 = reinterpret_cast<const uint32_t*>(&a0);
  const uint32_t* bw0 = reinterpret_cast<const uint32_t*>(&b0);
  if (!two) {
    uint4 o;
    uint32_t* ow = reinterpret_cast<uint32_t*>(&o);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int lo = cen_add(bf_int(aw0[q] & 0xffffu), bf_int(bw0[q] & 0xffffu), m);
      const int hi = cen_add(bf_int(aw0[q] >> 16), bf_int(bw0[q] >> 16), m);
      ow[q] = int_bf(lo) | (int_bf(hi) << 16);
    }
    *reinterpret_cast<uint4*>(c) = o;
    return;
  }
  const uint4 a1 = *reinterpret_cast<const uint4*>(a + ps);
  const uint4 b1 = *reinterpret_cast<const uint4*>(b + ps);
  const uint32_t* aw1 = reinterpret_cast<const uint32_t*>(&a1);
  const uint32_t* bw1 = reinterpret_cast<const uint32_t*>(&b1);
  uint4 o0, o1, os;
  uint32_t* w0 = reinterpret_cast<uint32_t*>(&o0);
  uint32_t* w1 = reinterpret_cast<uint32_t*>(&o1);
  uint32_t* wsum = reinterpret_cast<uint32_t*>(&os);
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    uint32_t r0w = 0, r1w = 0, rsw = 0;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int sh = 16 * h;
      const int ra = bf_int((aw0[q] >> sh) & 0xffffu) + 128 * bf_int((aw1[q] >> sh) & 0xffffu);
      const int rb = bf_int((bw0[q] >> sh) & 0xffffu) + 128 * bf_int((bw1[q] >> sh) & 0xffffu);
      const int r = cen_add(ra, rb, m);
      const int y = r & 127;                     // r mod 128 in [0, 128)
      const int r0 = y > 64 ? y - 128 : y;       // balanced split: r0 in (-64, 64]
      const int r1 = (r - r0) / 128;
      r0w |= int_bf(r0) << sh;
      r1w |= int_bf(r1) << sh;
      rsw |= int_bf(r0 + r1) << sh;
    }
    w0[q] = r0w;
    w1[q] = r1w;
    wsum[q] = rsw;
  }
  *reinterpret_cast<uint4*>(c) = o0;
  *reinterpret_cast<uint4*>(c + ps) = o1;
  *reinterpret_cast<uint4*>(c + 2 * ps) = os;
}

// v_r = v_0 - v_1 and v_i = v_2 - v_0 - v_1 (mod m_l), written over v_0 and
// v_1: one thread per (modulus, 8 consecutive outputs).
__global__ void __launch_bounds__(256) k_combine_complex(const __grid_constant__ DevTables T, int64_t items) {
  const int64_t it = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (it >= items) return;
  const ProbDev& P0 = T.probs[0];
  const ProbDev& P1 = T.probs[1];
  const ProbDev& P2 = T.probs[2];
  const int64_t per_l = P0.upitch / 8;
  const int l = (int)(it / per_l);
  const int64_t off = (int64_t)l * P0.upitch + 8 * (it - (int64_t)l * per_l);
  const uint32_t m = T.mods[l].m;
  const uint4 x = *reinterpret_cast<const uint4*>(P0.u + off);
  const uint4 y = *reinterpret_cast<const uint4*>(P1.u + off);
  const uint4 z = *reinterpret_cast<const uint4*>(P2.u + off);
  const uint32_t* xw = reinterpret_cast<const uint32_t*>(&x);
  const uint32_t* yw = reinterpret_cast<const uint32_t*>(&y);
  const uint32_t* zw = reinterpret_cast<const uint32_t*>(&z);
  uint4 vr, vi;
  uint32_t* rw = reinterpret_cast<uint32_t*>(&vr);
  uint32_t* iw = reinterpret_cast<uint32_t*>(&vi);
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    uint32_t rr = 0, ii = 0;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int sh = 16 * h;
      const uint32_t v0 = (xw[q] >> sh) & 0xffffu, v1 = (yw[q] >> sh) & 0xffffu, v2 = (zw[q] >> sh) & 0xffffu;
      uint32_t r = v0 + m - v1;                  // in [1, 2m)
      r = r >= m ? r - m : r;
      uint32_t i = v2 + 2 * m - v0 - v1;         // in [1, 3m)
      i = i >= m ? i - m : i;
      i = i >= m ? i - m : i;
      rr |= r << sh;
      ii |= i << sh;
    }
    rw[q] = rr;
    iw[q] = ii;
  }
  *reinterpret_cast<uint4*>(P0.u + off) = vr;
  *reinterpret_cast<uint4*>(P1.u + off) = vi;
}

}  // namespace

cudaError_t launch_plane_sum(const DevTables& t, int64_t items_a, int64_t items_b, cudaStream_t s) {
  const int64_t n = items_a + items_b;
  if (n == 0) return cudaSuccess;
  k_plane_sum<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(t, items_a, items_b);
  return cudaGetLastError();
}

cudaError_t launch_combine_complex(const DevTables& t, int64_t items, cudaStream_t s) {
  if (items == 0) return cudaSuccess;
  k_combine_complex<<<(unsigned)((items + 255) / 256), 256, 0, s>>>(t, items);
  return cudaGetLastError();
}

}  // namespace oz2
