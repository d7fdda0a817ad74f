// Pieces shared by the plane GEMM kernels (one SM per 128 x 256 tile, and a
// CTA pair per 256 x 256 tile): the exact reductions of the epilogue and the
// deterministic job order that the producer, MMA and epilogue roles walk.
#pragma once

#include <cstdint>

#include "oz2_internal.h"
#include "tc_ptx.cuh"

namespace oz2 {
namespace plane {

__device__ __forceinline__ uint32_t barrett32(uint32_t x, uint32_t m, uint32_t mu) {
  uint32_t q = __umulhi(x, mu);
  uint32_t r = x - q * m;
  return r >= m ? r - m : r;
}

// x: exact integer held in fp32 with |x| < 2^25.  Returns x mod m in [0, m).
// q = rint(x * rcp) is within 0.52 of x/m, so r = x - q m lies in
// (-0.52 m, 0.52 m) and is computed exactly by the fma; one correction
// brings it into [0, m).
__device__ __forceinline__ uint32_t fmod_small(float x, float mf, float rcp) {
  const float q = rintf(x * rcp);
  float r = fmaf(-q, mf, x);
  r = r < 0.f ? r + mf : r;
  // exact float -> int of 0 <= r < 2^23 without a conversion instruction
  return __float_as_uint(r + 8388608.0f) - 0x4B000000u;
}

// exact int -> float of 0 <= x < 2^23 without a conversion instruction
__device__ __forceinline__ float small_u2f(uint32_t x) {
  return __uint_as_float(0x4B000000u + x) - 8388608.0f;
}

// One accumulation job: plane `plane` of unit `u` over K chunk `chunk`.
struct Job {
  Unit u;
  int slot;
  int plane;
  int chunk;
  bool first;       // first job of the unit: the MMA overwrites the slot
  bool last;        // last job of the unit: the epilogue writes u_l
  uint32_t kmul;    // write-back multiplier (not last)
};

// Deterministic job order shared by the producer, MMA and epilogue roles:
// units s, s+2, s+4, ... of the CTA's list go to TMEM slot s, and the jobs of
// the two slot streams alternate.
struct JobIter {
  const DevTables* T;
  int ubeg, n;
  int uidx[2], job[2], turn;

  __device__ void init(const DevTables* t, int b, int e) {
    T = t; ubeg = b; n = e - b;
    uidx[0] = 0; uidx[1] = 1; job[0] = job[1] = 0; turn = 0;
  }
  __device__ bool next(Job& j) {
    int s = turn;
    if (uidx[s] >= n) {
      s ^= 1;
      if (uidx[s] >= n) return false;
    }
    const Unit u = T->units[ubeg + uidx[s]];
    const ProbDev& P = T->probs[u.prob];
    const bool two = u.ell >= P.L1;
    const int nch = P.nchunks;
    const int njobs = (two ? 3 : 1) * nch;
    const int jj = job[s];
    const int pi = jj / nch;
    j.u = u;
    j.slot = s;
    j.chunk = jj - pi * nch;
    if (two) {
      const int g0 = P.L1 + 3 * (u.ell - P.L1);
      j.plane = g0 + (pi == 0 ? 0 : (pi == 1 ? 2 : 1));   // P0, Ps, P2
    } else {
      j.plane = u.ell;
    }
    j.first = jj == 0;
    j.last = jj == njobs - 1;
    j.kmul = 1u;
    if (!j.last && j.chunk == nch - 1) {
      const ModConst& mc = T->mods[u.ell];
      j.kmul = pi == 0 ? mc.kmul01 : mc.kmul12;
    }
    if (++job[s] == njobs) {
      job[s] = 0;
      uidx[s] += 2;
    }
    turn = s ^ 1;
    return true;
  }
};

// Debugging aid: the exact sum of each plane product before any reduction,
// when K fits in one accumulation chunk.  A job's accumulator holds its
// plane's sum plus the value the unit's previous job wrote back; that job
// leaves the written-back value in this plane's debug slot, so
// dbg_plane_sums subtracts it, and dbg_write_back leaves the current job's
// for the next plane (Karatsuba order P0, Ps, P2 = planes g0, g0 + 2, g0 + 1).
// Both read the 32 columns at taddr from tensor memory themselves (whole warp)
// and are kept out of line, so that the epilogue's registers and code stay as
// they are when no dump is asked for.
static __device__ __noinline__ void dbg_plane_sums(int32_t* dbg, int plane, bool first, int M, int N, int row,
                                                   int col0, uint32_t taddr) {
  uint32_t v[32];
  tc::tmem_ld32(taddr, v);
  if (row >= M) return;
  int32_t* d = dbg + ((int64_t)plane * M + row) * N + col0;
  for (int i = 0; i < 32 && col0 + i < N; ++i) {
    const int32_t acc = __float2int_rn(__uint_as_float(v[i]));
    d[i] = first ? acc : acc - d[i];
  }
}
static __device__ __noinline__ void dbg_write_back(int32_t* dbg, int plane, int ell, int L1, int M, int N,
                                                   int row, int col0, uint32_t taddr) {
  uint32_t v[32];
  tc::tmem_wait_st();
  tc::tmem_ld32(taddr, v);
  if (row >= M || ell < L1) return;
  const int g0 = L1 + 3 * (ell - L1);
  const int next = plane == g0 ? g0 + 2 : g0 + 1;
  int32_t* d = dbg + ((int64_t)next * M + row) * N + col0;
  for (int i = 0; i < 32 && col0 + i < N; ++i) d[i] = __float2int_rn(__uint_as_float(v[i]));
}

}  // namespace plane
}  // namespace oz2
