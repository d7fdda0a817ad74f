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

// A job's epilogue constants, gathered before its accumulator is ready (the
// loads run while the epilogue waits for the slot; the chunk loop then reads
// no global memory but the optional debug dump).
struct EpiConst {
  float mf, rcp;
  uint32_t m, mu;
  uint32_t mul;       // write-back: the next plane's Karatsuba factor; last job:
                      // kfin M_l^{-1} mod m_l, so that the stored value is the
                      // CRT's v_l = (c mod m_l) M_l^{-1} mod m_l (Sec. 4.4)
  int M, N, row, col0, L1, ell;
  uint16_t* urow;     // u of this modulus, row `row`
  int32_t* dbg;
  bool vec_ok;        // rows of u start 16-byte aligned
};

// v_l tiles of one epilogue warp through shared memory: two 2 KB buffers of
// 32 rows x 64 bytes in the 64-byte swizzle (16-byte chunk q of row r at
// r 64 + 16 (q ^ ((r >> 1) & 3)): the eight rows of a store phase hit eight
// different bank groups), each written to u by one TMA store.  map is null
// when u's rows are not 16-byte multiples; then every thread stores its row.
struct UStage {
  const CUtensorMap* map;
  uint32_t sbuf;      // shared address of the warp's two buffers
  uint32_t n;         // tiles staged so far (warp-uniform)
};

__device__ __forceinline__ EpiConst epi_const(const DevTables& T, const Job& j, int row, int col0) {
  const ProbDev& P = T.probs[j.u.prob];
  const ModConst mc = T.mods[j.u.ell];
  EpiConst e;
  e.mf = (float)mc.m;
  e.rcp = mc.rcp;
  e.m = mc.m;
  e.mu = mc.mu;
  e.M = P.M;
  e.N = P.N;
  e.row = row;
  e.col0 = col0;
  e.L1 = P.L1;
  e.ell = j.u.ell;
  e.urow = P.u + (int64_t)j.u.ell * P.upitch + (int64_t)row * P.N;
  e.dbg = P.dbg_prods;
  e.vec_ok = (P.N & 7) == 0;
  e.mul = j.last ? barrett32(mc.kfin * __ldg(crt_view(T.crt_pool, P).Minv + j.u.ell), mc.m, mc.mu) : j.kmul;
  return e;
}

// One 32-column chunk of a job's accumulator (v, read from taddr; columns
// e.col0 + cc ..): reduce mod m, then either write the residue back into
// TMEM times the next plane's factor, or store v_l.
__device__ __forceinline__ void epi_chunk(const Job& j, const EpiConst& e, uint32_t (&v)[32], uint32_t taddr,
                                          int cc, UStage& us) {
  const int col = e.col0 + cc;
  if (e.dbg != nullptr) dbg_plane_sums(e.dbg, j.plane, j.first, e.M, e.N, e.row, col, taddr);
  if (!j.last) {
#pragma unroll
    for (int i = 0; i < 32; ++i) {
      uint32_t r = fmod_small(__uint_as_float(v[i]), e.mf, e.rcp);
      if (e.mul != 1u) r = barrett32(r * e.mul, e.m, e.mu);
      v[i] = __float_as_uint(small_u2f(r));
    }
    tc::tmem_st32(taddr, v);
    if (e.dbg != nullptr) dbg_write_back(e.dbg, j.plane, j.u.ell, e.L1, e.M, e.N, e.row, col, taddr);
    return;
  }
#pragma unroll
  for (int i = 0; i < 32; ++i) {
    uint32_t r = fmod_small(__uint_as_float(v[i]), e.mf, e.rcp);
    if (e.mul != 1u) r = barrett32(r * e.mul, e.m, e.mu);
    v[i] = r;
  }
  if (us.map != nullptr) {
    const int lane = threadIdx.x & 31;
    const uint32_t buf = us.sbuf + (us.n & 1u) * 2048u;
    if (us.n >= 2) {                               // the buffer's previous store has read it
      if (lane == 0) tc::bulk_wait_read<1>();
      __syncwarp();
    }
#pragma unroll
    for (int q = 0; q < 4; ++q)
      tc::st_shared_v4(buf + (uint32_t)(lane * 64 + 16 * (q ^ ((lane >> 1) & 3))), v[8 * q] | (v[8 * q + 1] << 16),
                       v[8 * q + 2] | (v[8 * q + 3] << 16), v[8 * q + 4] | (v[8 * q + 5] << 16),
                       v[8 * q + 6] | (v[8 * q + 7] << 16));
    tc::fence_proxy_async_smem();
    __syncwarp();
    if (lane == 0) {
      tc::tma_store_3d(us.map, buf, col, e.row - lane, e.ell);   // rows >= M, columns >= N are not written
      tc::bulk_commit();
    }
    ++us.n;
    return;
  }
  if (e.row >= e.M) return;
  if (e.vec_ok && col + 32 <= e.N) {
    uint4* dst = reinterpret_cast<uint4*>(e.urow + col);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      uint4 w;
      w.x = v[8 * q + 0] | (v[8 * q + 1] << 16);
      w.y = v[8 * q + 2] | (v[8 * q + 3] << 16);
      w.z = v[8 * q + 4] | (v[8 * q + 5] << 16);
      w.w = v[8 * q + 6] | (v[8 * q + 7] << 16);
      dst[q] = w;
    }
  } else {
#pragma unroll
    for (int i = 0; i < 32; ++i)
      if (col + i < e.N) e.urow[col + i] = (uint16_t)v[i];
  }
}

// The epilogue of one job over NC chunks of 32 columns at tbase, the TMEM
// load of each chunk in flight while the one before it is reduced.  Ends
// with every TMEM store of the job complete.
template <int NC>
__device__ __forceinline__ void epi_job(const Job& j, const EpiConst& e, uint32_t tbase, UStage& us) {
  static_assert(NC % 2 == 0, "chunks go in pairs");
  uint32_t va[32], vb[32];
  tc::tmem_ld32_nowait(tbase, va);
  tc::tmem_ld_wait_regs(va);
#pragma unroll 1
  for (int c = 0; c < NC; c += 2) {
    tc::tmem_ld32_nowait(tbase + (uint32_t)(32 * (c + 1)), vb);
    epi_chunk(j, e, va, tbase + (uint32_t)(32 * c), 32 * c, us);
    tc::tmem_ld_wait_regs(vb);
    if (c + 2 < NC) tc::tmem_ld32_nowait(tbase + (uint32_t)(32 * (c + 2)), va);
    epi_chunk(j, e, vb, tbase + (uint32_t)(32 * (c + 1)), 32 * (c + 1), us);
    if (c + 2 < NC) tc::tmem_ld_wait_regs(va);
  }
  if (!j.last) tc::tmem_wait_st();
}

}  // namespace plane
}  // namespace oz2
