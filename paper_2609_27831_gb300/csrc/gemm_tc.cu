// Stages 3-4 of the Ozaki-II flow (Sec. 4.1): one exact integer GEMM per
// residue plane and the reduction of each product mod m_l, with the
// Karatsuba combine of the three two-limb planes (Eq. 4-5) fused into the
// epilogue.
//
// Engine: tcgen05.mma kind::f16 with bf16 operands.  Every plane entry is an
// integer with |r| <= 127, exact in bf16; products are exact in fp32 and the
// fp32 accumulator in TMEM stays exact while every partial sum is an integer
// below 2^24.  K is therefore processed in chunks of at most 1024
// (127^2 * 1024 + 16191 < 2^24).  Between chunks (and between the three
// Karatsuba planes of a two-limb modulus) the epilogue warps read the
// accumulator, reduce it mod m and write the small residue back into TMEM, so
// the next chunk accumulates on top of it: no running state lives in registers
// and no partial product ever leaves the SM.
//
// Persistent grouped kernel: one CTA per SM walks its list of (problem,
// modulus, 128x256 output tile) units; two TMEM accumulator slots of 256
// columns alternate between two unit streams so that the MMA of one job
// overlaps the epilogue of the other.
//
// Warp roles: warp 0 = TMA producer, warp 1 = MMA issuer (+ TMEM owner),
// warps 2..9 = epilogue (two per TMEM lane quadrant, 128 columns each).
#include <climits>

#include "oz2_internal.h"
#include "plane_common.cuh"
#include "tc_ptx.cuh"

namespace oz2 {

namespace {

using namespace tc;
using namespace plane;

constexpr int kTileABytes = kBM * kBK * 2;            // 16 KB
constexpr int kTileBBytes = kBN * kBK * 2;            // 32 KB
constexpr int kStageBytes = kTileABytes + kTileBBytes;
constexpr int kEpiWarps = 8;                          // a multiple of 4 (one per TMEM lane quadrant)
constexpr int kEpiCols = kBN / (kEpiWarps / 4);       // columns of a slot per epilogue warp
constexpr int kThreads = 64 + kEpiWarps * 32;
constexpr int kStageOff = kStages * kStageBytes + 1024;      // v_l staging, after the barriers
constexpr int kSmemBytes = kStageOff + kEpiWarps * 4096 + 1024 /*align*/;
// Instruction descriptor: D = f32, A = B = bf16, both K-major, M = 128, N = 256.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kBN >> 3) << 17) |
                            ((uint32_t)(kBM >> 4) << 24);

__device__ __forceinline__ void umma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t acc) {
  tc::umma_bf16(d_tmem, a, b, kIdesc, acc);
}
__global__ void __launch_bounds__(kThreads, 1) k_gemm_tc(const __grid_constant__ DevTables T) {
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  uint8_t* smem = smem_raw + (base - raw);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + kStages * kStageBytes);
  uint64_t* full = bars;                 // [kStages]
  uint64_t* empty = bars + kStages;      // [kStages]
  uint64_t* slot_full = bars + 2 * kStages;   // [2]
  uint64_t* slot_free = bars + 2 * kStages + 2;   // [2]
  uint64_t* drain = bars + 2 * kStages + 4;       // [1] abort drain of the MMA pipe
  volatile int* abort_flag = reinterpret_cast<volatile int*>(bars + 2 * kStages + 5);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * kStages + 6);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int cta = blockIdx.x;
  const int ubeg = T.cta_begin[cta], uend = T.cta_begin[cta + 1];

  if (threadIdx.x == 0) {
    for (int i = 0; i < kStages; ++i) {
      mbar_init(full + i, 1);
      mbar_init(empty + i, 1);
    }
    for (int s = 0; s < 2; ++s) {
      mbar_init(slot_full + s, 1);
      mbar_init(slot_free + s, kEpiWarps * 32);
    }
    mbar_init(drain, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(
                     smem_u32(tmem_slot))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0 && lane == 0) {
    // ------------------------------------------------------------ producer
    JobIter it;
    it.init(&T, ubeg, uend);
    Job j;
    int st = 0;
    uint32_t ph = 0;
    int issued_phase[kStages];
    for (int i = 0; i < kStages; ++i) issued_phase[i] = -1;
    bool ok = true;
    while (ok && it.next(j)) {
      const ProbDev& P = T.probs[j.u.prob];
      const CUtensorMap* ma = T.tmaps + 2 * j.u.prob;
      const CUtensorMap* mb = ma + 1;
      const int k0 = j.chunk * P.kchunk;
      const int k1 = min(P.K, k0 + P.kchunk);
      for (int k = k0; k < k1; k += kBK) {
        if (!mbar_wait(empty + st, ph ^ 1u, abort_flag, T.status, T.spin_limit)) { ok = false; break; }
        mbar_expect_tx(full + st, kStageBytes);
        const uint32_t sa = base + st * kStageBytes;
        tma_load_3d(sa, ma, smem_u32(full + st), k, j.u.tm * kBM, j.plane);
        tma_load_3d(sa + kTileABytes, mb, smem_u32(full + st), k, j.u.tn * kBN, j.plane);
        issued_phase[st] = (int)ph;
        if (++st == kStages) { st = 0; ph ^= 1u; }
      }
    }
    if (!ok) {
      // let copies already in flight land before the CTA exits
      for (int i = 0; i < kStages; ++i) {
        if (issued_phase[i] >= 0) {
          for (uint32_t t = 0; t < kSpinLimit && !mbar_try_wait(full + i, (uint32_t)issued_phase[i]); ++t) {}
        }
      }
    }
  } else if (warp == 1 && lane == 0) {
    // ------------------------------------------------------------ MMA issuer
    JobIter it;
    it.init(&T, ubeg, uend);
    Job j;
    int st = 0;
    uint32_t ph = 0;
    int uses[2] = {0, 0};
    bool ok = true;
    bool any = false;
    while (ok && it.next(j)) {
      const ProbDev& P = T.probs[j.u.prob];
      const int s = j.slot;
      const int k0 = j.chunk * P.kchunk;
      const int k1 = min(P.K, k0 + P.kchunk);
      if (uses[s] > 0) {
        if (!mbar_wait(slot_free + s, (uint32_t)((uses[s] - 1) & 1), abort_flag, T.status, T.spin_limit)) { ok = false; break; }
      }
      ++uses[s];
      tc_fence_after();
      const uint32_t d = tmem + (uint32_t)(s * kBN);
      bool acc = !j.first;
      for (int k = k0; k < k1; k += kBK) {
        if (!mbar_wait(full + st, ph, abort_flag, T.status, T.spin_limit)) { ok = false; break; }
        tc_fence_after();
        const uint32_t sa = base + st * kStageBytes;
        const uint64_t da = desc_sw128(sa);
        const uint64_t db = desc_sw128(sa + kTileABytes);
#pragma unroll
        for (int kk = 0; kk < kBK / 16; ++kk) {
          umma(d, da + (uint64_t)(2 * kk), db + (uint64_t)(2 * kk), acc ? 1u : 0u);
          acc = true;
        }
        umma_commit(empty + st);
        any = true;
        if (++st == kStages) { st = 0; ph ^= 1u; }
      }
      if (!ok) break;
      umma_commit(slot_full + s);
    }
    if (!ok && any) {
      // drain issued MMAs before TMEM is released
      umma_commit(drain);
      for (uint32_t t = 0; t < kSpinLimit && !mbar_try_wait(drain, 0); ++t) {}
    }
  } else if (warp >= 2) {
    // ------------------------------------------------------------ epilogue
    const int ew = warp - 2;
    const int quad = warp & 3;          // TMEM lane quadrant this warp may access
    const int half = ew >> 2;           // column range of the 256-column slot
    JobIter it;
    it.init(&T, ubeg, uend);
    Job j;
    int uses[2] = {0, 0};
    UStage us{nullptr, base + (uint32_t)(kStageOff + ew * 4096), 0u};
    while (it.next(j)) {
      const int s = j.slot;
      const int row = j.u.tm * kBM + quad * 32 + lane;
      const uint32_t tbase = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(s * kBN + half * kEpiCols);
      const EpiConst e = epi_const(T, j, row, j.u.tn * kBN + half * kEpiCols);
      us.map = T.probs[j.u.prob].u_map ? T.tmaps + 5 * T.count + j.u.prob : nullptr;
      if (!mbar_wait(slot_full + s, (uint32_t)(uses[s] & 1), abort_flag, T.status, T.spin_limit)) break;
      ++uses[s];
      tc_fence_after();
      epi_job<kEpiCols / 32>(j, e, tbase, us);
      tc_fence_before();
      mbar_arrive(slot_free + s);
    }
    if (lane == 0) bulk_wait_all();                  // the v_l stores are complete before the CTA exits
  }

  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem) : "memory");
  }
}

// ---------------------------------------------------------------------------
// CUDA-core cross-check engine: the same unit list, exact int32 dot products
// of the bf16 planes, Karatsuba combine in int64.  Slow; used to test the
// tensor-core engine.  Block = one unit's 32 x 32 sub-tile.
// Entry: {unit index, sub-tile row, sub-tile col, 0}.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int bf2i(uint16_t h) {
  return (int)__uint_as_float(((uint32_t)h) << 16);
}

__global__ void __launch_bounds__(256) k_gemm_simt(DevTables T, const int4* __restrict__ list) {
  __shared__ int sa[3][32][33];
  __shared__ int sb[3][32][33];
  const int4 e = list[blockIdx.x];
  const Unit u = T.units[e.x];
  const ProbDev& P = T.probs[u.prob];
  const bool two = u.ell >= P.L1;
  const int np = two ? 3 : 1;
  const int g0 = two ? P.L1 + 3 * (u.ell - P.L1) : u.ell;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 32 x 8
  const int row0 = u.tm * kBM + e.y * 32, col0 = u.tn * kBN + e.z * 32;
  int acc[3][4];
  for (int p = 0; p < 3; ++p)
    for (int q = 0; q < 4; ++q) acc[p][q] = 0;
  const int64_t psA = (int64_t)P.M * P.Kp, psB = (int64_t)P.N * P.Kp;
  for (int k0 = 0; k0 < P.K; k0 += 32) {
    for (int p = 0; p < np; ++p) {
      for (int q = 0; q < 4; ++q) {
        const int rr = ty + 8 * q;
        const int k = k0 + tx;
        const int ra = row0 + rr, cb = col0 + rr;
        sa[p][rr][tx] = (ra < P.M && k < P.K) ? bf2i(P.pa[(g0 + p) * psA + (int64_t)ra * P.Kp + k]) : 0;
        sb[p][rr][tx] = (cb < P.N && k < P.K) ? bf2i(P.pb[(g0 + p) * psB + (int64_t)cb * P.Kp + k]) : 0;
      }
    }
    __syncthreads();
    for (int p = 0; p < np; ++p)
      for (int q = 0; q < 4; ++q) {
        const int rr = ty + 8 * q;
        int s = 0;
        for (int kk = 0; kk < 32; ++kk) s += sa[p][rr][kk] * sb[p][tx][kk];
        acc[p][q] += s;
      }
    __syncthreads();
  }
  const int64_t m = T.mods[u.ell].m;
  for (int q = 0; q < 4; ++q) {
    const int row = row0 + ty + 8 * q, col = col0 + tx;
    if (row >= P.M || col >= P.N) continue;
    int64_t v;
    if (!two) {
      v = acc[0][q];
    } else {
      const int64_t P0 = acc[0][q], P2 = acc[1][q], Ps = acc[2][q];
      v = P0 + 128 * (Ps - P0 - P2) + 16384 * P2;
    }
    v %= m;
    if (v < 0) v += m;
    v = v * __ldg(crt_view(T.crt_pool, P).Minv + u.ell) % m;   // v_l for the CRT
    P.u[(int64_t)u.ell * P.upitch + (int64_t)row * P.N + col] = (uint16_t)v;
  }
}

}  // namespace

cudaError_t init_gemm_attributes() {
  return cudaFuncSetAttribute(k_gemm_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
}

cudaError_t launch_gemm_tc(const DevTables& t, int grid, cudaStream_t s) {
  k_gemm_tc<<<grid, kThreads, kSmemBytes, s>>>(t);
  return cudaGetLastError();
}

cudaError_t launch_gemm_simt(const DevTables& t, const int32_t* unit_list, int nunits,
                             cudaStream_t s) {
  if (nunits == 0) return cudaSuccess;
  k_gemm_simt<<<nunits, 256, 0, s>>>(t, reinterpret_cast<const int4*>(unit_list));
  return cudaGetLastError();
}

}  // namespace oz2
