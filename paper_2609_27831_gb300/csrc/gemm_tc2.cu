// Stages 3-4 of the Ozaki-II flow (Sec. 4.1) on CTA pairs: one exact integer
// GEMM per residue plane and the reduction of each product mod m_l with the
// Karatsuba combine of Eq. 4-5, as in the one-SM kernel (gemm_tc.cu), but
// each 256 x 256 output tile is computed by a cluster of two CTAs on two SMs
// with tcgen05.mma.cta_group::2.
//
// Why pairs: one SM's 128 x 256 tile needs 48 KB of operands per 64-wide K
// block; a pair's 256 x 256 tile needs 64 KB for twice the products, 32 KB per
// SM (its 128 rows of A and its half of the 256 columns of B).  Operand traffic
// from L2 per product drops by a third, and six stages fit in shared memory
// instead of four.
//
// Roles, in both CTAs of a pair (cluster rank r = 0 is the leader):
//   warp 0 lane 0  producer: TMA loads of the CTA's A rows (tm 256 + 128 r ..)
//                  and B rows (tn 256 + 128 r ..) into its own ring; both
//                  CTAs' loads complete on the leader's `full` barrier
//   warp 1         TMEM owner (512 columns, allocated for the pair); in the
//                  leader, lane 0 issues the MMAs (M = 256, N = 256, K = 16)
//                  and commits to both CTAs' `empty` and `slot_full` barriers
//   warps 2..9     epilogue of the CTA's 128 rows (two warps per TMEM lane
//                  quadrant, 128 columns each), exactly as in the one-SM
//                  kernel; one lane per warp then arrives on the leader's
//                  `slot_free` barrier
// Every wait is bounded (DevTables::spin_limit); a timeout sets the status
// word and the CTA's abort flag, drains the copies and MMAs in flight and
// reaches the final cluster barrier, after which both CTAs free the TMEM.
#include <climits>

#include "oz2_internal.h"
#include "plane_common.cuh"
#include "tc_ptx.cuh"

namespace oz2 {

namespace {

using namespace tc;
using namespace plane;

constexpr int kRows = 128;                            // A rows and B rows per CTA
constexpr int kTileBytes = kRows * kBK * 2;           // 16 KB
constexpr int kStageBytes2 = 2 * kTileBytes;          // 32 KB per CTA
constexpr int kStages2 = 6;
constexpr int kEpiWarps = 8;                          // a multiple of 4 (one per TMEM lane quadrant)
constexpr int kEpiCols = kBN / (kEpiWarps / 4);       // columns of a slot per epilogue warp
constexpr int kThreads2 = 64 + kEpiWarps * 32;
constexpr int kStageOff2 = kStages2 * kStageBytes2 + 1024;   // v_l staging, after the barriers
constexpr int kSmemBytes2 = kStageOff2 + kEpiWarps * 4096 + 1024 /*align*/;
// D = f32, A = B = bf16, both K-major, M = 256 (the pair), N = 256.
constexpr uint32_t kIdesc2 = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(256 >> 3) << 17) |
                             ((uint32_t)(256 >> 4) << 24);

__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
// shared::cluster address of the same shared-memory object in CTA `rank`
__device__ __forceinline__ uint32_t map_to(uint32_t saddr, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(saddr), "r"(rank));
  return r;
}
__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// TMA load into this CTA's shared memory, completing on a barrier that may
// live in the peer CTA (shared::cluster address)
__device__ __forceinline__ void tma_load_3d_pair(uint32_t dst, const CUtensorMap* map, uint32_t bar_cluster,
                                                 int c0, int c1, int c2) {
  asm volatile(
      "cp.async.bulk.tensor.3d.cta_group::2.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4, %5}], [%2];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(bar_cluster), "r"(c0), "r"(c1), "r"(c2)
      : "memory");
}
__device__ __forceinline__ void umma_pair(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(kIdesc2), "r"(acc)
      : "memory");
}
// arrive once on the barrier at this shared-memory offset in both CTAs of the pair
__device__ __forceinline__ void commit_pair(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(
          smem_u32(bar)),
      "h"((uint16_t)3)
      : "memory");
}
// arrive on a barrier that may live in the peer CTA (default .release.cta
// semantics: the slot's TMEM reads are ordered by tcgen05.wait::ld and the
// tcgen05 fences around the arrive and the leader's wait, not by the memory
// model, so no cluster-scope fence is needed)
__device__ __forceinline__ void arrive_cluster(uint32_t bar_cluster) {
  asm volatile("mbarrier.arrive.shared::cluster.b64 _, [%0];" ::"r"(bar_cluster) : "memory");
}

__global__ void __launch_bounds__(kThreads2, 1) k_gemm_tc2(const __grid_constant__ DevTables T) {
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;     // the same offset in both CTAs (same kernel, same smem)
  uint8_t* smem = smem_raw + (base - raw);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + kStages2 * kStageBytes2);
  uint64_t* full = bars;                             // [kStages2] leader: both CTAs' loads
  uint64_t* empty = bars + kStages2;                 // [kStages2] MMAs done with the stage
  uint64_t* slot_full = bars + 2 * kStages2;         // [2] accumulator ready
  uint64_t* slot_free = bars + 2 * kStages2 + 2;     // [2] leader: both CTAs' epilogues done
  uint64_t* drain = bars + 2 * kStages2 + 4;         // [1] leader: abort drain of the MMA pipe
  volatile int* abort_flag = reinterpret_cast<volatile int*>(bars + 2 * kStages2 + 5);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * kStages2 + 6);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t rank = cluster_rank();
  const bool leader = rank == 0;
  const int pair = blockIdx.x >> 1;
  const int ubeg = T.cta_begin[pair], uend = T.cta_begin[pair + 1];

  if (threadIdx.x == 0) {
    for (int i = 0; i < kStages2; ++i) {
      mbar_init(full + i, 1);
      mbar_init(empty + i, 1);
    }
    for (int s = 0; s < 2; ++s) {
      mbar_init(slot_full + s, 1);
      mbar_init(slot_free + s, 2 * kEpiWarps);
    }
    mbar_init(drain, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(smem_u32(tmem_slot))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  cluster_sync();                                    // barriers of both CTAs initialised, TMEM allocated
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0 && lane == 0) {
    // ------------------------------------------------------------ producer (both CTAs)
    JobIter it;
    it.init(&T, ubeg, uend);
    Job j;
    int st = 0;
    uint32_t ph = 0;
    int issued_phase[kStages2];
    for (int i = 0; i < kStages2; ++i) issued_phase[i] = -1;
    const uint32_t full_leader0 = map_to(smem_u32(full), 0);
    bool ok = true;
    while (ok && it.next(j)) {
      const ProbDev& P = T.probs[j.u.prob];
      const CUtensorMap* ma = T.tmaps + 2 * j.u.prob;
      const CUtensorMap* mb = ma + 1;
      const int k0 = j.chunk * P.kchunk;
      const int k1 = min(P.K, k0 + P.kchunk);
      const int arow = j.u.tm * 256 + (int)rank * kRows;
      const int brow = j.u.tn * 256 + (int)rank * kRows;
      for (int k = k0; k < k1; k += kBK) {
        if (!mbar_wait(empty + st, ph ^ 1u, abort_flag, T.status, T.spin_limit)) { ok = false; break; }
        if (leader) mbar_expect_tx(full + st, 2u * kStageBytes2);
        const uint32_t sa = base + st * kStageBytes2;
        const uint32_t fb = full_leader0 + (uint32_t)(st * 8);
        tma_load_3d_pair(sa, ma, fb, k, arow, j.plane);
        tma_load_3d_pair(sa + kTileBytes, mb, fb, k, brow, j.plane);
        issued_phase[st] = (int)ph;
        if (++st == kStages2) { st = 0; ph ^= 1u; }
      }
    }
    if (!ok) {
      if (leader) {
        // let the copies in flight (this CTA's and the peer's) land before the pair exits
        for (int i = 0; i < kStages2; ++i) {
          if (issued_phase[i] >= 0) {
            for (uint32_t t = 0; t < kSpinLimit && !mbar_try_wait(full + i, (uint32_t)issued_phase[i]); ++t) {}
          }
        }
      } else {
        // the peer's copies complete on the leader's barriers, which it cannot
        // poll: give any copy still in flight 100 us to land in its ring
        for (int t = 0; t < 100; ++t) __nanosleep(1000);
      }
    }
  } else if (warp == 1 && lane == 0 && leader) {
    // ------------------------------------------------------------ MMA issuer (leader)
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
        if (!mbar_wait(slot_free + s, (uint32_t)((uses[s] - 1) & 1), abort_flag, T.status, T.spin_limit)) {
          ok = false;
          break;
        }
      }
      ++uses[s];
      tc_fence_after();
      const uint32_t d = tmem + (uint32_t)(s * kBN);
      bool acc = !j.first;
      for (int k = k0; k < k1; k += kBK) {
        if (!mbar_wait(full + st, ph, abort_flag, T.status, T.spin_limit)) { ok = false; break; }
        tc_fence_after();
        const uint32_t sa = base + st * kStageBytes2;
        const uint64_t da = desc_sw128(sa);
        const uint64_t db = desc_sw128(sa + kTileBytes);
#pragma unroll
        for (int kk = 0; kk < kBK / 16; ++kk) {
          umma_pair(d, da + (uint64_t)(2 * kk), db + (uint64_t)(2 * kk), acc ? 1u : 0u);
          acc = true;
        }
        commit_pair(empty + st);
        any = true;
        if (++st == kStages2) { st = 0; ph ^= 1u; }
      }
      if (!ok) break;
      commit_pair(slot_full + s);
    }
    if (!ok && any) {
      // drain issued MMAs before TMEM is released
      asm volatile("tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       smem_u32(drain))
                   : "memory");
      for (uint32_t t = 0; t < kSpinLimit && !mbar_try_wait(drain, 0); ++t) {}
    }
  } else if (warp >= 2) {
    // ------------------------------------------------------------ epilogue (both CTAs)
    const int ew = warp - 2;
    const int quad = warp & 3;          // TMEM lane quadrant this warp may access
    const int half = ew >> 2;           // column range of the 256-column slot
    const uint32_t free_leader = map_to(smem_u32(slot_free), 0);
    JobIter it;
    it.init(&T, ubeg, uend);
    Job j;
    int uses[2] = {0, 0};
    UStage us{nullptr, base + (uint32_t)(kStageOff2 + ew * 4096), 0u};
    while (it.next(j)) {
      const int s = j.slot;
      const int row = j.u.tm * 256 + (int)rank * kRows + quad * 32 + lane;
      const uint32_t tbase = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(s * kBN + half * kEpiCols);
      const EpiConst e = epi_const(T, j, row, j.u.tn * kBN + half * kEpiCols);
      us.map = T.probs[j.u.prob].u_map ? T.tmaps + 5 * T.count + j.u.prob : nullptr;
      if (!mbar_wait(slot_full + s, (uint32_t)(uses[s] & 1), abort_flag, T.status, T.spin_limit)) break;
      ++uses[s];
      tc_fence_after();
      epi_job<kEpiCols / 32>(j, e, tbase, us);
      tc_fence_before();
      __syncwarp();
      if (lane == 0) arrive_cluster(free_leader + (uint32_t)(s * 8));
    }
    if (lane == 0) bulk_wait_all();                  // the v_l stores are complete before the CTA exits
  }

  __syncwarp();
  tc_fence_before();
  cluster_sync();                                    // every MMA of the pair is complete and read
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, 512;" ::"r"(tmem) : "memory");
  }
}

}  // namespace

cudaError_t init_gemm2_attributes() {
  return cudaFuncSetAttribute(k_gemm_tc2, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes2);
}

// `pairs` CTA pairs (clusters of two); T.cta_begin holds pairs + 1 unit ranges.
cudaError_t launch_gemm_tc2(const DevTables& t, int pairs, cudaStream_t s) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3((unsigned)(2 * pairs), 1, 1);
  cfg.blockDim = dim3(kThreads2, 1, 1);
  cfg.dynamicSmemBytes = kSmemBytes2;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 2;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_gemm_tc2, t);
}

}  // namespace oz2
