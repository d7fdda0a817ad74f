// Internal structures shared by the host planner (api.cu) and the sm_103a
// kernels (prep.cu, gemm_tc.cu, crt.cu).  Not part of the public ABI.
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>
#include <cuda.h>

#include "ozaki2.h"

namespace oz2 {

// Tile of the tensor-core plane GEMM (UMMA M x N, K block of one 128-byte
// swizzle row of bf16).
constexpr int kBM = 128;
constexpr int kBN = 256;
constexpr int kBK = 64;
constexpr int kStages = 4;
constexpr int kMaxKChunk = 1024;   // 127^2 * 1024 + 16191 < 2^24: fp32 accumulation stays exact

// Polls of a bounded mbarrier wait before it gives up (the launch's
// DevTables::spin_limit; a plan may lower it to test the timeout path).
constexpr uint32_t kDefaultSpinLimit = 1u << 26;

constexpr int kMaxP = 2048;
// Tensor maps per problem descriptor, at i + n count for problem i of count:
// A planes (2 i), B planes (2 i + 1), tensor-core CRT table (n = 2), u tiles
// read by the CRT (n = 3), residue table (n = 4), v_l tiles stored by the
// plane GEMM (n = 5).
constexpr int kMapsPerProblem = 6;
constexpr int kMaxK = 133000;      // Sec. 4.3(a) implementation cap

// Per-modulus constants (index = position in the global modulus list).
struct ModConst {
  uint32_t m;       // modulus
  uint32_t mu;      // floor(2^32 / m)  (Barrett reduction of 32-bit values, and the
                    //                   fixed-point CRT quotient estimate)
  uint32_t c24;     // 2^24 mod m
  float rcp;        // 1/m rounded to nearest float (epilogue reduction of exact fp32 sums)
  uint32_t kmul01;  // Karatsuba coefficient carry between the P0 and Ps planes (two-limb)
  uint32_t kmul12;  // ... between the Ps and P2 planes (two-limb)
  uint32_t kfin;    // final coefficient (two-limb: 16256 mod m; one-limb: 1)
  uint32_t pad;
};

// Per-problem descriptor read by the kernels.
struct ProbDev {
  // inputs / outputs (caller memory)
  const uint64_t* a_limbs; const int32_t* a_exp; const int8_t* a_sign;
  int64_t a_ld, a_ps;
  const uint64_t* b_limbs; const int32_t* b_exp; const int8_t* b_sign;
  int64_t b_ld, b_ps;
  uint64_t* c_limbs; int32_t* c_exp; int8_t* c_sign;
  int64_t c_ld, c_ps;
  // workspace regions
  int32_t* e;            // [M] row exponents of A
  int32_t* f;            // [N] column exponents of B
  uint16_t* pa;          // bf16 bits [G][M][Kp]
  uint16_t* pb;          // bf16 bits [G][N][Kp]
  uint16_t* u;           // [L][upitch]: v_l = u_l M_l^{-1} mod m_l per output (the plane GEMM's result)
  // shape and parameters
  int32_t M, N, K, p, nl, t;
  int32_t L, L1, G, Kp;
  int32_t W16;           // 16-bit digits of a (t+1)-bit integer
  int32_t D32;           // 32-bit digits of the CRT accumulator
  int32_t crt_off;       // offset (uint32 words) of this problem's CRT tables in the pool
  int32_t tiles_m, tiles_n;
  int32_t nchunks, kchunk;
  int32_t kind;          // 0 = multiple-precision limbs, 1 = binary64 input/output
  int32_t pad0;
  const double* a_f64; const double* b_f64; double* c_f64;   // binary64 mode
  int64_t a_f64_ld, b_f64_ld, c_f64_ld;
  int32_t a_f64_trans, b_f64_trans;                          // binary64 operand read transposed
  int32_t e_scale_mode, pad1;                                // backward scaling (see fp64 notes)
  const int32_t* ext_scale;                                  // per-line extra exponent (backward)
  int32_t ext_scale_axis;
  int32_t crt_gskip;     // crt_mode 2, long finish: groups of 32 Y columns below this one are not
                         // formed (the finish's fast form starts at it; stored group g is crt_gskip + g)
  int32_t DS;            // digit stride of the CRT tables (digits of the kernel class)
  int32_t crt_mode;      // 0: CUDA-core CRT; 1: column sums on the tensor cores (one kernel);
                         // 2: column sums on the tensor cores written as digits R, then the finish
  uint32_t* dbg_chat;    // optional: [M*N][D32+1] sign word + |c_hat| digits
  int32_t crt_kpad;      // tensor-core CRT: K = 2L padded to a multiple of 64
  int32_t crt_npad;      // tensor-core CRT: 7-bit pieces of S padded to a multiple of 16
  int32_t crt_np;        // tensor-core CRT: 7-bit pieces of S (columns of Y)
  int32_t crt_nvbuf;     // crt_mode 2: V buffers in TMEM (2 where kpad + nslot cw <= 512)
  int64_t upitch;        // row pitch of u [L][upitch]: M*N rounded up to a multiple of 8
  int32_t res_mode;      // 0: residues on the CUDA cores; 1: byte GEMM on the tensor cores;
                         // 2: the byte GEMM, warp-specialised (bytes in TMEM, table streamed)
  int32_t res_kpad;      // tensor-core residues: bytes of a (t+1)-bit integer, padded to 64
  int32_t res_npad;      // tensor-core residues: table rows L1 + 2 (L - L1), padded to 16
  int32_t crt_nchunk;    // crt_mode 2: chunks of crt_cw columns of Y
  int32_t crt_cw;        // crt_mode 2: columns of Y per chunk (a multiple of 32)
  uint32_t* crt_q;       // crt_mode 2: group sums Q_g as [ngrp][9][upitch] words
  uint32_t* crt_alpha;   // crt_mode 2: quotient estimates alpha~ [upitch]
  int32_t crt_ngrp;      // crt_mode 2: groups of 32 columns, nchunk cw / 32
  int32_t res_cw;        // res_mode 2: columns of Y per chunk (a multiple of 32)
  int32_t res_nchunk;    // res_mode 2: chunks
  int32_t crt_nslot;     // crt_mode 2: TMEM accumulator slots (1 or 2)
  int32_t res_nabuf;     // res_mode 2: byte buffers (A) in TMEM (2 or 4)
  int32_t u_map;         // 1: tensor map 5 * count + i stores v_l tiles (N a multiple of 8)
  int32_t* dbg_prods;    // optional (K within one chunk): [G][M][N] exact plane sums before reduction
};

// CRT tables of one modulus prefix, laid out in a uint32 pool at crt_off,
// digit rows padded with zeros to the stride DS:
//   P      [DS]            little-endian digits of P
//   negP   [DS]            2^(32 D32) - P (digits >= D32 zero)
//   negH1  [DS]            2^(32 D32) - (floor(P/2) + 1)
//   Minv   [L]             M_l^{-1} mod m_l
//   Mdig   [L][DS]         digits of M_l = P / m_l
// The long CRT finish skips forming the lowest group sums (ProbDev::crt_gskip)
// only up to this many accumulator digits: its full form then rebuilds R from
// v_l in a per-thread array of this size.
constexpr int kCrtSkipMaxDigits = 256;

struct CrtView {
  const uint32_t* P; const uint32_t* negP; const uint32_t* negH1;
  const uint32_t* Minv; const uint32_t* Mdig;
};

__host__ __device__ inline CrtView crt_view(const uint32_t* pool, const ProbDev& pr) {
  const uint32_t* b = pool + pr.crt_off;
  CrtView v;
  v.P = b;
  v.negP = b + pr.DS;
  v.negH1 = b + 2 * pr.DS;
  v.Minv = b + 3 * pr.DS;
  v.Mdig = b + 3 * pr.DS + pr.L;
  return v;
}

// One (modulus, output tile) work unit of the grouped GEMM.
struct Unit {
  uint16_t prob;
  uint16_t ell;    // modulus index within the problem
  uint16_t tm;     // output tile row
  uint16_t tn;     // output tile column
};

// Device-resident launch data of a plan (library-owned).
struct DevTables {
  const ModConst* mods;      // [Lmax]
  const uint32_t* t16;       // [Lmax][W16max]: 2^(16 d) mod m_l
  int32_t w16max;
  int32_t lmax;
  const uint32_t* crt_pool;
  const ProbDev* probs;
  const Unit* units;
  const int32_t* cta_begin;  // [grid + 1] unit ranges per persistent CTA
  const CUtensorMap* tmaps;  // [kMapsPerProblem * count]: see kMapsPerProblem
  int32_t* status;           // device status word
  int32_t count;
  uint32_t spin_limit;       // iterations of a bounded mbarrier wait before it gives up
};

// Status bits of the device status word.
constexpr int kStatusCrtRange = 1;     // R outside [0, 2P) after the quotient estimate
constexpr int kStatusTimeout = 2;      // a bounded mbarrier wait gave up
constexpr int kStatusBadUnit = 4;      // a unit index out of range

// Launchers (defined in the .cu files).
cudaError_t launch_scan(const DevTables& t, int count, const int32_t* blk_prefix_rows,
                        const int32_t* blk_prefix_cols, int nblk_rows, int nblk_cols,
                        cudaStream_t s);
cudaError_t launch_residues(const DevTables& t, int w16_class, const int32_t* blk_list,
                            int nblk, int smem_bytes, cudaStream_t s);
cudaError_t launch_gemm_tc(const DevTables& t, int grid, cudaStream_t s);
// CTA-pair plane GEMM (256 x 256 tiles): `pairs` clusters of two CTAs,
// t.cta_begin holding pairs + 1 unit ranges.
cudaError_t launch_gemm_tc2(const DevTables& t, int pairs, cudaStream_t s);
cudaError_t launch_gemm_simt(const DevTables& t, const int32_t* unit_list, int nunits,
                             cudaStream_t s);
// INT8 mma.sync engine: blocks {unit index (units in problem order), half of the 256 columns}.
cudaError_t launch_gemm_s8(const DevTables& t, const int32_t* list, int n, cudaStream_t s);
cudaError_t launch_crt(const DevTables& t, int cls, const int32_t* blk_list, int nblk, int lmax,
                       cudaStream_t s);
// Tensor-core CRT for one-lane class `cls` (0..8): tiles of 128 outputs.
cudaError_t launch_crt_tc(const DevTables& t, int cls, const int32_t* tiles, int ntiles, int kpad_max,
                          int npad_max, int lmax, int sms, cudaStream_t s);
int crt_tc_smem_bytes(int cls, int kpad_max, int npad_max, int lmax, int nbuf);
// Tensor-core CRT sums of any length (crt_mode 2): tiles of 128 outputs
// {problem, tile}; R digits to the workspace.  Then the finish of long
// accumulators (> 40 digits), blocks of 128 outputs {problem, block}.
cudaError_t launch_crt_mm(const DevTables& t, const int32_t* tiles, int ntiles, int cw_max, int grid,
                          int blocks_one, cudaStream_t s);
int crt_mm_chunk(int kpad, int npad, int* nslot);
int crt_mm_smem_bytes(int cw_max, int lmax, int* stages);
// the finish of one-lane classes after the tensor-core sums (the host uses it up to 24 digits)
cudaError_t launch_crt_fin_short(const DevTables& t, int cls, const int32_t* blk, int nblk, cudaStream_t s);
int crt_finish_long_smem(int dmax, int nlmax);
cudaError_t launch_crt_finish_long(const DevTables& t, const int32_t* blk, int nblk, int dmax, int nlmax,
                                   cudaStream_t s);
// Tensor-core residues: persistent tiles of 4 lines x 32 k.
cudaError_t launch_residues_tc(const DevTables& t, const int32_t* tiles, int ntiles, int kpad_max, int npad_max,
                               int lmax, int sms, cudaStream_t s);
int residue_tc_smem_bytes(int kpad, int npad, int lmax);
// Warp-specialised tensor-core residues (res_mode 2): the same tiles.
cudaError_t launch_residues_mm(const DevTables& t, const int32_t* tiles, int ntiles, int cw_max, int tcols,
                               int sms, cudaStream_t s);
void residue_mm_geometry(int kpad, int npad, int* cw, int* nabuf);
int residue_mm_smem_bytes(int cw_max, int lmax, int tcols, int* stages);

// Internal plan variants used by the binary64 mode.
struct PlanExtra {
  int64_t inner = 0;     // choose moduli for inner length max(K, inner)
  int force_t = 0;       // use this internal width t
  int force_L = 0;       // use exactly this many moduli (must still meet the CRT bound)
  int kind = 0;          // 1: binary64 output (C.limbs is a double*, C.ld its stride)
  bool skip_a = false;   // A planes are written by the caller; row exponents are 0
  bool skip_b = false;   // B planes are written by the caller; column exponents are 0
};
struct PlanFacts {
  int t, L, G, Kp;
  size_t off_e, off_f, off_pa, off_pb, ws_bytes;
};
int plan_create_ex(int64_t M, int64_t N, int64_t K, int p, const ozaki2_opts* opts,
                   const PlanExtra& ex, ozaki2_plan* out);
int plan_query(ozaki2_plan pl, PlanFacts* f);
int plan_run(ozaki2_plan pl, const ozaki2_problem* q, void* ws, size_t ws_bytes, cudaStream_t s);

// Residue kernel W16 classes and CRT lane-group classes (host picks per problem).
int residue_class_for(int w16);        // -> class index, or -1
int residue_class_w16(int cls);
int residue_class_ept(int cls);       // elements per thread of that class (block: 32 EPT k x 8 lines)
constexpr int kCrtClassCount = 12;
int crt_class_for(int d32);            // -> class index, or -1
int crt_class_elems_per_block(int cls);
int crt_class_digits(int cls);

}  // namespace oz2
