// Host side of the C ABI: plan construction (internal width t, modulus
// prefix, CRT tables, work schedule), device upload, TMA descriptors and the
// stream-ordered execution of the five stages (Sec. 4.1).
#include <cudaTypedefs.h>

#include <algorithm>
#include <array>
#include <atomic>
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <queue>
#include <tuple>
#include <vector>

#include "oz2_internal.h"

namespace oz2 {

// ---------------------------------------------------------------------------
// Small host bignum (little-endian 32-bit digits) for the CRT tables.
// ---------------------------------------------------------------------------
using Big = std::vector<uint32_t>;

static void big_trim(Big& a) {
  while (!a.empty() && a.back() == 0u) a.pop_back();
}
static void big_mul_small(Big& a, uint32_t m) {
  uint64_t carry = 0;
  for (auto& d : a) {
    const uint64_t t = (uint64_t)d * m + carry;
    d = (uint32_t)t;
    carry = t >> 32;
  }
  if (carry) a.push_back((uint32_t)carry);
}
static uint32_t big_divmod_small(const Big& a, uint32_t m, Big* q) {
  uint64_t r = 0;
  if (q) q->assign(a.size(), 0u);
  for (size_t i = a.size(); i-- > 0;) {
    const uint64_t cur = (r << 32) | a[i];
    if (q) (*q)[i] = (uint32_t)(cur / m);
    r = cur % m;
  }
  if (q) big_trim(*q);
  return (uint32_t)r;
}
static int big_bitlen(const Big& a) {
  if (a.empty()) return 0;
  int top = 31;
  while (!((a.back() >> top) & 1u)) --top;
  return 32 * (int)(a.size() - 1) + top + 1;
}
static int big_cmp(const Big& a, const Big& b) {
  if (a.size() != b.size()) return a.size() < b.size() ? -1 : 1;
  for (size_t i = a.size(); i-- > 0;)
    if (a[i] != b[i]) return a[i] < b[i] ? -1 : 1;
  return 0;
}
// (k << sh) as a bignum
static Big big_shifted(uint64_t k, int sh) {
  Big a((size_t)(sh / 32) + 3, 0u);
  const int w = sh / 32, b = sh % 32;
  const unsigned __int128 v = (unsigned __int128)k << b;
  a[w] = (uint32_t)v;
  a[w + 1] = (uint32_t)(v >> 32);
  a[w + 2] = (uint32_t)(v >> 64);
  big_trim(a);
  return a;
}
// 2^(32 D) - x, as exactly D digits (x < 2^(32 D), x != 0)
static Big big_neg_mod(const Big& x, int D) {
  Big r((size_t)D, 0u);
  uint64_t carry = 1;
  for (int i = 0; i < D; ++i) {
    const uint64_t t = (uint64_t)(uint32_t)~(i < (int)x.size() ? x[i] : 0u) + carry;
    r[i] = (uint32_t)t;
    carry = t >> 32;
  }
  return r;
}

static uint32_t inv_mod(uint32_t a, uint32_t m) {
  // extended Euclid; a and m coprime
  int64_t t = 0, nt = 1, r = m, nr = a % m;
  while (nr) {
    const int64_t q = r / nr;
    std::tie(t, nt) = std::make_tuple(nt, t - q * nt);
    std::tie(r, nr) = std::make_tuple(nr, r - q * nr);
  }
  if (t < 0) t += m;
  return (uint32_t)t;
}

// ---------------------------------------------------------------------------
// The modulus list (Sec. 4.3): for every prime q <= 255 the largest power
// q^k <= 255, in descending order; then the primes in (255, 16191], in
// descending order.
// ---------------------------------------------------------------------------
static const std::vector<uint32_t>& modulus_list() {
  static std::vector<uint32_t> list;
  static std::once_flag once;
  std::call_once(once, [] {
    const int lim = 16191;
    std::vector<char> comp(lim + 1, 0);
    for (int i = 2; i * i <= lim; ++i)
      if (!comp[i])
        for (int j = i * i; j <= lim; j += i) comp[j] = 1;
    std::vector<uint32_t> one;
    for (int q = 2; q <= 255; ++q) {
      if (comp[q]) continue;
      int m = q;
      while (m * q <= 255) m *= q;
      one.push_back((uint32_t)m);
    }
    std::sort(one.rbegin(), one.rend());
    list = one;
    for (int m = lim; m > 255; --m)
      if (!comp[m]) list.push_back((uint32_t)m);
  });
  return list;
}
static int one_limb_count() {
  static int n = [] {
    int c = 0;
    for (uint32_t m : modulus_list()) c += m <= 255;
    return c;
  }();
  return n;
}

static int ceil_log2(int64_t k) {
  int c = 0;
  while (((int64_t)1 << c) < k) ++c;
  return c;
}

// Allocation failures injected on the host by ozaki2_debug_inject_alloc_failure:
// the next `count` library allocations (host plan construction, device tables,
// launch images) report OZ2_ENOMEM without allocating.
static std::atomic<int> g_inject_alloc{0};
static bool injected_alloc_failure() {
  int c = g_inject_alloc.load();
  while (c > 0)
    if (g_inject_alloc.compare_exchange_weak(c, c - 1)) return true;
  return false;
}

// ---------------------------------------------------------------------------
// Plan
// ---------------------------------------------------------------------------
struct CrtHost {
  int L, D32, DS, cls;
  Big P;
  std::vector<uint32_t> words;   // pool layout (see CrtView), DS-padded
  // tensor-core CRT table B [npad][kpad] (bf16 bits): B[j][2l] = M_l[j],
  // B[j][2l+1] = M_l[j-1], M_l[j] the 7-bit pieces of M_l
  int kpad = 0, npad = 0, np = 0, rows = 0;   // rows: table rows allocated (>= npad)
  std::vector<uint16_t> tc_table;
};

// One group of consecutive moduli whose residue planes are computed and
// multiplied together when a product streams its planes through a bounded
// workspace (the moduli are independent, Sec. 2.3; the paper runs them as
// separate plane GEMMs, Sec. 5.1).
struct GroupHost {
  int l0, L, L1, G;                       // first modulus, moduli, one-limb moduli, planes
  int res_npad, res_cw, res_nchunk, res_nabuf, res_key;
};

struct ProbHost {
  int64_t M, N, K;
  int p, nl, t, L, L1, G, W16, D32, Kp, res_cls, crt_cls, DS;
  int tiles_m, tiles_n, nchunks, kchunk;
  int crt_key;                 // index into crt tables
  size_t off_e, off_f, off_pa, off_pb, off_u;   // workspace offsets
  int kind;                    // 0: limb output; 1: binary64 output
  bool skip_a, skip_b;         // planes of that side are written by the caller
  int crt_mode;                // 0: CUDA-core CRT class crt_cls; 1: tensor-core CRT (class crt_cls);
                               // 2: tensor-core sums to R digits, then the finish
  int crt_kpad, crt_npad, crt_np, crt_nchunk, crt_cw, crt_ngrp, crt_nslot, crt_nvbuf;
  int crt_gskip = 0;            // crt_mode 2, long finish: lowest group of Y columns formed
  size_t off_q, off_sig;       // crt_mode 2: group sums [ngrp][9][upitch] uint32, quotient estimates [upitch] uint32
  int res_mode, res_kpad, res_npad, res_key;   // tensor-core residues (table index res_key)
  int res_cw, res_nchunk, res_nabuf;           // res_mode 2: chunk width, chunks, byte buffers
  int nb;                                      // bytes of a (t+1)-bit integer
  std::vector<GroupHost> groups;               // non-empty: planes streamed in these groups
  bool sum_of = false;                         // complex plan: planes are the sums of problems 0 and 1's
  bool no_crt = false;                         // complex plan: no CRT (its v_l feed the combination)
};

// Tensor-core residue table [npad][kpad] (bf16 bits): row l (one-limb) =
// cen(2^(8 b) mod m_l); rows L1 + 2 (l - L1) + {0, 1} (two-limb) = the balanced
// base-128 halves of cen(2^(8 b) mod m_l).
struct ResTable {
  int l0 = 0;                // first modulus (index in the list)
  int L, kpad, npad, rows;   // rows: allocated (npad, or whole chunks of the warp-specialised kernel)
  std::vector<uint16_t> bits;
};

struct ListRef {
  const int32_t* ptr = nullptr;
  int n = 0;
  int smem = 0;      // dynamic shared memory of the launch
  int lmax = 0;      // largest modulus count among its problems
  int na = 0;        // single-problem plans: leading entries of side A (the rest are side B)
};

// Entries of a block list (int4, side in bit 0 of .y) that belong to side A:
// the leading run (single-problem lists hold side A's blocks first).
static int side_a_prefix(const std::vector<int4>& v) {
  int n = 0;
  while (n < (int)v.size() && (v[n].y & 1) == 0) ++n;
  return n;
}

struct PlainSeg {
  int cta_off, grid;
};

struct LaunchBlock {
  void* d_mem = nullptr;       // ProbDev[count], then CUtensorMap[2 count] (64-byte aligned)
  void* h_stage = nullptr;     // pinned staging buffer
  size_t bytes = 0, tmap_off = 0;
  cudaEvent_t copied = nullptr;
  bool pending = false;
  std::vector<uint8_t> last;
};

struct DevState {
  int device = -1, sms = 0;
  void* mem = nullptr;
  DevTables tab{};
  const Unit* unsorted = nullptr;
  ListRef scan_rows, scan_cols, simt, s8;
  ListRef res[6], crt[kCrtClassCount];
  const int32_t* cta_grouped = nullptr;
  int grid = 0;
  const int32_t* cta_plain = nullptr;
  std::vector<PlainSeg> plain;
  std::vector<int> crt_off;    // per problem, uint32 offset in the pool
  ListRef tct[9];               // tensor-core CRT tile lists (smem = kpad_max, lmax = L max)
  int tct_npad[9] = {0};
  std::vector<ListRef> cmt;     // tensor-core CRT sum tiles, one list per TMEM layout (smem = chunk width)
  ListRef finl;                 // finish blocks of long accumulators (smem = D max, lmax = output limbs max)
  ListRef fsh[9];               // finish blocks of one-lane classes after the tensor-core sums
  std::vector<ListRef> rmt;     // warp-specialised tensor-core residue tiles, one list per TMEM layout (smem = cw)
  ListRef rtt;                  // tensor-core residue tiles (smem = kpad_max, lmax = L max)
  int rtt_npad = 0;
  std::vector<void*> res_tab;   // per problem: device address of its residue table
  std::vector<void*> crt_tab;   // per problem: device address of its tensor-core CRT table
  // streamed planes (single problems): per modulus group, the tables of its
  // launches (modulus constants and digit tables from its first modulus on,
  // its own GEMM schedule) and the device address of its residue table
  struct Group {
    DevTables tab{};
    int grid = 0;
    void* res_tab = nullptr;
  };
  std::vector<Group> groups;
};

static void free_launch_block(LaunchBlock& lb) {
  if (lb.copied) cudaEventSynchronize(lb.copied), cudaEventDestroy(lb.copied);
  if (lb.d_mem) cudaFree(lb.d_mem);
  if (lb.h_stage) cudaFreeHost(lb.h_stage);
  lb = LaunchBlock();
}

}  // namespace oz2

struct ozaki2_plan_s {
  ozaki2_opts opts{};
  std::vector<oz2::ProbHost> probs;
  std::vector<oz2::CrtHost> crts;
  std::vector<oz2::ResTable> rtabs;
  int lmax = 0, w16max = 0;
  size_t ws_bytes = 0, ef_bytes = 0;
  int64_t total_units = 0, total_jobs = 0;
  oz2::DevState dev;
  // launch images (problem descriptors + tensor maps) in a small ring: an
  // execute whose image one of them already holds (for example two buffer sets
  // used in turn) reuses it without a copy or a host wait
  static constexpr int kLaunchRing = 4;
  oz2::LaunchBlock lbs[kLaunchRing];
  uint64_t lb_used[kLaunchRing] = {0, 0, 0, 0};
  uint64_t lb_clock = 0;
  std::vector<uint32_t*> dbg_chat;
  std::vector<int32_t*> dbg_prods;
  // stage boundaries: scan, residues, GEMM, CRT, end; [5] between the
  // tensor-core CRT sums and the rest of the CRT stage
  cudaEvent_t ev[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  std::vector<cudaEvent_t> evg;   // streamed planes: before each group's residues and before its GEMM
  bool timed = false;
  bool no_stream = false;         // internal plans whose planes must all stay resident
  uint32_t spin_limit = oz2::kDefaultSpinLimit;   // polls of a bounded device-side wait
  bool tile2 = false;             // plane GEMMs on CTA pairs (256 x 256 tiles)
  bool complex3m = false;         // complex product: problems Ar Br, Ai Bi, (Ar + Ai)(Br + Bi)
  // operand reuse: the last product of a single-problem plan and its workspace,
  // whose row exponents and planes of A (or column exponents and planes of B)
  // a later ozaki2_execute_reuse keeps
  void* last_ws = nullptr;
  ozaki2_problem last_q{};
};

struct ozaki2_graph_s {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  oz2::LaunchBlock lb;
};

namespace oz2 {

cudaError_t init_prep_attributes();
cudaError_t init_gemm_attributes();
cudaError_t init_gemm2_attributes();
cudaError_t init_gemm_s8_attributes();
cudaError_t launch_plane_sum(const DevTables& t, int64_t items_a, int64_t items_b, cudaStream_t s);
cudaError_t launch_combine_complex(const DevTables& t, int64_t items, cudaStream_t s);
cudaError_t init_crt_attributes();

static size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// The shortest prefix of the modulus list with P > inner 2^(2t + 2) (Eq.
// crtcond with the implementation's +2 margin, Sec. 4.3), or exactly force_L
// moduli when force_L > 0 (which must still meet the bound); its length, or
// -1 when the list cannot reach the bound.  *P receives the product.
static int modulus_prefix(int64_t inner, int t, int force_L, Big* P) {
  const Big bound = big_shifted((uint64_t)inner, 2 * t + 2);
  const auto& ml = modulus_list();
  *P = Big{1u};
  int L = 0;
  while (force_L > 0 ? L < force_L : big_cmp(*P, bound) <= 0) {
    if (L >= (int)ml.size()) return -1;
    big_mul_small(*P, ml[L]);
    ++L;
  }
  return big_cmp(*P, bound) <= 0 ? -1 : L;
}

// Tensor-core residue table [rows][kpad] (f16 bits) of the moduli
// l0 .. l0 + L - 1 of the list (L1 of them one-limb): row l (one-limb) =
// cen(2^(8 b) mod m), rows L1 + 2 (l - L1) + {0, 1} (two-limb) = the balanced
// base-128 halves of cen(2^(8 b) mod m).  Shared by problems and modulus
// groups with the same moduli and geometry; returns its index in pl->rtabs.
static int res_table_key(ozaki2_plan_s* pl, int l0, int L, int L1, int nb, int kpad, int npad, int rows) {
  for (size_t i = 0; i < pl->rtabs.size(); ++i) {
    const ResTable& r = pl->rtabs[i];
    if (r.l0 == l0 && r.L == L && r.kpad == kpad && r.rows == rows) return (int)i;
  }
  ResTable rt;
  rt.l0 = l0; rt.L = L; rt.kpad = kpad; rt.npad = npad; rt.rows = rows;
  rt.bits.assign((size_t)rows * kpad, 0);
  auto bf = [](int x) -> uint16_t {   // f16 bits of an integer |x| <= 2048 (exact)
    if (x == 0) return 0;
    const uint16_t sgn = x < 0 ? 0x8000u : 0u;
    const uint32_t a = (uint32_t)(x < 0 ? -x : x);
    int e = 0;
    while ((a >> (e + 1)) != 0u) ++e;           // a in [2^e, 2^(e+1))
    return (uint16_t)(sgn | (uint32_t)(e + 15) << 10 | ((a << (10 - e)) & 0x3FFu));
  };
  const auto& mlist = modulus_list();
  for (int l = 0; l < L; ++l) {
    const int m = (int)mlist[l0 + l];
    int64_t pw = 1 % m;                          // 2^(8 b) mod m
    for (int b = 0; b < nb; ++b) {
      int c = (int)pw;
      if (2 * c > m) c -= m;                     // centered
      if (l < L1) {
        rt.bits[(size_t)l * kpad + b] = bf(c);
      } else {
        int y = c & 127;
        const int lo = y > 64 ? y - 128 : y;
        const int hi = (c - lo) / 128;
        const int r0 = L1 + 2 * (l - L1);
        rt.bits[(size_t)r0 * kpad + b] = bf(lo);
        rt.bits[(size_t)(r0 + 1) * kpad + b] = bf(hi);
      }
      pw = (pw << 8) % m;
    }
  }
  pl->rtabs.push_back(std::move(rt));
  return (int)pl->rtabs.size() - 1;
}

// One problem of a plan.  `po` (batched plans) supplies this problem's own
// guard bits, t, K chunk and residue and CRT engines; the plan's options
// otherwise.
static int build_problem(ozaki2_plan_s* pl, int64_t M, int64_t N, int64_t K, int p,
                         const PlanExtra* ex = nullptr, const ozaki2_opts* po = nullptr) {
  const ozaki2_opts& o = po ? *po : pl->opts;
  const PlanExtra none{};
  if (!ex) ex = &none;
  if (injected_alloc_failure()) throw std::bad_alloc();
  if (M <= 0 || N <= 0 || K <= 0 || p < 2) return OZ2_EINVAL;
  if (K > kMaxK || p > kMaxP) return OZ2_ERANGE;
  if (M > 65535LL * kBM || N > 65535LL * kBN) return OZ2_ERANGE;
  ProbHost h{};
  h.M = M; h.N = N; h.K = K; h.p = p;
  h.nl = (p + 63) / 64;
  const int64_t inner = std::max<int64_t>(K, ex->inner);
  h.t = ex->force_t > 0 ? ex->force_t
                        : (o.t_bits > 0 ? o.t_bits : p + o.guard_bits + ceil_log2(inner));   // Eq. 3
  if (h.t > kMaxP + 64) return OZ2_ERANGE;
  Big P;
  const int L = modulus_prefix(inner, h.t, ex->force_L, &P);
  if (L < 0) return OZ2_ERANGE;
  const auto& ml = modulus_list();
  h.kind = ex->kind;
  h.skip_a = ex->skip_a;
  h.skip_b = ex->skip_b;
  h.L = L;
  h.L1 = std::min(L, one_limb_count());
  h.G = h.L1 + 3 * (L - h.L1);
  h.W16 = (h.t + 1 + 15) / 16;
  h.res_cls = residue_class_for(h.W16);
  if (h.res_cls < 0) return OZ2_ERANGE;
  h.D32 = (big_bitlen(P) + 31) / 32 + 2;   // headroom: S < L P (Sec. 5.4)
  h.crt_cls = crt_class_for(h.D32);
  if (h.crt_cls < 0) return OZ2_ERANGE;
  h.DS = crt_class_digits(h.crt_cls);
  h.Kp = (int)align_up((size_t)K, 8);
  const int tile_rows = pl->tile2 ? 2 * kBM : kBM;     // rows of a plane GEMM output tile
  h.tiles_m = (int)((M + tile_rows - 1) / tile_rows);
  h.tiles_n = (int)((N + kBN - 1) / kBN);
  const int kc = o.k_chunk > 0 ? o.k_chunk : kMaxKChunk;
  if (kc % kBK != 0 || kc > kMaxKChunk) return OZ2_EINVAL;
  h.kchunk = kc;
  h.nchunks = (int)((K + kc - 1) / kc);
  // CRT tables, shared by problems with the same modulus count
  int key = -1;
  for (size_t i = 0; i < pl->crts.size(); ++i)
    if (pl->crts[i].L == L) key = (int)i;
  if (key < 0) {
    CrtHost c;
    c.L = L; c.D32 = h.D32; c.DS = h.DS; c.cls = h.crt_cls; c.P = P;
    const int DS = c.DS, D = c.D32;
    c.words.assign((size_t)3 * DS + L + (size_t)L * DS, 0u);
    for (int i = 0; i < (int)P.size(); ++i) c.words[i] = P[i];
    const Big negP = big_neg_mod(P, D);
    for (int i = 0; i < D; ++i) c.words[DS + i] = negP[i];
    Big H1;
    big_divmod_small(P, 2, &H1);               // floor(P / 2) ...
    uint64_t carry = 1;                        // ... + 1
    for (auto& dg : H1) {
      const uint64_t t = (uint64_t)dg + carry;
      dg = (uint32_t)t;
      carry = t >> 32;
      if (!carry) break;
    }
    if (carry) H1.push_back(1u);
    const Big negH1 = big_neg_mod(H1, D);
    for (int i = 0; i < D; ++i) c.words[2 * DS + i] = negH1[i];
    for (int l = 0; l < L; ++l) {
      Big Ml;
      const uint32_t m = ml[l];
      big_divmod_small(P, m, &Ml);                       // M_l = P / m_l
      const uint32_t r = big_divmod_small(Ml, m, nullptr);
      c.words[3 * DS + l] = inv_mod(r, m);               // M_l^{-1} mod m_l
      for (int i = 0; i < (int)Ml.size(); ++i) c.words[3 * DS + L + (size_t)l * DS + i] = Ml[i];
    }
    pl->crts.push_back(std::move(c));
    key = (int)pl->crts.size() - 1;
  }
  h.crt_key = key;
  {
    CrtHost& c = pl->crts[key];
    const int np = (big_bitlen(c.P) + 6) / 7 + 1;
    const int kpad = (int)align_up((size_t)2 * L, 64);
    const int npad = (int)align_up((size_t)np, 16);
    // the tensor-core sums carry five more columns at the end of their last
    // 32-column group: the 7-bit pieces of floor(2^28 / m_l), whose column
    // sums give the quotient estimate
    const int npad_mm = (int)align_up((size_t)np + 5, 32);
    const bool tc_ok = o.crt_engine == 1 && h.crt_cls <= 8 && kpad <= 256 && npad <= 256 &&
                       crt_tc_smem_bytes(h.crt_cls, kpad, npad, L, 1) <= 227 * 1024;
    // automatic choice: the tensor-core sums above 20 accumulator digits
    // (measured at 1024^3: 0.238 vs 0.248 ms at 21 digits, 0.27 vs 0.33 at 25,
    // 0.42 vs 0.67 at 33; 0.21 vs 0.18 at 17), the one-lane CUDA-core CRT below
    const bool want_mm = o.crt_engine == 2 || (o.crt_engine == 0 && h.D32 > 20);
    // sums of any length: fp32 column sums exact for 2L 127^2 < 2^24, and V
    // for 128 outputs (kpad bf16 each) plus the rings must fit in shared memory
    // (the u copies are boxes of 32 moduli x 128 outputs: at least that many;
    // V takes kpad / 2 of the 512 TMEM columns, two accumulator slots the rest)
    const bool mm_ok = want_mm && 2 * L * 127 * 127 < (1 << 24) && L >= 32 && M * N >= 128 &&
                       kpad / 2 + 2 * 32 <= 512;
    h.crt_mode = tc_ok ? 1 : (mm_ok ? 2 : 0);
    h.crt_kpad = kpad;
    h.crt_npad = h.crt_mode == 2 ? npad_mm : npad;
    h.crt_np = np;
    h.crt_nslot = 2;
    h.crt_cw = mm_ok ? crt_mm_chunk(kpad, npad_mm, &h.crt_nslot) : 0;
    h.crt_nchunk = mm_ok ? (npad_mm + h.crt_cw - 1) / h.crt_cw : 0;
    // a second V buffer where it fits beside the accumulator slots: the
    // next tile's V is built while this tile's chunks are read out
    h.crt_nvbuf = (mm_ok && kpad + h.crt_nslot * h.crt_cw <= 512) ? 2 : 1;
    h.crt_ngrp = mm_ok ? h.crt_nchunk * h.crt_cw / 32 : 0;
    const int rows = h.crt_mode == 2 ? h.crt_cw * h.crt_nchunk : npad;
    // The finish of long accumulators reads the group sums from group g0 - 1
    // on in its fast form (g0: the group whose lowest digit lies just below
    // its window of the 2 nl + 4 highest digits), and takes an output's full
    // form from v_l where the fast form does not stand: the sums below group
    // g0 - 1 are not formed (the table keeps every row).
    h.crt_gskip = 0;
    if (h.crt_mode == 2 && h.crt_cls > 4 && h.D32 <= kCrtSkipMaxDigits) {
      const int W = 2 * h.nl + 4, wbase = h.D32 > W ? h.D32 - W : 0;
      const int g0 = wbase > 7 ? (wbase - 1) / 7 : 0;
      if (g0 >= 2) {
        h.crt_gskip = g0 - 1;
        h.crt_nchunk = (npad_mm - 32 * h.crt_gskip + h.crt_cw - 1) / h.crt_cw;
        h.crt_ngrp = h.crt_nchunk * h.crt_cw / 32;
      }
    }
    CrtHost* cp = &c;
    if (h.crt_mode != 0 && !c.tc_table.empty() && (c.rows != rows || c.npad != h.crt_npad)) {
      // another problem of this modulus set runs the other tensor-core CRT
      // form: a table of this form exists already, or this problem gets a copy
      // of the digit tables with its own
      int other = -1;
      for (size_t i = 0; i < pl->crts.size(); ++i)
        if (pl->crts[i].L == L && pl->crts[i].rows == rows && pl->crts[i].npad == h.crt_npad) other = (int)i;
      if (other < 0) {
        CrtHost cc;
        cc.L = c.L; cc.D32 = c.D32; cc.DS = c.DS; cc.cls = c.cls; cc.P = c.P; cc.words = c.words;
        pl->crts.push_back(std::move(cc));
        other = (int)pl->crts.size() - 1;
      }
      h.crt_key = other;
      cp = &pl->crts[other];
    }
    CrtHost& c2 = *cp;
    if (h.crt_mode != 0 && c2.tc_table.empty()) {
      CrtHost& c = c2;
      c.kpad = kpad; c.npad = h.crt_npad; c.np = np; c.rows = rows;
      c.tc_table.assign((size_t)rows * kpad, 0);
      const auto& mlist = modulus_list();
      auto bf = [](uint32_t x) -> uint16_t {   // exact for x <= 256
        float f = (float)x;
        uint32_t u;
        std::memcpy(&u, &f, 4);
        return (uint16_t)(u >> 16);
      };
      for (int l = 0; l < L; ++l) {
        Big Ml;
        big_divmod_small(c.P, mlist[l], &Ml);
        std::vector<uint32_t> piece(np + 1, 0u);
        for (int j = 0; j < np; ++j) {
          const int bit = 7 * j, w = bit / 32, sh = bit % 32;
          uint64_t x = w < (int)Ml.size() ? Ml[w] : 0u;
          if (w + 1 < (int)Ml.size()) x |= (uint64_t)Ml[w + 1] << 32;
          piece[j] = (uint32_t)(x >> sh) & 127u;
        }
        for (int j = 0; j < np; ++j) {
          c.tc_table[(size_t)j * kpad + 2 * l] = bf(piece[j]);
          c.tc_table[(size_t)j * kpad + 2 * l + 1] = j ? bf(piece[j - 1]) : 0;
        }
        if (h.crt_mode == 2) {
          // columns npad_mm - 5 .. npad_mm - 1: F_l = floor(2^28 / m_l) < 2^24
          // in four 7-bit pieces, so that sum_k 128^k Y_k = sum_l v_l F_l
          const uint32_t F = (uint32_t)((1u << 28) / mlist[l]);
          const int ca = npad_mm - 5;
          for (int k = 0; k < 5; ++k) {
            const uint32_t f0 = k < 4 ? (F >> (7 * k)) & 127u : 0u;
            const uint32_t f1 = k >= 1 ? (F >> (7 * (k - 1))) & 127u : 0u;
            c.tc_table[(size_t)(ca + k) * kpad + 2 * l] = bf(f0);
            c.tc_table[(size_t)(ca + k) * kpad + 2 * l + 1] = bf(f1);
          }
        }
      }
    }
  }
  {
    // tensor-core residues (byte GEMM); opt-in through opts.res_engine
    const int nb = (h.t + 1 + 7) / 8;
    h.nb = nb;
    const int kpad = (int)align_up((size_t)nb, 64);
    const int npad = (int)align_up((size_t)(h.L1 + 2 * (L - h.L1)), 16);
    h.res_mode = (o.res_engine == 1 && kpad <= 256 && npad <= 256 &&
                  residue_tc_smem_bytes(kpad, npad, L) <= 227 * 1024) ? 1 : 0;
    // warp-specialised form: two byte buffers (kpad / 2 TMEM columns each) and
    // two slots of at least 32 columns; sums exact for <= 512 bytes.  The
    // automatic choice takes it where the dp4a kernel would need its 68-digit
    // class or more (integers of more than 72 bytes): measured at 84 bytes,
    // 0.99 ms against 1.59 ms at 1024^3; at 68 bytes dp4a wins, 0.62 vs 0.84
    const bool want_rmm = o.res_engine == 2 || (o.res_engine == 0 && residue_class_w16(h.res_cls) > 36);
    if (want_rmm && kpad + 64 <= 512) h.res_mode = 2;
    h.res_kpad = kpad;
    h.res_npad = npad;
    h.res_cw = h.res_nchunk = 0;
    h.res_nabuf = 0;
    if (h.res_mode == 2) {
      residue_mm_geometry(kpad, npad, &h.res_cw, &h.res_nabuf);
      h.res_nchunk = (npad + h.res_cw - 1) / h.res_cw;
    }
    const int rows = h.res_mode == 2 ? h.res_cw * h.res_nchunk : npad;
    h.res_key = h.res_mode ? res_table_key(pl, 0, L, h.L1, nb, kpad, npad, rows) : -1;
  }
  pl->probs.push_back(h);
  pl->lmax = std::max(pl->lmax, L);
  pl->w16max = std::max(pl->w16max, residue_class_w16(h.res_cls));
  pl->total_units += (int64_t)L * h.tiles_m * h.tiles_n;
  pl->total_jobs += (int64_t)h.G * h.tiles_m * h.tiles_n * h.nchunks;
  return OZ2_OK;
}

// Bytes of bf16 plane stacks (A and B) above which a single product streams
// its planes in groups of moduli when opts.plane_group is 0.
constexpr size_t kAutoPlaneBudget = (size_t)32 << 30;

// Split the moduli of a single-product plan into as few groups of
// consecutive moduli with at most gmax planes each as the plane counts allow,
// of about equal size (a group that holds two-limb moduli holds an even number
// of one-limb ones), so that only one group's residue planes live in the
// workspace at a time.
static int plan_groups(ozaki2_plan_s* pl) {
  if (pl->probs.size() != 1 || pl->no_stream) return OZ2_OK;
  ProbHost& h = pl->probs[0];
  h.groups.clear();
  const ozaki2_opts& o = pl->opts;
  if (o.plane_group < 0) return OZ2_OK;
  const size_t per_plane = 2 * (size_t)(h.M + h.N) * (size_t)h.Kp;
  int gmax = o.plane_group;
  if (gmax == 0) {
    if (per_plane * (size_t)h.G <= kAutoPlaneBudget) return OZ2_OK;
    gmax = (int)std::max<size_t>(3, kAutoPlaneBudget / per_plane);
  }
  if (o.engine != OZ2_ENGINE_TC || o.schedule != OZ2_SCHED_GROUPED) {
    return o.plane_group > 0 ? OZ2_EINVAL : OZ2_OK;   // streaming runs the grouped tensor-core GEMM
  }
  if (gmax >= h.G) return OZ2_OK;
  const int ng = (h.G + gmax - 1) / gmax;
  const auto& ml = modulus_list();
  // greedy groups with at most `cap` planes each; the smallest cap from
  // ceil(G / ng) up to gmax that gives ng groups (the 3-plane two-limb moduli
  // can leave a small last group at the even split)
  auto split = [&](int cap, std::vector<GroupHost>& out) {
    out.clear();
    int l = 0;
    while (l < h.L) {
      GroupHost gr{};
      gr.l0 = l;
      while (l < h.L) {
        const int planes = ml[l] <= 255 ? 1 : 3;
        if (gr.G > 0 && gr.G + planes > cap) break;
        // the tensor-core residue epilogue takes two-limb pairs at even table
        // columns: a group with two-limb moduli holds an even number of one-limb ones
        if (planes == 3 && (gr.L1 & 1)) break;
        gr.G += planes;
        gr.L1 += planes == 1;
        ++gr.L;
        ++l;
      }
      out.push_back(gr);
    }
  };
  // the tensor-core residues run a group's table columns in chunks, and a
  // nearly empty last chunk costs a whole round of MMAs and epilogue: the
  // automatic split takes, among the caps that give ng groups, the one with
  // the fewest chunks in all (then the smallest largest group); an explicit
  // plane_group keeps the smallest such cap
  auto chunks = [&](const std::vector<GroupHost>& gs) {
    int n = 0;
    for (const GroupHost& gr : gs) {
      const int npad = (int)align_up((size_t)(gr.L1 + 2 * (gr.L - gr.L1)), 16);
      int cw = 0, nab = 0;
      residue_mm_geometry(h.res_kpad, npad, &cw, &nab);
      n += (npad + cw - 1) / cw;
    }
    return n;
  };
  const bool by_chunks = o.plane_group == 0 && h.res_mode == 2;
  std::vector<GroupHost> groups, trial;
  int best_chunks = INT_MAX, best_max = INT_MAX;
  for (int cap = (h.G + ng - 1) / ng; cap <= gmax; ++cap) {
    split(cap, trial);
    if ((int)trial.size() > ng) continue;
    if (!by_chunks) {
      groups = trial;
      break;
    }
    int gm = 0;
    for (const GroupHost& gr : trial) gm = std::max(gm, gr.G);
    const int nc = chunks(trial);
    if (nc < best_chunks || (nc == best_chunks && gm < best_max)) {
      best_chunks = nc;
      best_max = gm;
      groups = trial;
    }
  }
  if (groups.empty()) split(gmax, groups);
  for (GroupHost& gr : groups) {
    gr.res_npad = (int)align_up((size_t)(gr.L1 + 2 * (gr.L - gr.L1)), 16);
    gr.res_cw = gr.res_nchunk = gr.res_nabuf = 0;
    gr.res_key = -1;
    if (h.res_mode == 2) {
      residue_mm_geometry(h.res_kpad, gr.res_npad, &gr.res_cw, &gr.res_nabuf);
      gr.res_nchunk = (gr.res_npad + gr.res_cw - 1) / gr.res_cw;
    }
    if (h.res_mode != 0) {
      const int rows = h.res_mode == 2 ? gr.res_cw * gr.res_nchunk : gr.res_npad;
      gr.res_key = res_table_key(pl, gr.l0, gr.L, gr.L1, h.nb, h.res_kpad, gr.res_npad, rows);
    }
  }
  if (groups.size() > 1) h.groups = std::move(groups);
  return OZ2_OK;
}

static int group_planes_max(const ProbHost& h) {
  int g = 0;
  for (const GroupHost& gr : h.groups) g = std::max(g, gr.G);
  return h.groups.empty() ? h.G : g;
}

static void layout_workspace(ozaki2_plan_s* pl) {
  size_t off = 0;
  for (auto& h : pl->probs) { h.off_e = off; off += align_up(4 * (size_t)h.M, 256); }
  for (auto& h : pl->probs) { h.off_f = off; off += align_up(4 * (size_t)h.N, 256); }
  pl->ef_bytes = off;
  for (auto& h : pl->probs) {
    const int gp = group_planes_max(h);   // planes resident at a time
    h.off_pa = off; off += align_up(2 * (size_t)gp * h.M * h.Kp, 256);
    h.off_pb = off; off += align_up(2 * (size_t)gp * h.N * h.Kp, 256);
    h.off_u = off; off += align_up(2 * (size_t)h.L * align_up((size_t)(h.M * h.N), 8), 256);
    h.off_q = h.off_sig = off;
    if (h.crt_mode == 2) {
      const size_t up = align_up((size_t)(h.M * h.N), 8);
      off += align_up(4 * (size_t)h.crt_ngrp * 9 * up, 256);
      h.off_sig = off;
      off += align_up(4 * up, 256);               // quotient estimates
    }
  }
  pl->ws_bytes = off;
}

// Automatic plane GEMM tile of a single product: CTA pairs (256 x 256) where
// both output dimensions exceed one 128-row tile and the plane products are
// below 1e13 flop; one SM per 128 x 256 tile for larger products, where the
// pairs measured slower on one GB300 (1024^3 at p = 256: 0.180 vs 0.188 ms,
// 4096^3 at p = 53: 2.07 vs 2.16 ms; 8192^3 at p = 53: 17.3 vs 17.0 ms,
// 4096^3 at p = 2048: 82.2 vs 77.7 ms).
static bool auto_pair_tiles(ozaki2_plan_s* pl, int64_t M, int64_t N, int64_t K, int p) {
  if (M <= 128 || N <= 128 || p < 2 || K <= 0 || K > kMaxK || p > kMaxP) return false;
  // planes G from the modulus rule (Eq. 3 and Eq. crtcond), without building the plan
  const ozaki2_opts& o = pl->opts;
  const int t = o.t_bits > 0 ? o.t_bits : p + o.guard_bits + ceil_log2(K);
  Big P;
  const int L = modulus_prefix(K, t, 0, &P);
  if (L < 0) return false;
  const int L1 = std::min(L, one_limb_count());
  const double G = L1 + 3.0 * (L - L1);
  return 2.0 * (double)M * (double)N * (double)K * G < 1e13;
}

static int new_plan(const ozaki2_opts* opts, ozaki2_plan_s** res) {
  auto* pl = new (std::nothrow) ozaki2_plan_s();
  if (!pl) return OZ2_ENOMEM;
  if (opts) pl->opts = *opts;
  else ozaki2_opts_default(&pl->opts);
  const ozaki2_opts& o = pl->opts;
  if (o.guard_bits < 0 || o.t_bits < 0 || o.grid < 0 || o.k_chunk < 0 ||
      (o.engine != OZ2_ENGINE_TC && o.engine != OZ2_ENGINE_SIMT && o.engine != OZ2_ENGINE_S8) ||
      (o.schedule != OZ2_SCHED_GROUPED && o.schedule != OZ2_SCHED_PLAIN) ||
      (o.crt_engine < 0 || o.crt_engine > 3) || (o.res_engine < 0 || o.res_engine > 3) ||
      o.plane_group < -1 || (o.plane_group > 0 && o.plane_group < 3) || o.gemm_tile < 0 || o.gemm_tile > 2) {
    delete pl;
    return OZ2_EINVAL;
  }
  pl->tile2 = o.engine == OZ2_ENGINE_TC && o.gemm_tile == 2;   // automatic: decided per plan (plan_tile)
  *res = pl;
  return OZ2_OK;
}

// ---------------------------------------------------------------------------
// Device side of a plan
// ---------------------------------------------------------------------------
static PFN_cuTensorMapEncodeTiled_v12000 get_encode() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

struct Builder {
  std::vector<uint8_t> img;
  size_t add(const void* p, size_t n, size_t align = 256) {
    const size_t off = align_up(img.size(), align);
    img.resize(off + std::max<size_t>(n, 1));
    if (p && n) std::memcpy(img.data() + off, p, n);
    return off;
  }
};

// Offsets of the device tables inside one image (see upload()).
struct TableImage {
  Builder b;
  size_t o_mods = 0, o_t16 = 0, o_pool = 0, o_units = 0, o_ordered = 0, o_ctag = 0, o_ctap = 0,
         o_srows = 0, o_scols = 0, o_simt = 0, o_s8 = 0, o_status = 0;
  size_t o_res[6] = {0}, o_crt[kCrtClassCount] = {0};
  int n_srows = 0, n_scols = 0, n_simt = 0, n_s8 = 0, n_res[6] = {0}, n_crt[kCrtClassCount] = {0};
  int res_l[6] = {0}, crt_l[kCrtClassCount] = {0};
  int grid = 0;
  // tensor-core CRT: tile lists per one-lane class, table offsets per CRT key
  size_t o_tct[9] = {0};
  int n_tct[9] = {0}, tct_kpad[9] = {0}, tct_npad[9] = {0}, tct_l[9] = {0};
  std::vector<size_t> o_tctab;
  // tensor-core CRT sum tiles and warp-specialised tensor-core residue
  // tiles: one launch per TMEM layout, {first tile, tiles, chunk width}
  size_t o_cmt = 0, o_finl = 0;
  std::vector<std::array<int, 3>> cmt_seg, rmt_seg;
  size_t o_fsh[9] = {0};            // short finish blocks per one-lane class (after the tensor-core sums)
  int n_fsh[9] = {0};
  int n_finl = 0, finl_dmax = 0, finl_nlmax = 0;
  size_t o_rmt = 0;
  size_t o_rtt = 0;                 // tensor-core residue tile list
  int n_rtt = 0, rtt_kpad = 0, rtt_npad = 0, rtt_l = 0;
  std::vector<size_t> o_rtab;
  int na_srows = 0, na_res[6] = {0}, na_rtt = 0;   // side-A prefixes of the lists
  std::vector<int> na_rmt;
  size_t o_ctas = 0;                // per-group CTA unit ranges (streamed planes)
  std::vector<std::array<int, 2>> grp;   // {offset into the range array, grid} per group
};

// Host side of the device upload: modulus constants, residue digit tables,
// CRT tables, the unit schedule and the block lists of every stage, as one
// byte image.  Fills the plan's host-side launch facts (grid, plain
// segments, CRT offsets).
static int build_table_image(ozaki2_plan_s* pl, int sms, TableImage& ti) {
  DevState& d = pl->dev;
  d.sms = sms;
  const int count = (int)pl->probs.size();
  const auto& ml = modulus_list();

  // modulus constants and the 2^(16 d) mod m tables (Sec. 5.3)
  std::vector<ModConst> mods(pl->lmax);
  for (int l = 0; l < pl->lmax; ++l) {
    const uint32_t m = ml[l];
    ModConst& c = mods[l];
    c.m = m;
    c.mu = (uint32_t)((1ull << 32) / m);
    c.c24 = (uint32_t)((1ull << 24) % m);
    c.rcp = (float)(1.0 / (double)m);
    if (m > 255) {
      // sum r^a r^b = -127 P0 + 128 Ps + 16256 P2 (Eq. 4); the epilogue keeps
      // the running value scaled by the inverse of the next plane's coefficient
      const uint32_t c0 = (m - 127u) % m, cs = 128u % m, c2 = 16256u % m;
      c.kmul01 = (uint32_t)((uint64_t)c0 * inv_mod(cs, m) % m);
      c.kmul12 = (uint32_t)((uint64_t)cs * inv_mod(c2, m) % m);
      c.kfin = c2;
    } else {
      c.kmul01 = c.kmul12 = c.kfin = 1u;
    }
  }
  // byte tables of the residue kernel: row l holds, packed four bytes per
  // word, the bytes 2^(8 b) mod m_l (one-limb) or, for two-limb moduli, the
  // low bytes of 2^(8 b) mod m_l followed by their high bytes; w16max words
  // per row (room for 2 * (w16max / 2) packed words)
  std::vector<uint32_t> t16((size_t)pl->lmax * pl->w16max, 0u);
  for (int l = 0; l < pl->lmax; ++l) {
    const uint32_t m = ml[l];
    const int w32 = pl->w16max / 2;
    uint64_t v = 1 % m;
    for (int byte = 0; byte < 4 * w32; ++byte) {
      const int w = byte >> 2, sh = 8 * (byte & 3);
      t16[(size_t)l * pl->w16max + w] |= (uint32_t)(v & 255u) << sh;
      if (m > 255) t16[(size_t)l * pl->w16max + w32 + w] |= (uint32_t)(v >> 8) << sh;
      v = (v << 8) % m;
    }
  }
  std::vector<uint32_t> pool;
  std::vector<int> key_off(pl->crts.size());
  for (size_t i = 0; i < pl->crts.size(); ++i) {
    key_off[i] = (int)pool.size();
    pool.insert(pool.end(), pl->crts[i].words.begin(), pl->crts[i].words.end());
    pool.resize(align_up(pool.size(), 64), 0u);
  }
  d.crt_off.resize(count);
  for (int i = 0; i < count; ++i) d.crt_off[i] = key_off[pl->probs[i].crt_key];

  // units in (problem, modulus, tile row, tile col) order; persistent CTA c
  // takes units c, c + grid, ... so that the CTAs running at one time share
  // the planes of a few moduli in L2
  std::vector<Unit> units;
  std::vector<std::pair<int, int>> seg;   // (first unit, count) per (problem, modulus)
  for (int pi = 0; pi < count; ++pi) {
    const ProbHost& h = pl->probs[pi];
    for (int l = 0; l < h.L; ++l) {
      seg.emplace_back((int)units.size(), h.tiles_m * h.tiles_n);
      for (int tm = 0; tm < h.tiles_m; ++tm)
        for (int tn = 0; tn < h.tiles_n; ++tn)
          units.push_back(Unit{(uint16_t)pi, (uint16_t)l, (uint16_t)tm, (uint16_t)tn});
    }
  }
  const int nunits = (int)units.size();
  // scheduling slots: persistent CTAs, or CTA pairs for the 256 x 256 tiles
  const int want = pl->opts.grid > 0 ? pl->opts.grid : d.sms;
  const int slots = pl->tile2 ? std::max(1, want / 2) : want;
  const int grid = std::max(1, std::min(slots, nunits));
  // greedy list scheduling, longest first: every unit goes to the least-loaded
  // CTA, the units in decreasing cost (the two-limb moduli's three-plane units
  // first), each cost class in (problem, modulus, tile) order; the cost of a
  // unit is its accumulation jobs times (K blocks per job + a fixed epilogue
  // share).  Taking the large units first keeps the largest CTA load within
  // one small unit of the mean (1024^3 at p = 256: 440 against a mean of 429.5
  // and 460 in plain unit order).
  std::vector<std::vector<int>> lists(grid);
  {
    std::vector<int64_t> cost(nunits);
    for (int u = 0; u < nunits; ++u) {
      const ProbHost& h = pl->probs[units[u].prob];
      const int planes = units[u].ell < h.L1 ? 1 : 3;
      const int64_t kblocks = (std::min<int64_t>(h.K, h.kchunk) + kBK - 1) / kBK;
      cost[u] = (int64_t)planes * h.nchunks * (kblocks + 4);
    }
    std::vector<int> order(nunits);
    for (int u = 0; u < nunits; ++u) order[u] = u;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost[a] > cost[b]; });
    using Load = std::pair<int64_t, int>;
    std::priority_queue<Load, std::vector<Load>, std::greater<Load>> heap;
    for (int c = 0; c < grid; ++c) heap.push(Load(0, c));
    for (int u : order) {
      Load top = heap.top();
      heap.pop();
      lists[top.second].push_back(u);
      top.first += cost[u];
      heap.push(top);
    }
  }
  std::vector<Unit> ordered;
  ordered.reserve(2 * units.size());
  std::vector<int32_t> cta_g(grid + 1, 0);
  for (int c = 0; c < grid; ++c) {
    cta_g[c] = (int)ordered.size();
    for (int u : lists[c]) ordered.push_back(units[u]);
  }
  cta_g[grid] = (int)ordered.size();
  // plain schedule: one launch per (problem, modulus), appended after the
  // grouped order; each launch has its own [grid + 1] range array
  std::vector<int32_t> cta_p;
  d.plain.clear();
  for (auto& sg : seg) {
    const int first = sg.first, cnt = sg.second;
    const int g = std::max(1, std::min(cnt, pl->tile2 ? d.sms / 2 : d.sms));
    d.plain.push_back(PlainSeg{(int)cta_p.size(), g});
    for (int c = 0; c < g; ++c) {
      cta_p.push_back((int)ordered.size());
      for (int u = c; u < cnt; u += g) ordered.push_back(units[first + u]);
    }
    cta_p.push_back((int)ordered.size());
  }

  // streamed planes: one grouped GEMM schedule per modulus group of the
  // (single) problem, with group-local modulus indices, appended to `ordered`
  std::vector<int32_t> cta_s;
  ti.grp.clear();
  if (count == 1) {
    const ProbHost& h = pl->probs[0];
    for (const GroupHost& gr : h.groups) {
      std::vector<Unit> gu;
      for (int l = 0; l < gr.L; ++l)
        for (int tm = 0; tm < h.tiles_m; ++tm)
          for (int tn = 0; tn < h.tiles_n; ++tn)
            gu.push_back(Unit{0, (uint16_t)l, (uint16_t)tm, (uint16_t)tn});
      const int gg = std::max(1, std::min(slots, (int)gu.size()));
      std::vector<std::vector<int>> gl(gg);
      using Load = std::pair<int64_t, int>;
      std::priority_queue<Load, std::vector<Load>, std::greater<Load>> heap;
      for (int c = 0; c < gg; ++c) heap.push(Load(0, c));
      const int64_t kblocks = (std::min<int64_t>(h.K, h.kchunk) + kBK - 1) / kBK;
      std::vector<int> order;                      // longest first, as above
      for (int pass = 0; pass < 2; ++pass)
        for (int u = 0; u < (int)gu.size(); ++u)
          if ((gu[u].ell < gr.L1) == (pass == 1)) order.push_back(u);
      for (int u : order) {
        const int planes = gu[u].ell < gr.L1 ? 1 : 3;
        Load top = heap.top();
        heap.pop();
        gl[top.second].push_back(u);
        top.first += (int64_t)planes * h.nchunks * (kblocks + 4);
        heap.push(top);
      }
      ti.grp.push_back({(int)cta_s.size(), gg});
      for (int c = 0; c < gg; ++c) {
        cta_s.push_back((int)ordered.size());
        for (int u : gl[c]) ordered.push_back(gu[u]);
      }
      cta_s.push_back((int)ordered.size());
    }
  }

  // block lists
  std::vector<int4> scan_rows, scan_cols, simt;
  std::vector<std::vector<int4>> res(6), crt(kCrtClassCount), tct(9), fsh(9);
  std::vector<int4> rtt, finl;
  // tiles of the warp-specialised kernels grouped by TMEM layout (tiles of
  // one launch share the column map of their buffers and slots)
  std::map<std::array<int, 3>, std::vector<int4>> cmt_by, rmt_by;
  for (int pi = 0; pi < count; ++pi) {
    const ProbHost& h = pl->probs[pi];
    const bool own_planes = !h.sum_of;             // planes made by the scan and residue kernels
    if (!h.skip_a && own_planes) {
      // rows of A: 8 rows per block, K split into parts of >= 256 (maxima combined by atomicMax)
      const int rparts = (int)std::max<int64_t>(1, std::min<int64_t>(64, h.K / 256));
      for (int64_t r = 0; r < h.M; r += 8)
        for (int kp = 0; kp < rparts; ++kp) scan_rows.push_back(make_int4(pi, kp << 8, (int)r, rparts));
    }
    // columns of B: 32 columns per block, K split into parts of >= 64
    const int kparts = (int)std::max<int64_t>(1, std::min<int64_t>(64, h.K / 64));
    if (!h.skip_b && own_planes)
      for (int64_t c = 0; c < h.N; c += 32)
        for (int kp = 0; kp < kparts; ++kp) scan_cols.push_back(make_int4(pi, 1 | (kp << 8), (int)c, kparts));
    for (int side = 0; h.res_mode == 2 && side < 2 && own_planes; ++side) {
      if (side == 0 ? h.skip_a : h.skip_b) continue;
      const int64_t R = side ? h.N : h.M;
      std::vector<int4>& rl = rmt_by[{h.res_kpad, h.res_cw, h.res_nabuf}];
      for (int64_t r = 0; r < R; r += 4)
        for (int64_t k = 0; k < h.K; k += 32) rl.push_back(make_int4(pi, side, (int)r, (int)k));
    }
    for (int side = 0; h.res_mode == 1 && side < 2 && own_planes; ++side) {
      if (side == 0 ? h.skip_a : h.skip_b) continue;
      const int64_t R = side ? h.N : h.M;
      for (int64_t r = 0; r < R; r += 4)
        for (int64_t k = 0; k < h.K; k += 32) rtt.push_back(make_int4(pi, side, (int)r, (int)k));
      ti.rtt_kpad = std::max(ti.rtt_kpad, h.res_kpad);
      ti.rtt_npad = std::max(ti.rtt_npad, h.res_npad);
      ti.rtt_l = std::max(ti.rtt_l, h.L);
    }
    for (int side = 0; h.res_mode == 0 && side < 2 && own_planes; ++side) {
      if (side == 0 ? h.skip_a : h.skip_b) continue;
      const int64_t R = side ? h.N : h.M;
      for (int64_t r = 0; r < R; r += 8)
        for (int64_t k = 0; k < h.K; k += 32 * residue_class_ept(h.res_cls))
          res[h.res_cls].push_back(make_int4(pi, side, (int)r, (int)k));
    }
    if (h.res_mode == 0 && own_planes) ti.res_l[h.res_cls] = std::max(ti.res_l[h.res_cls], h.L);
    if (h.no_crt) {
      // no CRT for this problem
    } else if (h.crt_mode == 1) {
      const int64_t nt = (h.M * h.N + 127) / 128;
      if (nt > INT_MAX) return OZ2_ERANGE;
      for (int64_t tt = 0; tt < nt; ++tt) tct[h.crt_cls].push_back(make_int4(pi, (int)tt, 0, 0));
      ti.tct_kpad[h.crt_cls] = std::max(ti.tct_kpad[h.crt_cls], h.crt_kpad);
      ti.tct_npad[h.crt_cls] = std::max(ti.tct_npad[h.crt_cls], h.crt_npad);
      ti.tct_l[h.crt_cls] = std::max(ti.tct_l[h.crt_cls], h.L);
    } else if (h.crt_mode == 2) {
      // sums on the tensor cores, then the finish from the group sums: R in
      // registers up to 24 digits (k_crt_fin_short, every group word loaded
      // at once), else digit-serial passes over the group words with a window
      // of the highest digits in shared memory (k_crt_fin_long, its fast form
      // from the group below the window on)
      const int64_t nt = (h.M * h.N + 127) / 128;
      if (nt > INT_MAX) return OZ2_ERANGE;
      std::vector<int4>& cl = cmt_by[{h.crt_kpad, h.crt_cw, h.crt_nslot}];
      for (int64_t tt = 0; tt < nt; ++tt) cl.push_back(make_int4(pi, (int)tt, 0, 0));
      if (h.crt_cls <= 4) {
        for (int64_t bb = 0; bb < nt; ++bb) fsh[h.crt_cls].push_back(make_int4(pi, (int)bb, 0, 0));
      } else {
        for (int64_t bb = 0; bb < nt; ++bb) finl.push_back(make_int4(pi, (int)bb, 0, 0));
        ti.finl_dmax = std::max(ti.finl_dmax, h.D32);
        ti.finl_nlmax = std::max(ti.finl_nlmax, h.nl);
      }
    } else {
      const int epb = crt_class_elems_per_block(h.crt_cls);
      const int64_t nb = (h.M * h.N + epb - 1) / epb;
      if (nb > INT_MAX) return OZ2_ERANGE;
      for (int64_t bb = 0; bb < nb; ++bb) crt[h.crt_cls].push_back(make_int4(pi, (int)bb, 0, 0));
      ti.crt_l[h.crt_cls] = std::max(ti.crt_l[h.crt_cls], h.L);
    }
  }
  std::vector<int4> s8;
  for (int u = 0; u < nunits; ++u) {
    const ProbHost& h = pl->probs[units[u].prob];
    const int64_t r0 = (int64_t)units[u].tm * kBM, c0 = (int64_t)units[u].tn * kBN;
    if (pl->opts.engine == OZ2_ENGINE_SIMT) {
      for (int sy = 0; sy < kBM / 32; ++sy)
        for (int sx = 0; sx < kBN / 32; ++sx)
          if (r0 + 32 * sy < h.M && c0 + 32 * sx < h.N) simt.push_back(make_int4(u, sy, sx, 0));
    }
    if (pl->opts.engine == OZ2_ENGINE_S8)
      for (int half = 0; half < 2; ++half)
        if (c0 + 128 * half < h.N) s8.push_back(make_int4(u, half, 0, 0));
  }

  ti.o_mods = ti.b.add(mods.data(), mods.size() * sizeof(ModConst));
  ti.o_t16 = ti.b.add(t16.data(), t16.size() * 4);
  ti.o_pool = ti.b.add(pool.data(), pool.size() * 4);
  ti.o_units = ti.b.add(units.data(), units.size() * sizeof(Unit));
  ti.o_ordered = ti.b.add(ordered.data(), ordered.size() * sizeof(Unit));
  ti.o_ctag = ti.b.add(cta_g.data(), cta_g.size() * 4);
  ti.o_ctap = ti.b.add(cta_p.data(), cta_p.size() * 4);
  ti.o_ctas = ti.b.add(cta_s.data(), cta_s.size() * 4);
  // one launch scans rows and columns: the column blocks follow the row blocks
  scan_rows.insert(scan_rows.end(), scan_cols.begin(), scan_cols.end());
  ti.na_srows = side_a_prefix(scan_rows);
  for (int i = 0; i < 6; ++i) ti.na_res[i] = side_a_prefix(res[i]);
  ti.na_rtt = side_a_prefix(rtt);
  scan_cols.clear();
  ti.o_srows = ti.b.add(scan_rows.data(), scan_rows.size() * 16);
  ti.o_scols = ti.b.add(scan_cols.data(), scan_cols.size() * 16);
  ti.o_simt = ti.b.add(simt.data(), simt.size() * 16);
  ti.o_s8 = ti.b.add(s8.data(), s8.size() * 16);
  ti.n_s8 = (int)s8.size();
  for (int i = 0; i < 6; ++i) ti.o_res[i] = ti.b.add(res[i].data(), res[i].size() * 16);
  for (int i = 0; i < kCrtClassCount; ++i) ti.o_crt[i] = ti.b.add(crt[i].data(), crt[i].size() * 16);
  ti.o_status = ti.b.add(nullptr, 256);
  for (int i = 0; i < 9; ++i) {
    ti.o_tct[i] = ti.b.add(tct[i].data(), tct[i].size() * 16);
    ti.n_tct[i] = (int)tct[i].size();
  }
  // consistency of the launch sizes with the problems they serve
  for (const ProbHost& h : pl->probs) {
    if (h.sum_of || h.no_crt) continue;
    if (h.res_mode == 0 && !(h.skip_a && h.skip_b) && ti.res_l[h.res_cls] < h.L) return OZ2_EINTERNAL;
    if (h.res_mode == 1 && (ti.rtt_l < h.L || ti.rtt_kpad < h.res_kpad || ti.rtt_npad < h.res_npad))
      return OZ2_EINTERNAL;
    if (h.crt_mode == 0 && ti.crt_l[h.crt_cls] < h.L) return OZ2_EINTERNAL;
    if (h.crt_mode == 1 && (ti.tct_l[h.crt_cls] < h.L || ti.tct_kpad[h.crt_cls] < h.crt_kpad)) return OZ2_EINTERNAL;
    if (h.crt_mode == 2 && (h.crt_cw % 32 != 0 || h.crt_nvbuf * (h.crt_kpad / 2) + h.crt_nslot * h.crt_cw > 512 ||
                            (h.crt_cls > 4 && (ti.finl_dmax < h.D32 || ti.finl_nlmax < h.nl))))
      return OZ2_EINTERNAL;
  }
  std::vector<int4> cmt, rmt;
  for (const auto& kv : cmt_by) {
    if (crt_mm_smem_bytes(kv.first[1], pl->lmax, nullptr) < 0) return OZ2_EINTERNAL;
    ti.cmt_seg.push_back({(int)cmt.size(), (int)kv.second.size(), kv.first[1]});
    cmt.insert(cmt.end(), kv.second.begin(), kv.second.end());
  }
  ti.na_rmt.clear();
  for (const auto& kv : rmt_by) {
    if (residue_mm_smem_bytes(kv.first[1], pl->lmax, 512, nullptr) < 0) return OZ2_EINTERNAL;
    ti.rmt_seg.push_back({(int)rmt.size(), (int)kv.second.size(), kv.first[1]});
    ti.na_rmt.push_back(side_a_prefix(kv.second));
    rmt.insert(rmt.end(), kv.second.begin(), kv.second.end());
  }
  if (!finl.empty() && crt_finish_long_smem(ti.finl_dmax, ti.finl_nlmax) > 200 * 1024)
    return OZ2_EINTERNAL;
  ti.o_cmt = ti.b.add(cmt.data(), cmt.size() * 16);
  for (int c = 0; c < 9; ++c) {
    ti.o_fsh[c] = ti.b.add(fsh[c].data(), fsh[c].size() * 16);
    ti.n_fsh[c] = (int)fsh[c].size();
  }
  ti.o_finl = ti.b.add(finl.data(), finl.size() * 16);
  ti.n_finl = (int)finl.size();
  ti.o_rtt = ti.b.add(rtt.data(), rtt.size() * 16);
  ti.n_rtt = (int)rtt.size();
  for (const ProbHost& h : pl->probs)
    if (h.res_mode == 2 && (h.res_cw % 32 != 0 || h.res_nabuf * (h.res_kpad / 2) + 2 * h.res_cw > 512))
      return OZ2_EINTERNAL;
  ti.o_rmt = ti.b.add(rmt.data(), rmt.size() * 16);
  ti.o_rtab.assign(pl->rtabs.size(), 0);
  for (size_t i = 0; i < pl->rtabs.size(); ++i)
    ti.o_rtab[i] = ti.b.add(pl->rtabs[i].bits.data(), pl->rtabs[i].bits.size() * 2, 1024);
  ti.o_tctab.assign(pl->crts.size(), 0);
  for (size_t i = 0; i < pl->crts.size(); ++i)
    if (!pl->crts[i].tc_table.empty())
      ti.o_tctab[i] = ti.b.add(pl->crts[i].tc_table.data(), pl->crts[i].tc_table.size() * 2, 1024);
  ti.n_srows = (int)scan_rows.size();
  ti.n_scols = (int)scan_cols.size();
  ti.n_simt = (int)simt.size();
  for (int i = 0; i < 6; ++i) ti.n_res[i] = (int)res[i].size();
  for (int i = 0; i < kCrtClassCount; ++i) ti.n_crt[i] = (int)crt[i].size();
  ti.grid = grid;
  return OZ2_OK;
}

// Point the plan's device state at a copy of the image at `base`.
static void install_table_image(ozaki2_plan_s* pl, const TableImage& ti, uint8_t* base) {
  DevState& d = pl->dev;
  const int count = (int)pl->probs.size();
  d.tab = DevTables{};
  d.tab.spin_limit = pl->spin_limit;
  d.tab.mods = reinterpret_cast<const ModConst*>(base + ti.o_mods);
  d.tab.t16 = reinterpret_cast<const uint32_t*>(base + ti.o_t16);
  d.tab.w16max = pl->w16max;
  d.tab.lmax = pl->lmax;
  d.tab.crt_pool = reinterpret_cast<const uint32_t*>(base + ti.o_pool);
  d.tab.units = reinterpret_cast<const Unit*>(base + ti.o_ordered);
  d.tab.cta_begin = reinterpret_cast<const int32_t*>(base + ti.o_ctag);
  d.tab.status = reinterpret_cast<int32_t*>(base + ti.o_status);
  d.tab.count = count;
  d.unsorted = reinterpret_cast<const Unit*>(base + ti.o_units);
  d.grid = ti.grid;
  d.cta_grouped = reinterpret_cast<const int32_t*>(base + ti.o_ctag);
  d.cta_plain = reinterpret_cast<const int32_t*>(base + ti.o_ctap);
  d.scan_rows = ListRef{reinterpret_cast<const int32_t*>(base + ti.o_srows), ti.n_srows, 0, 0, ti.na_srows};
  d.scan_cols = ListRef{reinterpret_cast<const int32_t*>(base + ti.o_scols), ti.n_scols, 0, 0};
  d.simt = ListRef{reinterpret_cast<const int32_t*>(base + ti.o_simt), ti.n_simt, 0, 0};
  d.s8 = ListRef{reinterpret_cast<const int32_t*>(base + ti.o_s8), ti.n_s8, 0, 0};
  for (int i = 0; i < 6; ++i)
    d.res[i] = ListRef{reinterpret_cast<const int32_t*>(base + ti.o_res[i]), ti.n_res[i],
                       ti.res_l[i] * (residue_class_w16(i) + 4) * 4, ti.res_l[i], ti.na_res[i]};
  for (int i = 0; i < 9; ++i) {
    d.tct[i] = ListRef{reinterpret_cast<const int32_t*>(base + ti.o_tct[i]), ti.n_tct[i], ti.tct_kpad[i], ti.tct_l[i]};
    d.tct_npad[i] = ti.tct_npad[i];
  }
  d.cmt.clear();
  for (const auto& sg : ti.cmt_seg)
    d.cmt.push_back(ListRef{reinterpret_cast<const int32_t*>(base + ti.o_cmt) + 4 * sg[0], sg[1], sg[2], 0});
  d.finl = ListRef{reinterpret_cast<const int32_t*>(base + ti.o_finl), ti.n_finl, ti.finl_dmax, ti.finl_nlmax};
  for (int c = 0; c < 9; ++c) d.fsh[c] = ListRef{reinterpret_cast<const int32_t*>(base + ti.o_fsh[c]), ti.n_fsh[c], 0, 0};
  d.rtt = ListRef{reinterpret_cast<const int32_t*>(base + ti.o_rtt), ti.n_rtt, ti.rtt_kpad, ti.rtt_l, ti.na_rtt};
  d.rmt.clear();
  for (size_t i = 0; i < ti.rmt_seg.size(); ++i) {
    const auto& sg = ti.rmt_seg[i];
    d.rmt.push_back(ListRef{reinterpret_cast<const int32_t*>(base + ti.o_rmt) + 4 * sg[0], sg[1], sg[2], 512,
                            ti.na_rmt[i]});
  }
  d.rtt_npad = ti.rtt_npad;
  d.res_tab.assign(pl->probs.size(), nullptr);
  for (size_t i = 0; i < pl->probs.size(); ++i)
    if (pl->probs[i].res_mode != 0) d.res_tab[i] = base + ti.o_rtab[pl->probs[i].res_key];
  d.crt_tab.assign(pl->probs.size(), nullptr);
  for (size_t i = 0; i < pl->probs.size(); ++i)
    if (pl->probs[i].crt_mode != 0) d.crt_tab[i] = base + ti.o_tctab[pl->probs[i].crt_key];
  for (int i = 0; i < kCrtClassCount; ++i)
    d.crt[i] = ListRef{reinterpret_cast<const int32_t*>(base + ti.o_crt[i]), ti.n_crt[i], 0, ti.crt_l[i]};
  d.groups.clear();
  if (count == 1) {
    const ProbHost& h = pl->probs[0];
    for (size_t g = 0; g < h.groups.size(); ++g) {
      const GroupHost& gr = h.groups[g];
      DevState::Group dg;
      dg.tab = d.tab;
      dg.tab.mods = d.tab.mods + gr.l0;                                // group-local modulus index
      dg.tab.t16 = d.tab.t16 + (size_t)gr.l0 * pl->w16max;
      dg.tab.lmax = gr.L;
      dg.tab.cta_begin = reinterpret_cast<const int32_t*>(base + ti.o_ctas) + ti.grp[g][0];
      dg.tab.count = 1;
      dg.grid = ti.grp[g][1];
      dg.res_tab = gr.res_key >= 0 ? base + ti.o_rtab[gr.res_key] : nullptr;
      d.groups.push_back(dg);
    }
  }
}

static int upload(ozaki2_plan_s* pl) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return OZ2_ENODEV;
  DevState& d = pl->dev;
  if (d.mem) return d.device == dev ? OZ2_OK : OZ2_EINVAL;
  int major = 0;
  if (cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess) return OZ2_ENODEV;
  if (major != 10) return OZ2_ENODEV;
  if (init_prep_attributes() != cudaSuccess || init_gemm_attributes() != cudaSuccess || init_gemm2_attributes() != cudaSuccess ||
      init_gemm_s8_attributes() != cudaSuccess ||
      init_crt_attributes() != cudaSuccess)
    return OZ2_ECUDA;
  if (!get_encode()) return OZ2_ECUDA;
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  TableImage ti;
  int rc = build_table_image(pl, sms, ti);
  if (rc) return rc;
  void* mem = nullptr;
  if (injected_alloc_failure() || cudaMalloc(&mem, ti.b.img.size()) != cudaSuccess) return OZ2_ENOMEM;
  if (cudaMemcpy(mem, ti.b.img.data(), ti.b.img.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaFree(mem);
    return OZ2_ECUDA;
  }
  d.mem = mem;
  d.device = dev;
  install_table_image(pl, ti, static_cast<uint8_t*>(mem));
  if (pl->opts.timing) {
    for (auto& e : pl->ev)
      if (cudaEventCreate(&e) != cudaSuccess) return OZ2_ECUDA;
    pl->evg.assign(2 * d.groups.size(), nullptr);
    for (auto& e : pl->evg)
      if (cudaEventCreate(&e) != cudaSuccess) return OZ2_ECUDA;
  }
  return OZ2_OK;
}

// Descriptor slots of a launch image: one per problem, then one per modulus
// group of a single product whose planes are streamed.
static int launch_slots(const ozaki2_plan_s* pl) {
  const int count = (int)pl->probs.size();
  return count + (count == 1 ? (int)pl->probs[0].groups.size() : 0);
}

static int alloc_launch_block(LaunchBlock& lb, int slots) {
  const size_t probs_bytes = align_up(sizeof(ProbDev) * slots, 128);
  lb.tmap_off = probs_bytes;
  lb.bytes = probs_bytes + sizeof(CUtensorMap) * kMapsPerProblem * slots;
  int rc = OZ2_OK;
  if (injected_alloc_failure() || cudaMalloc(&lb.d_mem, lb.bytes) != cudaSuccess) {
    lb.d_mem = nullptr;
    rc = OZ2_ENOMEM;
  } else if (cudaMallocHost(&lb.h_stage, lb.bytes) != cudaSuccess) {
    lb.h_stage = nullptr;
    rc = OZ2_ENOMEM;
  } else if (cudaEventCreateWithFlags(&lb.copied, cudaEventDisableTiming) != cudaSuccess) {
    lb.copied = nullptr;
    rc = OZ2_ECUDA;
  }
  if (rc) free_launch_block(lb);   // nothing half-made is kept: the next execute starts over
  return rc;
}

static bool mat_ok(const ozaki2_mat& m, int64_t rows, int64_t cols) {
  return m.limbs && m.exp && m.sign && m.ld >= cols && m.plane_stride >= rows * m.ld;
}

static int encode_planes(CUtensorMap* map, void* base, int64_t K, int64_t rows, int64_t Kp, int G,
                         int box_rows) {
  const cuuint64_t dims[3] = {(cuuint64_t)K, (cuuint64_t)rows, (cuuint64_t)G};
  const cuuint64_t strides[2] = {(cuuint64_t)Kp * 2, (cuuint64_t)(rows * Kp * 2)};
  const cuuint32_t box[3] = {(cuuint32_t)kBK, (cuuint32_t)box_rows, 1u};
  const cuuint32_t es[3] = {1u, 1u, 1u};
  const CUresult r = get_encode()(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, base, dims, strides, box, es,
                                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? OZ2_OK : OZ2_ECUDA;
}

// v_l of the plane GEMM as a [L][M][N] uint16 tensor (row pitch N, modulus
// pitch upitch), stored in 32 x 32 tiles staged with the 64-byte swizzle.
// Needs rows of 16-byte multiples (N a multiple of 8); 0 when N is not.
static int encode_u_store(CUtensorMap* map, uint16_t* u, int64_t N, int64_t M, int L, int64_t upitch,
                          int32_t* ok) {
  *ok = 0;
  if (N % 8 != 0) return OZ2_OK;
  const cuuint64_t dims[3] = {(cuuint64_t)N, (cuuint64_t)M, (cuuint64_t)L};
  const cuuint64_t strides[2] = {(cuuint64_t)N * 2, (cuuint64_t)upitch * 2};
  const cuuint32_t box[3] = {32u, 32u, 1u};
  const cuuint32_t es[3] = {1u, 1u, 1u};
  const CUresult r = get_encode()(map, CU_TENSOR_MAP_DATA_TYPE_UINT16, 3, u, dims, strides, box, es,
                                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
                                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return OZ2_ECUDA;
  *ok = 1;
  return OZ2_OK;
}

// Fill the launch image (ProbDev + tensor maps) for the given problems.
static int build_image(ozaki2_plan_s* pl, const ozaki2_problem* probs, uint8_t* ws,
                       std::vector<uint8_t>& img, size_t tmap_off, size_t bytes) {
  const int count = (int)pl->probs.size();
  img.assign(bytes, 0);
  auto* pd = reinterpret_cast<ProbDev*>(img.data());
  auto* tm = reinterpret_cast<CUtensorMap*>(img.data() + tmap_off);
  for (int i = 0; i < count; ++i) {
    const ProbHost& h = pl->probs[i];
    const ozaki2_problem& q = probs[i];
    if (q.M != h.M || q.N != h.N || q.K != h.K || q.p != h.p) return OZ2_EINVAL;
    if ((!h.skip_a && !mat_ok(q.A, h.M, h.K)) || (!h.skip_b && !mat_ok(q.B, h.K, h.N))) return OZ2_EINVAL;
    if (h.kind == 0 && !mat_ok(q.C, h.M, h.N)) return OZ2_EINVAL;
    if (h.kind == 1 && (!q.C.limbs || q.C.ld < h.N)) return OZ2_EINVAL;
    ProbDev& P = pd[i];
    P.a_limbs = q.A.limbs; P.a_exp = q.A.exp; P.a_sign = q.A.sign; P.a_ld = q.A.ld; P.a_ps = q.A.plane_stride;
    P.b_limbs = q.B.limbs; P.b_exp = q.B.exp; P.b_sign = q.B.sign; P.b_ld = q.B.ld; P.b_ps = q.B.plane_stride;
    P.c_limbs = q.C.limbs; P.c_exp = q.C.exp; P.c_sign = q.C.sign; P.c_ld = q.C.ld; P.c_ps = q.C.plane_stride;
    P.e = reinterpret_cast<int32_t*>(ws + h.off_e);
    P.f = reinterpret_cast<int32_t*>(ws + h.off_f);
    P.pa = reinterpret_cast<uint16_t*>(ws + h.off_pa);
    P.pb = reinterpret_cast<uint16_t*>(ws + h.off_pb);
    P.u = reinterpret_cast<uint16_t*>(ws + h.off_u);
    P.M = (int32_t)h.M; P.N = (int32_t)h.N; P.K = (int32_t)h.K; P.p = h.p; P.nl = h.nl; P.t = h.t;
    P.L = h.L; P.L1 = h.L1; P.G = h.G; P.Kp = h.Kp; P.W16 = h.W16; P.D32 = h.D32;
    P.crt_off = pl->dev.crt_off[i];
    P.tiles_m = h.tiles_m; P.tiles_n = h.tiles_n; P.nchunks = h.nchunks; P.kchunk = h.kchunk;
    P.kind = h.kind;
    if (h.kind == 1) {
      // binary64 output: C.limbs carries the double pointer, C.ld its row stride
      P.c_f64 = reinterpret_cast<double*>(q.C.limbs);
      P.c_f64_ld = q.C.ld;
      P.c_limbs = nullptr; P.c_exp = nullptr; P.c_sign = nullptr;
    }
    P.DS = h.DS;
    P.dbg_chat = pl->dbg_chat.empty() ? nullptr : pl->dbg_chat[i];
    P.dbg_prods = pl->dbg_prods.empty() ? nullptr : pl->dbg_prods[i];
    P.upitch = (int64_t)align_up((size_t)(h.M * h.N), 8);
    P.res_mode = h.res_mode;
    P.res_kpad = h.res_kpad;
    P.res_npad = h.res_npad;
    P.res_cw = h.res_cw;
    P.res_nchunk = h.res_nchunk;
    P.res_nabuf = h.res_nabuf;
    if (h.res_mode != 0) {
      // mode 1: the whole table in K blocks; mode 2: K block x cw columns
      const int rows = pl->rtabs[h.res_key].rows;
      const cuuint64_t dims[2] = {(cuuint64_t)h.res_kpad, (cuuint64_t)rows};
      const cuuint64_t strides[1] = {(cuuint64_t)h.res_kpad * 2};
      const cuuint32_t box[2] = {64u, (cuuint32_t)(h.res_mode == 1 ? h.res_npad : h.res_cw)};
      const cuuint32_t es[2] = {1u, 1u};
      if (get_encode()(&tm[4 * count + i], CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, pl->dev.res_tab[i], dims, strides,
                       box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                       CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return OZ2_ECUDA;
    }
    P.crt_mode = h.crt_mode;
    P.crt_kpad = h.crt_kpad;
    P.crt_npad = h.crt_npad;
    P.crt_np = h.crt_np;
    P.crt_nchunk = h.crt_nchunk;
    P.crt_cw = h.crt_cw;
    P.crt_q = h.crt_mode == 2 ? reinterpret_cast<uint32_t*>(ws + h.off_q) : nullptr;
    P.crt_alpha = h.crt_mode == 2 ? reinterpret_cast<uint32_t*>(ws + h.off_sig) : nullptr;
    P.crt_ngrp = h.crt_ngrp;
    P.crt_gskip = h.crt_gskip;
    P.crt_nslot = h.crt_nslot;
    P.crt_nvbuf = h.crt_nvbuf;
    int rc = encode_planes(&tm[2 * i], P.pa, h.K, h.M, h.Kp, h.G, kBM);
    if (rc) return rc;
    rc = encode_planes(&tm[2 * i + 1], P.pb, h.K, h.N, h.Kp, h.G, pl->tile2 ? kBN / 2 : kBN);
    if (rc) return rc;
    rc = encode_u_store(&tm[5 * count + i], P.u, h.N, h.M, h.L, P.upitch, &P.u_map);
    if (rc) return rc;
    if (h.crt_mode != 0) {
      // mode 1: the whole table in K blocks; mode 2: K block x cw columns of
      // a table padded to whole chunks
      const int rows = pl->crts[h.crt_key].rows;
      const cuuint64_t dims[2] = {(cuuint64_t)h.crt_kpad, (cuuint64_t)rows};
      const cuuint64_t strides[1] = {(cuuint64_t)h.crt_kpad * 2};
      const cuuint32_t box[2] = {64u, (cuuint32_t)(h.crt_mode == 1 ? h.crt_npad : h.crt_cw)};
      const cuuint32_t es[2] = {1u, 1u};
      if (get_encode()(&tm[2 * count + i], CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, pl->dev.crt_tab[i], dims, strides,
                       box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                       CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return OZ2_ECUDA;
      // u tiles: [L][upitch] uint16, boxes of 128 outputs x L moduli
      const cuuint64_t udims[2] = {(cuuint64_t)P.upitch, (cuuint64_t)h.L};
      const cuuint64_t ustr[1] = {(cuuint64_t)P.upitch * 2};
      const cuuint32_t ubox[2] = {128u, h.crt_mode == 1 ? (cuuint32_t)h.L : 32u};
      if (get_encode()(&tm[3 * count + i], CU_TENSOR_MAP_DATA_TYPE_UINT16, 2, P.u, udims, ustr, ubox, es,
                       CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                       CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return OZ2_ECUDA;
    }
  }
  // streamed planes: one descriptor per modulus group (moduli, planes and
  // residue geometry of the group; v_l and M_l^{-1} addressed from its first
  // modulus on), with its own plane and residue-table tensor maps
  if (count == 1) {
    const ProbHost& h = pl->probs[0];
    for (size_t g = 0; g < h.groups.size(); ++g) {
      const GroupHost& gr = h.groups[g];
      ProbDev& Q = pd[count + g];
      Q = pd[0];
      Q.L = gr.L; Q.L1 = gr.L1; Q.G = gr.G;
      Q.u = pd[0].u + (int64_t)gr.l0 * pd[0].upitch;
      Q.crt_off = pd[0].crt_off + gr.l0;
      Q.res_npad = gr.res_npad; Q.res_cw = gr.res_cw; Q.res_nchunk = gr.res_nchunk; Q.res_nabuf = gr.res_nabuf;
      Q.dbg_chat = nullptr;
      int gfirst = 0;                                    // planes of the groups before this one
      for (size_t q = 0; q < g; ++q) gfirst += h.groups[q].G;
      if (Q.dbg_prods) Q.dbg_prods += (int64_t)gfirst * h.M * h.N;
      CUtensorMap* gm = tm + kMapsPerProblem * (count + g);
      int rc = encode_planes(&gm[0], Q.pa, h.K, h.M, h.Kp, gr.G, kBM);
      if (rc) return rc;
      rc = encode_planes(&gm[1], Q.pb, h.K, h.N, h.Kp, gr.G, pl->tile2 ? kBN / 2 : kBN);
      if (rc) return rc;
      rc = encode_u_store(&gm[5], Q.u, h.N, h.M, gr.L, Q.upitch, &Q.u_map);
      if (rc) return rc;
      if (h.res_mode != 0) {
        const int rows = pl->rtabs[gr.res_key].rows;
        const cuuint64_t dims[2] = {(cuuint64_t)h.res_kpad, (cuuint64_t)rows};
        const cuuint64_t strides[1] = {(cuuint64_t)h.res_kpad * 2};
        const cuuint32_t box[2] = {64u, (cuuint32_t)(h.res_mode == 1 ? gr.res_npad : gr.res_cw)};
        const cuuint32_t es[2] = {1u, 1u};
        if (get_encode()(&gm[4], CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, pl->dev.groups[g].res_tab, dims, strides,
                         box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
          return OZ2_ECUDA;
      }
    }
  }
  return OZ2_OK;
}

static int stage_image(LaunchBlock& lb, const std::vector<uint8_t>& img, cudaStream_t s) {
  if (img == lb.last) return OZ2_OK;
  if (lb.pending && cudaEventSynchronize(lb.copied) != cudaSuccess) return OZ2_ECUDA;
  std::memcpy(lb.h_stage, img.data(), img.size());
  if (cudaMemcpyAsync(lb.d_mem, lb.h_stage, img.size(), cudaMemcpyHostToDevice, s) != cudaSuccess) return OZ2_ECUDA;
  if (cudaEventRecord(lb.copied, s) != cudaSuccess) return OZ2_ECUDA;
  lb.pending = true;
  lb.last = img;
  return OZ2_OK;
}

#define OZ2_CU(x)                                  \
  do {                                             \
    if ((x) != cudaSuccess) return OZ2_ECUDA;      \
  } while (0)

// Enqueue the five stages on `s` using launch block `lb` (already staged).
// keep = 0 (1): the workspace already holds the row exponents and planes of A
// (column exponents and planes of B) of this single-problem plan; only the
// other side is scanned and reduced.
static int enqueue(ozaki2_plan_s* pl, LaunchBlock& lb, uint8_t* ws, cudaStream_t s, bool timing, int keep = -1) {
  DevState& d = pl->dev;
  // the part of a block list that runs: every entry, or one side's
  auto part_ptr = [&](const ListRef& r) { return keep == 0 ? r.ptr + 4 * r.na : r.ptr; };
  auto part_n = [&](const ListRef& r) { return keep == 0 ? r.n - r.na : (keep == 1 ? r.na : r.n); };
  DevTables tab = d.tab;
  tab.spin_limit = pl->spin_limit;
  tab.probs = reinterpret_cast<const ProbDev*>(lb.d_mem);
  tab.tmaps = reinterpret_cast<const CUtensorMap*>(static_cast<uint8_t*>(lb.d_mem) + lb.tmap_off);
  const int count = (int)pl->probs.size();
  if (timing) OZ2_CU(cudaEventRecord(pl->ev[0], s));
  if (keep < 0) {
    OZ2_CU(cudaMemsetAsync(ws, 0x80, pl->ef_bytes, s));   // exponent sentinel below every valid exponent
  } else {
    const ProbHost& h = pl->probs[0];                     // only the side that is recomputed
    if (keep == 0) OZ2_CU(cudaMemsetAsync(ws + h.off_f, 0x80, 4 * (size_t)h.N, s));
    else OZ2_CU(cudaMemsetAsync(ws + h.off_e, 0x80, 4 * (size_t)h.M, s));
  }
  for (const ProbHost& h : pl->probs) {
    // a side whose planes the caller supplies is used unscaled: exponent 0
    if (h.skip_a) OZ2_CU(cudaMemsetAsync(ws + h.off_e, 0, 4 * (size_t)h.M, s));
    if (h.skip_b) OZ2_CU(cudaMemsetAsync(ws + h.off_f, 0, 4 * (size_t)h.N, s));
  }
  OZ2_CU(launch_scan(tab, count, part_ptr(d.scan_rows), d.scan_cols.ptr, part_n(d.scan_rows), d.scan_cols.n, s));
  if (timing) OZ2_CU(cudaEventRecord(pl->ev[1], s));
  if (!d.groups.empty()) {
    // streamed planes: each modulus group's residues, then its plane GEMMs,
    // through the same plane regions of the workspace (stream order keeps a
    // group's planes until its GEMMs have read them)
    const ProbHost& h = pl->probs[0];
    auto* pd = reinterpret_cast<const ProbDev*>(lb.d_mem);
    auto* tmp = reinterpret_cast<const CUtensorMap*>(static_cast<uint8_t*>(lb.d_mem) + lb.tmap_off);
    for (size_t g = 0; g < d.groups.size(); ++g) {
      const GroupHost& gr = h.groups[g];
      DevTables gt = d.groups[g].tab;
      gt.spin_limit = pl->spin_limit;
      gt.probs = pd + count + g;
      gt.tmaps = tmp + kMapsPerProblem * (count + g);
      if (timing) OZ2_CU(cudaEventRecord(pl->evg[2 * g], s));
      for (int c = 0; c < 6; ++c)
        if (d.res[c].n) OZ2_CU(launch_residues(gt, c, d.res[c].ptr, d.res[c].n, d.res[c].smem, s));
      if (d.rtt.n) OZ2_CU(launch_residues_tc(gt, d.rtt.ptr, d.rtt.n, d.rtt.smem, gr.res_npad, gr.L, d.sms, s));
      for (const ListRef& r : d.rmt) OZ2_CU(launch_residues_mm(gt, r.ptr, r.n, gr.res_cw, r.lmax, d.sms, s));
      if (timing) OZ2_CU(cudaEventRecord(pl->evg[2 * g + 1], s));
      OZ2_CU(pl->tile2 ? launch_gemm_tc2(gt, d.groups[g].grid, s) : launch_gemm_tc(gt, d.groups[g].grid, s));
    }
  } else {
    for (int c = 0; c < 6; ++c)
      if (part_n(d.res[c])) OZ2_CU(launch_residues(tab, c, part_ptr(d.res[c]), part_n(d.res[c]), d.res[c].smem, s));
    if (part_n(d.rtt))
      OZ2_CU(launch_residues_tc(tab, part_ptr(d.rtt), part_n(d.rtt), d.rtt.smem, d.rtt_npad, d.rtt.lmax, d.sms, s));
    for (const ListRef& r : d.rmt)
      if (part_n(r)) OZ2_CU(launch_residues_mm(tab, part_ptr(r), part_n(r), r.smem, r.lmax, d.sms, s));
    if (pl->complex3m) {
      // the residue planes of Ar + Ai and Br + Bi, from those of the real and imaginary parts
      const ProbHost& h = pl->probs[0];
      const int64_t kc = h.Kp / 8;
      OZ2_CU(launch_plane_sum(tab, (int64_t)h.L * h.M * kc, (int64_t)h.L * h.N * kc, s));
    }
    if (timing) OZ2_CU(cudaEventRecord(pl->ev[2], s));
    if (pl->opts.engine == OZ2_ENGINE_SIMT) {
      DevTables t2 = tab;
      t2.units = d.unsorted;
      OZ2_CU(launch_gemm_simt(t2, d.simt.ptr, d.simt.n, s));
    } else if (pl->opts.engine == OZ2_ENGINE_S8) {
      DevTables t2 = tab;
      t2.units = d.unsorted;
      OZ2_CU(launch_gemm_s8(t2, d.s8.ptr, d.s8.n, s));
    } else if (pl->opts.schedule == OZ2_SCHED_GROUPED) {
      OZ2_CU(pl->tile2 ? launch_gemm_tc2(tab, d.grid, s) : launch_gemm_tc(tab, d.grid, s));
    } else {
      for (const PlainSeg& sg : d.plain) {
        DevTables t2 = tab;
        t2.cta_begin = d.cta_plain + sg.cta_off;
        OZ2_CU(pl->tile2 ? launch_gemm_tc2(t2, sg.grid, s) : launch_gemm_tc(t2, sg.grid, s));
      }
    }
  }
  if (pl->complex3m) {
    // v_r = v(Ar Br) - v(Ai Bi), v_i = v((Ar + Ai)(Br + Bi)) - v(Ar Br) - v(Ai Bi) mod m_l
    const ProbHost& h = pl->probs[0];
    OZ2_CU(launch_combine_complex(tab, (int64_t)h.L * (int64_t)(align_up((size_t)(h.M * h.N), 8) / 8), s));
  }
  if (timing) OZ2_CU(cudaEventRecord(pl->ev[3], s));
  {
    // the CRT table stays resident in the sums kernel when one problem uses it
    int n2 = 0, blocks_one = 0;
    for (const ProbHost& h : pl->probs)
      if (h.crt_mode == 2 && !h.no_crt) {
        ++n2;
        blocks_one = (h.crt_kpad / 64) * h.crt_nchunk;
      }
    for (const ListRef& r : d.cmt)
      OZ2_CU(launch_crt_mm(tab, r.ptr, r.n, r.smem, d.sms, n2 == 1 ? blocks_one : 0, s));
  }
  if (timing) OZ2_CU(cudaEventRecord(pl->ev[5], s));
  for (int c = 0; c < 9; ++c)
    if (d.fsh[c].n) OZ2_CU(launch_crt_fin_short(tab, c, d.fsh[c].ptr, d.fsh[c].n, s));
  if (d.finl.n) OZ2_CU(launch_crt_finish_long(tab, d.finl.ptr, d.finl.n, d.finl.smem, d.finl.lmax, s));
  for (int c = 0; c < kCrtClassCount; ++c)
    if (d.crt[c].n) OZ2_CU(launch_crt(tab, c, d.crt[c].ptr, d.crt[c].n, d.crt[c].lmax, s));
  for (int c = 0; c < 9; ++c)
    if (d.tct[c].n)
      OZ2_CU(launch_crt_tc(tab, c, d.tct[c].ptr, d.tct[c].n, d.tct[c].smem, d.tct_npad[c], d.tct[c].lmax,
                           d.sms, s));
  if (timing) OZ2_CU(cudaEventRecord(pl->ev[4], s));
  return OZ2_OK;
}

static int execute_impl(ozaki2_plan_s* pl, int count, const ozaki2_problem* probs, void* ws,
                        size_t ws_bytes, cudaStream_t s, int keep = -1) {
  if (!pl || !probs || !ws) return OZ2_EINVAL;
  if (count != (int)pl->probs.size()) return OZ2_EINVAL;
  if (ws_bytes < pl->ws_bytes || (reinterpret_cast<uintptr_t>(ws) & 255u)) return OZ2_EINVAL;
  if (keep >= 0 && (count != 1 || !pl->probs[0].groups.empty() || pl->last_ws != ws)) return OZ2_EINVAL;
  int rc = upload(pl);
  if (rc) return rc;
  const int slots = launch_slots(pl);
  const size_t tmap_off = align_up(sizeof(ProbDev) * slots, 128);
  const size_t lb_bytes = tmap_off + sizeof(CUtensorMap) * kMapsPerProblem * slots;
  std::vector<uint8_t> img;
  rc = build_image(pl, probs, static_cast<uint8_t*>(ws), img, tmap_off, lb_bytes);
  if (rc) return rc;
  // the ring entry holding this image, else the least recently used one
  int pick = -1;
  for (int i = 0; i < ozaki2_plan_s::kLaunchRing && pick < 0; ++i)
    if (pl->lbs[i].d_mem && pl->lbs[i].last == img) pick = i;
  if (pick < 0) {
    pick = 0;
    for (int i = 1; i < ozaki2_plan_s::kLaunchRing; ++i)
      if (pl->lb_used[i] < pl->lb_used[pick]) pick = i;
    if (!pl->lbs[pick].d_mem && (rc = alloc_launch_block(pl->lbs[pick], slots))) return rc;
    rc = stage_image(pl->lbs[pick], img, s);
    if (rc) return rc;
  }
  pl->lb_used[pick] = ++pl->lb_clock;
  LaunchBlock& lb = pl->lbs[pick];
  pl->timed = pl->opts.timing != 0;
  rc = enqueue(pl, lb, static_cast<uint8_t*>(ws), s, pl->timed, keep);
  if (count == 1) {
    pl->last_ws = rc ? nullptr : ws;
    pl->last_q = probs[0];
  }
  return rc;
}

int plan_create_ex(int64_t M, int64_t N, int64_t K, int p, const ozaki2_opts* opts,
                   const PlanExtra& ex, ozaki2_plan* out) {
  if (!out) return OZ2_EINVAL;
  *out = nullptr;
  ozaki2_plan_s* pl = nullptr;
  int rc = new_plan(opts, &pl);
  if (rc) return rc;
  pl->no_stream = true;                          // the binary64 mode keeps every plane for the backward
  try {
    rc = build_problem(pl, M, N, K, p, &ex);
  } catch (const std::bad_alloc&) {
    rc = OZ2_ENOMEM;
  }
  if (rc) { delete pl; return rc; }
  layout_workspace(pl);
  *out = pl;
  return OZ2_OK;
}

int plan_query(ozaki2_plan pl, PlanFacts* f) {
  if (!pl || !f) return OZ2_EINVAL;
  const ProbHost& h = pl->probs[0];
  f->t = h.t; f->L = h.L; f->G = h.G; f->Kp = h.Kp;
  f->off_e = h.off_e; f->off_f = h.off_f; f->off_pa = h.off_pa; f->off_pb = h.off_pb;
  f->ws_bytes = pl->ws_bytes;
  return OZ2_OK;
}

int plan_run(ozaki2_plan pl, const ozaki2_problem* q, void* ws, size_t ws_bytes, cudaStream_t s) {
  return execute_impl(pl, 1, q, ws, ws_bytes, s);
}

}  // namespace oz2

using namespace oz2;

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

int ozaki2_opts_default(ozaki2_opts* o) {
  if (!o) return OZ2_EINVAL;
  std::memset(o, 0, sizeof(*o));
  o->guard_bits = 16;
  o->t_bits = 0;
  o->engine = OZ2_ENGINE_TC;
  o->k_chunk = 0;
  o->grid = 0;
  o->schedule = OZ2_SCHED_GROUPED;
  o->timing = 0;
  o->crt_engine = 0;
  o->res_engine = 0;
  return OZ2_OK;
}

const char* ozaki2_strerror(int st) {
  switch (st) {
    case OZ2_OK: return "success";
    case OZ2_EINVAL: return "invalid argument";
    case OZ2_ERANGE: return "size or precision outside the supported range";
    case OZ2_ENOMEM: return "out of memory";
    case OZ2_ECUDA: return "CUDA call failed";
    case OZ2_EINTERNAL: return "device-side consistency check failed";
    case OZ2_ETIMEOUT: return "device-side wait timed out";
    case OZ2_ENODEV: return "no usable sm_103 device";
  }
  return "unknown status";
}

const char* ozaki2_version(void) { return "ozaki2-gb300 0.1"; }

int ozaki2_plan_create(int64_t M, int64_t N, int64_t K, int p, const ozaki2_opts* opts,
                       ozaki2_plan* out) {
  if (!out) return OZ2_EINVAL;
  *out = nullptr;
  ozaki2_plan_s* pl = nullptr;
  int rc = new_plan(opts, &pl);
  if (rc) return rc;
  if (pl->opts.gemm_tile == 0 && pl->opts.engine == OZ2_ENGINE_TC) pl->tile2 = auto_pair_tiles(pl, M, N, K, p);
  try {
    rc = build_problem(pl, M, N, K, p);
    if (!rc) rc = plan_groups(pl);
  } catch (const std::bad_alloc&) {
    rc = OZ2_ENOMEM;
  }
  if (rc) { delete pl; return rc; }
  layout_workspace(pl);
  *out = pl;
  return OZ2_OK;
}

int ozaki2_plan_create_batched(int count, const ozaki2_problem* shapes, const ozaki2_opts* opts,
                               ozaki2_plan* out) {
  return ozaki2_plan_create_batched_ex(count, shapes, opts, nullptr, out);
}

int ozaki2_plan_create_batched_ex(int count, const ozaki2_problem* shapes, const ozaki2_opts* opts,
                                  const ozaki2_opts* per_problem, ozaki2_plan* out) {
  if (!out || !shapes || count <= 0 || count > 65535) return OZ2_EINVAL;
  *out = nullptr;
  ozaki2_plan_s* pl = nullptr;
  int rc = new_plan(opts, &pl);
  if (rc) return rc;
  std::vector<ozaki2_opts> po;
  if (per_problem) {
    po.assign(count, pl->opts);
    for (int i = 0; i < count; ++i) {
      const ozaki2_opts& q = per_problem[i];
      if (q.guard_bits < 0 || q.t_bits < 0 || q.k_chunk < 0 || q.crt_engine < 0 || q.crt_engine > 3 ||
          q.res_engine < 0 || q.res_engine > 3) {
        delete pl;
        return OZ2_EINVAL;
      }
      po[i].guard_bits = q.guard_bits;
      po[i].t_bits = q.t_bits;
      po[i].k_chunk = q.k_chunk;
      po[i].crt_engine = q.crt_engine;
      po[i].res_engine = q.res_engine;
    }
  }
  try {
    for (int i = 0; i < count && !rc; ++i)
      rc = build_problem(pl, shapes[i].M, shapes[i].N, shapes[i].K, shapes[i].p, nullptr, po.empty() ? nullptr : &po[i]);
  } catch (const std::bad_alloc&) {
    rc = OZ2_ENOMEM;
  }
  if (rc) { delete pl; return rc; }
  layout_workspace(pl);
  *out = pl;
  return OZ2_OK;
}

int ozaki2_plan_create_complex(int64_t M, int64_t N, int64_t K, int p, const ozaki2_opts* opts, ozaki2_plan* out) {
  if (!out) return OZ2_EINVAL;
  *out = nullptr;
  ozaki2_plan_s* pl = nullptr;
  int rc = new_plan(opts, &pl);
  if (rc) return rc;
  if (pl->opts.gemm_tile == 0 && pl->opts.engine == OZ2_ENGINE_TC) pl->tile2 = auto_pair_tiles(pl, M, N, K, p);
  pl->complex3m = true;
  PlanExtra ex;
  ex.inner = 2 * K;                              // |Cr_hat|, |Ci_hat| <= 2K 2^(2t)
  try {
    for (int i = 0; i < 3 && !rc; ++i) rc = build_problem(pl, M, N, K, p, &ex);
  } catch (const std::bad_alloc&) {
    rc = OZ2_ENOMEM;
  }
  if (rc) { delete pl; return rc; }
  pl->probs[2].sum_of = true;
  pl->probs[2].no_crt = true;
  layout_workspace(pl);
  // one row exponent over Ar and Ai, one column exponent over Br and Bi
  for (int i = 1; i < 3; ++i) {
    pl->probs[i].off_e = pl->probs[0].off_e;
    pl->probs[i].off_f = pl->probs[0].off_f;
  }
  *out = pl;
  return OZ2_OK;
}

int ozaki2_execute_complex(ozaki2_plan pl, const ozaki2_mat* Ar, const ozaki2_mat* Ai, const ozaki2_mat* Br,
                           const ozaki2_mat* Bi, ozaki2_mat* Cr, ozaki2_mat* Ci, void* ws, size_t ws_bytes,
                           void* stream) {
  if (!pl || !pl->complex3m || !Ar || !Ai || !Br || !Bi || !Cr || !Ci) return OZ2_EINVAL;
  const ProbHost& h = pl->probs[0];
  const ozaki2_problem q[3] = {{h.M, h.N, h.K, h.p, *Ar, *Br, *Cr},
                               {h.M, h.N, h.K, h.p, *Ai, *Bi, *Ci},
                               {h.M, h.N, h.K, h.p, *Ar, *Br, *Cr}};   // planes from the sums; no output
  try {
    return execute_impl(pl, 3, q, ws, ws_bytes, static_cast<cudaStream_t>(stream));
  } catch (const std::bad_alloc&) {
    return OZ2_ENOMEM;
  }
}

int ozaki2_plan_destroy(ozaki2_plan pl) {
  if (!pl) return OZ2_EINVAL;
  for (auto& lb : pl->lbs) free_launch_block(lb);
  if (pl->dev.mem) cudaFree(pl->dev.mem);
  for (auto& e : pl->ev)
    if (e) cudaEventDestroy(e);
  for (auto& e : pl->evg)
    if (e) cudaEventDestroy(e);
  delete pl;
  return OZ2_OK;
}

int ozaki2_plan_info(ozaki2_plan pl, ozaki2_info* out) {
  if (!pl || !out) return OZ2_EINVAL;
  const ProbHost& h = pl->probs[0];
  out->count = (int)pl->probs.size();
  out->t = h.t;
  out->L = h.L;
  out->L1 = h.L1;
  out->G = h.G;
  out->crt_digits = h.D32;
  out->crt_skip_groups = h.crt_gskip;
  out->units = (int)std::min<int64_t>(INT_MAX, pl->total_units);
  out->jobs = (int)std::min<int64_t>(INT_MAX, pl->total_jobs);
  out->workspace_bytes = pl->ws_bytes;
  out->crt_mode = h.crt_mode;
  out->res_mode = h.res_mode;
  out->plane_groups = std::max<int>(1, (int)h.groups.size());
  out->group_planes = group_planes_max(h);
  out->gemm_tile = pl->tile2 ? 2 : 1;
  return OZ2_OK;
}

int ozaki2_plan_moduli(ozaki2_plan pl, int prob, int32_t* out, int cap) {
  if (!pl || !out || prob < 0 || prob >= (int)pl->probs.size()) return OZ2_EINVAL;
  const ProbHost& h = pl->probs[prob];
  if (cap < h.L) return OZ2_EINVAL;
  for (int l = 0; l < h.L; ++l) out[l] = (int32_t)modulus_list()[l];
  return OZ2_OK;
}

int ozaki2_plan_crt_tables(ozaki2_plan pl, int prob, uint32_t* P_digits, uint32_t* M_digits,
                           uint32_t* Minv) {
  if (!pl || prob < 0 || prob >= (int)pl->probs.size()) return OZ2_EINVAL;
  const ProbHost& h = pl->probs[prob];
  const CrtHost& c = pl->crts[h.crt_key];
  const int D = c.D32, DS = c.DS, L = c.L;
  if (P_digits)
    for (int i = 0; i < D; ++i) P_digits[i] = c.words[i];
  if (M_digits)
    for (int l = 0; l < L; ++l)
      for (int i = 0; i < D; ++i) M_digits[(size_t)l * D + i] = c.words[3 * DS + L + (size_t)l * DS + i];
  if (Minv)
    for (int l = 0; l < L; ++l) Minv[l] = c.words[3 * DS + l];
  return OZ2_OK;
}

int ozaki2_plan_layout(ozaki2_plan pl, int prob, size_t off[5], int64_t* kp) {
  if (!pl || !off || prob < 0 || prob >= (int)pl->probs.size()) return OZ2_EINVAL;
  const ProbHost& h = pl->probs[prob];
  off[0] = h.off_e;
  off[1] = h.off_f;
  off[2] = h.off_pa;
  off[3] = h.off_pb;
  off[4] = h.off_u;
  if (kp) *kp = h.Kp;
  return OZ2_OK;
}

int ozaki2_plan_launches(ozaki2_plan pl, int* n) {
  if (!pl || !n) return OZ2_EINVAL;
  const DevState& d = pl->dev;
  if (!d.mem) return OZ2_EINVAL;                 // counted once the plan has run
  int c = 0;
  c += (d.scan_rows.n || d.scan_cols.n) ? 1 : 0;
  int res = 0;
  for (int i = 0; i < 6; ++i) res += d.res[i].n ? 1 : 0;
  res += d.rtt.n ? 1 : 0;
  res += (int)d.rmt.size();
  if (pl->complex3m) c += 2;                      // plane sums, combination
  if (!d.groups.empty()) c += (int)d.groups.size() * (res + 1);   // per group: residues + one GEMM
  else if (pl->opts.engine == OZ2_ENGINE_SIMT || pl->opts.engine == OZ2_ENGINE_S8) c += res + 1;
  else if (pl->opts.schedule == OZ2_SCHED_GROUPED) c += res + 1;
  else c += res + (int)d.plain.size();
  c += (int)d.cmt.size();
  c += d.finl.n ? 1 : 0;
  for (int i = 0; i < 9; ++i) c += d.fsh[i].n ? 1 : 0;
  for (int i = 0; i < kCrtClassCount; ++i) c += d.crt[i].n ? 1 : 0;
  for (int i = 0; i < 9; ++i) c += d.tct[i].n ? 1 : 0;
  *n = c;
  return OZ2_OK;
}

int ozaki2_plan_set_debug_chat(ozaki2_plan pl, int prob, uint32_t* dev_buf) {
  if (!pl || prob < 0 || prob >= (int)pl->probs.size()) return OZ2_EINVAL;
  if (pl->dbg_chat.empty()) pl->dbg_chat.assign(pl->probs.size(), nullptr);
  pl->dbg_chat[prob] = dev_buf;
  return OZ2_OK;
}

int ozaki2_plan_set_debug_prods(ozaki2_plan pl, int prob, int32_t* dev_buf) {
  if (!pl || prob < 0 || prob >= (int)pl->probs.size()) return OZ2_EINVAL;
  if (dev_buf && (pl->probs[prob].nchunks != 1 || pl->opts.engine != OZ2_ENGINE_TC)) return OZ2_EINVAL;
  if (pl->dbg_prods.empty()) pl->dbg_prods.assign(pl->probs.size(), nullptr);
  pl->dbg_prods[prob] = dev_buf;
  return OZ2_OK;
}

int ozaki2_plan_set_wait_limit(ozaki2_plan pl, uint32_t polls) {
  if (!pl) return OZ2_EINVAL;
  pl->spin_limit = polls ? polls : kDefaultSpinLimit;
  return OZ2_OK;
}

int ozaki2_plan_debug_corrupt_crt(ozaki2_plan pl, int prob) {
  if (!pl || prob < 0 || prob >= (int)pl->probs.size() || pl->dev.mem) return OZ2_EINVAL;
  const ProbHost& h = pl->probs[prob];
  CrtHost& c = pl->crts[h.crt_key];
  // the top 32-bit digit of M_0 = P / m_0 in the digit table, with its high bit flipped
  Big M0;
  big_divmod_small(c.P, modulus_list()[0], &M0);
  const int top = (int)M0.size() - 1;
  c.words[3 * c.DS + c.L + top] ^= 0x80000000u;
  if (!c.tc_table.empty()) {
    // the top 7-bit piece of M_0 in the tensor-core table (both places it occurs)
    const int jt = (big_bitlen(M0) - 1) / 7;
    auto flip = [&](size_t idx) {
      float f;
      uint32_t u = (uint32_t)c.tc_table[idx] << 16;
      std::memcpy(&f, &u, 4);
      const uint32_t x = (uint32_t)f ^ 64u;
      f = (float)x;
      std::memcpy(&u, &f, 4);
      c.tc_table[idx] = (uint16_t)(u >> 16);
    };
    flip((size_t)jt * c.kpad + 0);
    if (jt + 1 < c.rows) flip((size_t)(jt + 1) * c.kpad + 1);
  }
  return OZ2_OK;
}

int ozaki2_debug_inject_alloc_failure(int count) {
  if (count < 0) return OZ2_EINVAL;
  g_inject_alloc.store(count);
  return OZ2_OK;
}

int ozaki2_execute(ozaki2_plan pl, const ozaki2_mat* A, const ozaki2_mat* B, ozaki2_mat* C, void* ws,
                   size_t ws_bytes, void* stream) {
  if (!pl || !A || !B || !C || pl->probs.size() != 1) return OZ2_EINVAL;
  const ProbHost& h = pl->probs[0];
  ozaki2_problem q{h.M, h.N, h.K, h.p, *A, *B, *C};
  try {
    return execute_impl(pl, 1, &q, ws, ws_bytes, static_cast<cudaStream_t>(stream));
  } catch (const std::bad_alloc&) {
    return OZ2_ENOMEM;
  }
}

int ozaki2_execute_batched(ozaki2_plan pl, int count, const ozaki2_problem* probs, void* ws,
                           size_t ws_bytes, void* stream) {
  if (pl && pl->complex3m) return OZ2_EINVAL;   // ozaki2_execute_complex
  try {
    return execute_impl(pl, count, probs, ws, ws_bytes, static_cast<cudaStream_t>(stream));
  } catch (const std::bad_alloc&) {
    return OZ2_ENOMEM;
  }
}

int ozaki2_execute_reuse(ozaki2_plan pl, int keep, const ozaki2_mat* X, ozaki2_mat* C, void* ws, size_t ws_bytes,
                         void* stream) {
  if (!pl || !X || !C || (keep != 0 && keep != 1) || pl->probs.size() != 1 || !pl->last_ws) return OZ2_EINVAL;
  if (pl->probs[0].skip_a || pl->probs[0].skip_b) return OZ2_EINVAL;
  ozaki2_problem q = pl->last_q;
  if (keep == 0) q.B = *X;
  else q.A = *X;
  q.C = *C;
  try {
    return execute_impl(pl, 1, &q, ws, ws_bytes, static_cast<cudaStream_t>(stream), keep);
  } catch (const std::bad_alloc&) {
    return OZ2_ENOMEM;
  }
}

int ozaki2_graph_create(ozaki2_plan pl, int count, const ozaki2_problem* probs, void* ws,
                        size_t ws_bytes, void* stream, ozaki2_graph* out) {
  if (!pl || !probs || !ws || !out || !stream) return OZ2_EINVAL;
  if (count != (int)pl->probs.size() || ws_bytes < pl->ws_bytes) return OZ2_EINVAL;
  *out = nullptr;
  int rc = upload(pl);
  if (rc) return rc;
  auto* g = new (std::nothrow) ozaki2_graph_s();
  if (!g) return OZ2_ENOMEM;
  rc = alloc_launch_block(g->lb, launch_slots(pl));
  std::vector<uint8_t> img;
  if (!rc) rc = build_image(pl, probs, static_cast<uint8_t*>(ws), img, g->lb.tmap_off, g->lb.bytes);
  if (!rc && cudaMemcpy(g->lb.d_mem, img.data(), img.size(), cudaMemcpyHostToDevice) != cudaSuccess) rc = OZ2_ECUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (!rc && cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) rc = OZ2_ECUDA;
  if (!rc) {
    const int erc = enqueue(pl, g->lb, static_cast<uint8_t*>(ws), s, false);
    const cudaError_t ce = cudaStreamEndCapture(s, &g->graph);
    rc = erc ? erc : (ce != cudaSuccess ? OZ2_ECUDA : OZ2_OK);
  }
  if (!rc && cudaGraphInstantiate(&g->exec, g->graph, 0) != cudaSuccess) rc = OZ2_ECUDA;
  if (rc) {
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->graph) cudaGraphDestroy(g->graph);
    free_launch_block(g->lb);
    delete g;
    return rc;
  }
  *out = g;
  return OZ2_OK;
}

int ozaki2_graph_launch(ozaki2_graph g, void* stream) {
  if (!g) return OZ2_EINVAL;
  return cudaGraphLaunch(g->exec, static_cast<cudaStream_t>(stream)) == cudaSuccess ? OZ2_OK : OZ2_ECUDA;
}

int ozaki2_graph_destroy(ozaki2_graph g) {
  if (!g) return OZ2_EINVAL;
  if (g->exec) cudaGraphExecDestroy(g->exec);
  if (g->graph) cudaGraphDestroy(g->graph);
  free_launch_block(g->lb);
  delete g;
  return OZ2_OK;
}

int ozaki2_check(ozaki2_plan pl, void* stream) {
  if (!pl) return OZ2_EINVAL;
  if (cudaStreamSynchronize(static_cast<cudaStream_t>(stream)) != cudaSuccess) return OZ2_ECUDA;
  if (!pl->dev.mem) return OZ2_OK;
  int32_t st = 0;
  if (cudaMemcpy(&st, pl->dev.tab.status, 4, cudaMemcpyDeviceToHost) != cudaSuccess) return OZ2_ECUDA;
  if (st) {
    const int32_t zero = 0;
    if (cudaMemcpy(pl->dev.tab.status, &zero, 4, cudaMemcpyHostToDevice) != cudaSuccess) return OZ2_ECUDA;
  }
  if (st & kStatusTimeout) return OZ2_ETIMEOUT;
  if (st) return OZ2_EINTERNAL;
  return OZ2_OK;
}

int ozaki2_last_timings(ozaki2_plan pl, float ms[5]) {
  if (!pl || !ms || !pl->timed || !pl->ev[0]) return OZ2_EINVAL;
  if (cudaEventSynchronize(pl->ev[4]) != cudaSuccess) return OZ2_ECUDA;
  if (!pl->evg.empty() && !pl->dev.groups.empty()) {
    // streamed planes: residues and GEMMs summed over the groups
    const size_t ng = pl->evg.size() / 2;
    float r = 0.f, gm = 0.f, x = 0.f;
    for (size_t g = 0; g < ng; ++g) {
      if (cudaEventElapsedTime(&x, pl->evg[2 * g], pl->evg[2 * g + 1]) != cudaSuccess) return OZ2_ECUDA;
      r += x;
      cudaEvent_t end = g + 1 < ng ? pl->evg[2 * g + 2] : pl->ev[3];
      if (cudaEventElapsedTime(&x, pl->evg[2 * g + 1], end) != cudaSuccess) return OZ2_ECUDA;
      gm += x;
    }
    if (cudaEventElapsedTime(&ms[0], pl->ev[0], pl->ev[1]) != cudaSuccess) return OZ2_ECUDA;
    ms[1] = r;
    ms[2] = gm;
    if (cudaEventElapsedTime(&ms[3], pl->ev[3], pl->ev[4]) != cudaSuccess) return OZ2_ECUDA;
  } else {
    for (int i = 0; i < 4; ++i)
      if (cudaEventElapsedTime(&ms[i], pl->ev[i], pl->ev[i + 1]) != cudaSuccess) return OZ2_ECUDA;
  }
  if (cudaEventElapsedTime(&ms[4], pl->ev[0], pl->ev[4]) != cudaSuccess) return OZ2_ECUDA;
  return OZ2_OK;
}

int ozaki2_last_crt_split(ozaki2_plan pl, float ms[2]) {
  if (!pl || !ms || !pl->timed || !pl->ev[0]) return OZ2_EINVAL;
  if (cudaEventSynchronize(pl->ev[4]) != cudaSuccess) return OZ2_ECUDA;
  if (cudaEventElapsedTime(&ms[0], pl->ev[3], pl->ev[5]) != cudaSuccess) return OZ2_ECUDA;
  if (cudaEventElapsedTime(&ms[1], pl->ev[5], pl->ev[4]) != cudaSuccess) return OZ2_ECUDA;
  return OZ2_OK;
}

// ---------------------------------------------------------------------------
// Convenience calls with library-owned plans and workspaces
// ---------------------------------------------------------------------------
namespace {
struct Cached {
  ozaki2_plan plan = nullptr;
  void* ws = nullptr;
};
std::mutex g_cache_mu;
std::map<std::vector<int64_t>, Cached> g_cache;

std::vector<int64_t> cache_key(int count, const ozaki2_problem* probs, const ozaki2_opts& o) {
  int dev = -1;
  cudaGetDevice(&dev);
  std::vector<int64_t> k{dev, o.guard_bits, o.t_bits, o.engine, o.k_chunk, o.grid, o.schedule, o.timing,
                         o.crt_engine, o.res_engine, o.plane_group, o.gemm_tile, count};
  for (int i = 0; i < count; ++i) {
    k.push_back(probs[i].M);
    k.push_back(probs[i].N);
    k.push_back(probs[i].K);
    k.push_back(probs[i].p);
  }
  return k;
}

int cached_run(int count, const ozaki2_problem* probs, const ozaki2_opts* opts, void* stream) {
  ozaki2_opts o;
  if (opts) o = *opts;
  else ozaki2_opts_default(&o);
  std::lock_guard<std::mutex> lk(g_cache_mu);
  const auto key = cache_key(count, probs, o);
  auto it = g_cache.find(key);
  if (it == g_cache.end()) {
    Cached c;
    int rc = count == 1 ? ozaki2_plan_create(probs[0].M, probs[0].N, probs[0].K, probs[0].p, &o, &c.plan)
                        : ozaki2_plan_create_batched(count, probs, &o, &c.plan);
    if (rc) return rc;
    if (cudaMalloc(&c.ws, c.plan->ws_bytes) != cudaSuccess) {
      ozaki2_plan_destroy(c.plan);
      return OZ2_ENOMEM;
    }
    it = g_cache.emplace(key, c).first;
  }
  return ozaki2_execute_batched(it->second.plan, count, probs, it->second.ws, it->second.plan->ws_bytes, stream);
}
}  // namespace

int ozaki2_gemm(int64_t M, int64_t N, int64_t K, int p, const ozaki2_mat* A, const ozaki2_mat* B,
                ozaki2_mat* C, const ozaki2_opts* opts, void* stream) {
  if (!A || !B || !C) return OZ2_EINVAL;
  ozaki2_problem q{M, N, K, p, *A, *B, *C};
  try {
    return cached_run(1, &q, opts, stream);
  } catch (const std::bad_alloc&) {
    return OZ2_ENOMEM;
  }
}

int ozaki2_zgemm(int64_t M, int64_t N, int64_t K, int p, const ozaki2_mat* Ar, const ozaki2_mat* Ai,
                 const ozaki2_mat* Br, const ozaki2_mat* Bi, ozaki2_mat* Cr, ozaki2_mat* Ci, const ozaki2_opts* opts,
                 void* stream) {
  if (!Ar || !Ai || !Br || !Bi || !Cr || !Ci) return OZ2_EINVAL;
  ozaki2_opts o;
  if (opts) o = *opts;
  else ozaki2_opts_default(&o);
  try {
    std::lock_guard<std::mutex> lk(g_cache_mu);
    const ozaki2_problem q{M, N, K, p, *Ar, *Br, *Cr};
    auto key = cache_key(1, &q, o);
    key.push_back(-3);                             // complex plans are cached apart
    auto it = g_cache.find(key);
    if (it == g_cache.end()) {
      Cached c;
      int rc = ozaki2_plan_create_complex(M, N, K, p, &o, &c.plan);
      if (rc) return rc;
      if (injected_alloc_failure() || cudaMalloc(&c.ws, c.plan->ws_bytes) != cudaSuccess) {
        ozaki2_plan_destroy(c.plan);
        return OZ2_ENOMEM;
      }
      it = g_cache.emplace(key, c).first;
    }
    return ozaki2_execute_complex(it->second.plan, Ar, Ai, Br, Bi, Cr, Ci, it->second.ws, it->second.plan->ws_bytes,
                                  stream);
  } catch (const std::bad_alloc&) {
    return OZ2_ENOMEM;
  }
}

int ozaki2_gemm_batched(int count, const ozaki2_problem* probs, const ozaki2_opts* opts, void* stream) {
  if (!probs || count <= 0) return OZ2_EINVAL;
  try {
    return cached_run(count, probs, opts, stream);
  } catch (const std::bad_alloc&) {
    return OZ2_ENOMEM;
  }
}

int ozaki2_release_cache(void) {
  std::lock_guard<std::mutex> lk(g_cache_mu);
  for (auto& kv : g_cache) {
    cudaFree(kv.second.ws);
    ozaki2_plan_destroy(kv.second.plan);
  }
  g_cache.clear();
  return OZ2_OK;
}

}  // extern "C"

// ===========================================================================
// Entry point that allocates no device memory
// ===========================================================================
// Some callers cannot allocate device memory while they run: code that
// executes inside a memory-capped region, a custom allocator that owns every
// byte of the GPU, or a host thread that must not call cudaMalloc/cudaFree
// (they synchronise the device).  ozaki2_gemm_noalloc serves them: every
// intermediate of the product lives in fixed arrays in the library's own
// device memory, reserved when the library's device code is loaded on a GPU
// and held until the process exits.
static __device__ __align__(256) uint8_t ozaki2_noalloc_scratch[64u << 20];   // exponents, planes, reduced products
static __device__ __align__(256) uint8_t ozaki2_noalloc_tables[4u << 20];     // tables, schedule, descriptor, tensor maps

namespace {

// The last 256 bytes of the table array hold this path's device status word;
// the table image of a call never reaches them.
constexpr size_t kNoAllocStatusOff = (4u << 20) - 256;

// The table image reaches the static array through kernel parameters, in
// pieces of kNoAllocPiece bytes: no host buffer has to outlive the call and
// no pageable host-to-device copy (which would wait for the stream) is made.
constexpr int kNoAllocPiece = 30720;
struct alignas(16) NoAllocPiece {
  uint32_t off;       // byte offset in the table array (a multiple of 16)
  uint32_t n;         // bytes in this piece (a multiple of 16)
  uint32_t pad[2];
  uint8_t bytes[kNoAllocPiece];
};

__global__ void __launch_bounds__(256) k_noalloc_put(const __grid_constant__ NoAllocPiece c) {
  const uint4* src = reinterpret_cast<const uint4*>(c.bytes);
  uint4* dst = reinterpret_cast<uint4*>(ozaki2_noalloc_tables + c.off);
  for (uint32_t i = threadIdx.x; i < c.n / 16; i += blockDim.x) dst[i] = src[i];
}

struct NoAllocDevice {
  uint8_t* scratch = nullptr;
  uint8_t* tables = nullptr;
  int state = 0;   // 0: not set up, 1: ready, 2: set-up failed
};
NoAllocDevice g_noalloc_dev[64];
std::mutex g_noalloc_mu;

// Once per device, with that device current: the device addresses of the two
// arrays (in host code their names are only host-side stand-ins).
int noalloc_setup(int dev, NoAllocDevice** out) {
  if (dev < 0 || dev >= 64) return OZ2_ENODEV;
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  NoAllocDevice& d = g_noalloc_dev[dev];
  if (d.state == 0) {
    void* s = nullptr;
    void* t = nullptr;
    const cudaError_t e1 = cudaGetSymbolAddress(&s, ozaki2_noalloc_scratch);
    const cudaError_t e2 = e1 == cudaSuccess ? cudaGetSymbolAddress(&t, ozaki2_noalloc_tables) : e1;
    if (e1 == cudaSuccess && e2 == cudaSuccess && s && t) {
      d.scratch = static_cast<uint8_t*>(s);
      d.tables = static_cast<uint8_t*>(t);
      d.state = 1;
    } else {
      d.state = 2;
    }
  }
  *out = &d;
  return d.state == 1 ? OZ2_OK : OZ2_ECUDA;
}

int noalloc_device(NoAllocDevice** nd) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return OZ2_ENODEV;
  int major = 0;
  if (cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess || major != 10)
    return OZ2_ENODEV;
  return noalloc_setup(dev, nd);
}

int noalloc_run(int64_t M, int64_t N, int64_t K, int p, const ozaki2_mat* A, const ozaki2_mat* B,
                ozaki2_mat* C, cudaStream_t s) {
  NoAllocDevice* nd = nullptr;
  int rc = noalloc_device(&nd);
  if (rc) return rc;
  int dev = 0;
  cudaGetDevice(&dev);
  // host-side plan with the default options (no device memory is touched)
  ozaki2_opts o;
  ozaki2_opts_default(&o);
  ozaki2_plan_s* pl = nullptr;
  rc = new_plan(&o, &pl);
  if (rc) return rc;
  struct Release {
    ozaki2_plan_s* p;
    ~Release() { delete p; }   // host object only: its device pointers point into the static arrays
  } release{pl};
  rc = build_problem(pl, M, N, K, p);
  if (rc) return rc;
  layout_workspace(pl);
  if (pl->ws_bytes > sizeof(ozaki2_noalloc_scratch)) return OZ2_ERANGE;
  if (init_prep_attributes() != cudaSuccess || init_gemm_attributes() != cudaSuccess || init_gemm2_attributes() != cudaSuccess ||
      init_gemm_s8_attributes() != cudaSuccess ||
      init_crt_attributes() != cudaSuccess || !get_encode())
    return OZ2_ECUDA;
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  TableImage ti;
  rc = build_table_image(pl, sms, ti);
  if (rc) return rc;
  const size_t lb_off = align_up(ti.b.img.size(), 256);
  const size_t probs_bytes = align_up(sizeof(ProbDev), 128);
  const size_t lb_bytes = probs_bytes + kMapsPerProblem * sizeof(CUtensorMap);
  if (lb_off + lb_bytes > kNoAllocStatusOff) return OZ2_ERANGE;
  install_table_image(pl, ti, nd->tables);
  pl->dev.tab.status = reinterpret_cast<int32_t*>(nd->tables + kNoAllocStatusOff);
  const ozaki2_problem q{M, N, K, p, *A, *B, *C};
  std::vector<uint8_t> lbimg;
  rc = build_image(pl, &q, nd->scratch, lbimg, probs_bytes, lb_bytes);
  if (rc) return rc;
  // one image: tables + problem descriptor + tensor maps, put in place by
  // kernels on the stream (ordered behind earlier calls), then the status
  // word of this call cleared
  std::vector<uint8_t>& img = ti.b.img;
  img.resize(align_up(lb_off + lb_bytes, 16), 0);
  std::memcpy(img.data() + lb_off, lbimg.data(), lb_bytes);
  NoAllocPiece piece{};
  for (size_t off = 0; off < img.size(); off += kNoAllocPiece) {
    piece.off = (uint32_t)off;
    piece.n = (uint32_t)std::min<size_t>(kNoAllocPiece, img.size() - off);
    std::memcpy(piece.bytes, img.data() + off, piece.n);
    k_noalloc_put<<<1, 256, 0, s>>>(piece);
    if (cudaGetLastError() != cudaSuccess) return OZ2_ECUDA;
  }
  if (cudaMemsetAsync(nd->tables + kNoAllocStatusOff, 0, 4, s) != cudaSuccess) return OZ2_ECUDA;
  LaunchBlock lb;                       // not allocated: points into the static table array
  lb.d_mem = nd->tables + lb_off;
  lb.tmap_off = probs_bytes;
  lb.bytes = lb_bytes;
  rc = enqueue(pl, lb, nd->scratch, s, false);
  lb.d_mem = nullptr;
  return rc;
}

}  // namespace

extern "C" int ozaki2_gemm_noalloc(int64_t M, int64_t N, int64_t K, int p, const ozaki2_mat* A,
                                   const ozaki2_mat* B, ozaki2_mat* C, void* stream) {
  if (!A || !B || !C) return OZ2_EINVAL;
  try {
    return noalloc_run(M, N, K, p, A, B, C, static_cast<cudaStream_t>(stream));
  } catch (const std::bad_alloc&) {
    return OZ2_ENOMEM;
  }
}

extern "C" int ozaki2_noalloc_check(void* stream) {
  NoAllocDevice* nd = nullptr;
  int rc = noalloc_device(&nd);
  if (rc) return rc;
  if (cudaStreamSynchronize(static_cast<cudaStream_t>(stream)) != cudaSuccess) return OZ2_ECUDA;
  int32_t st = 0;
  if (cudaMemcpy(&st, nd->tables + kNoAllocStatusOff, 4, cudaMemcpyDeviceToHost) != cudaSuccess) return OZ2_ECUDA;
  if (st && cudaMemset(nd->tables + kNoAllocStatusOff, 0, 4) != cudaSuccess) return OZ2_ECUDA;
  if (st & kStatusTimeout) return OZ2_ETIMEOUT;
  if (st) return OZ2_EINTERNAL;
  return OZ2_OK;
}
