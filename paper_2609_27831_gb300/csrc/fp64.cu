// binary64 mode: C = A B for row-major double matrices through the exact
// Ozaki-II path at p = 53, with a cache of the forward's residue planes for
// the backward products dA = dC B^T and dB = A^T dC.
//
// The paper has no backward; the reading used here keeps every residue of the
// forward.  With b_kj ~ b_hat_kj 2^(f_j - t):
//   dA_ik = sum_j dC_ij b_kj ~ 2^-t sum_j (dC_ij 2^f_j) b_hat_kj,
// so D1 = dC diag(2^f) is integerized per row (its own shared exponents) and
// multiplied with the cached planes of B_hat (transposed, unscaled).  With
// a_ik ~ a_hat_ik 2^(e_i - t):
//   dB_kj = sum_i a_ik dC_ij ~ 2^-t sum_i a_hat_ik (2^e_i dC_ij),
// so D2 = diag(2^e) dC is integerized per column and multiplied with the
// cached planes of A_hat (transposed, unscaled).  The forward picks its
// modulus set for inner length max(M, N, K) so that the same planes serve all
// three products.
#include <algorithm>
#include <map>
#include <mutex>
#include <new>
#include <vector>

#include "oz2_internal.h"

namespace oz2 {

namespace {

constexpr int32_t kSentinel = (int32_t)0x80808080;   // exponent of an all-zero line

// double -> one-limb p = 53 format, times 2^shift where shift comes from a
// per-column (axis 1) or per-row (axis 0) exponent array; an element whose
// line exponent is the all-zero sentinel is set to 0 (its partner line is all
// zero, so it contributes nothing).
__global__ void k_f64_to_mp(const double* __restrict__ src, int64_t ld, int rows, int cols,
                            const int32_t* __restrict__ shift, int axis, uint64_t* __restrict__ limbs,
                            int32_t* __restrict__ exps, int8_t* __restrict__ signs) {
  const int64_t n = (int64_t)rows * cols;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(idx / cols), c = (int)(idx - (int64_t)r * cols);
    const double x = src[(int64_t)r * ld + c];
    const uint64_t bits = (uint64_t)__double_as_longlong(x);
    const int be = (int)((bits >> 52) & 0x7ff);
    uint64_t mant = bits & ((1ull << 52) - 1);
    uint64_t sig = 0;
    int e = 0;
    if (be == 0x7ff || (be == 0 && mant == 0)) {
      sig = 0;                                   // zero, Inf, NaN -> 0 (Sec. 10)
    } else if (be == 0) {
      const int lz = __clzll(mant);              // subnormal: normalise
      sig = mant << lz;
      e = -1021 - (lz - 11);
    } else {
      sig = ((1ull << 52) | mant) << 11;
      e = be - 1022;                             // |x| in [2^(e-1), 2^e)
    }
    if (sig && shift) {
      const int32_t s = shift[axis ? c : r];
      if (s == kSentinel) sig = 0;
      else e += s;
    }
    limbs[idx] = sig;
    exps[idx] = sig ? e : 0;
    signs[idx] = (sig && (bits >> 63)) ? 1 : 0;
  }
}

// Plane transpose: src [G][R][src_pitch] (R rows, K valid columns) ->
// dst [G][K][dst_pitch] (K rows, R valid columns).
__global__ void k_transpose_planes(const uint16_t* __restrict__ src, int64_t src_pitch, int R, int K,
                                   uint16_t* __restrict__ dst, int64_t dst_pitch) {
  __shared__ uint16_t tile[32][33];
  const int g = blockIdx.z;
  const int r0 = blockIdx.y * 32, k0 = blockIdx.x * 32;
  const uint16_t* s = src + (int64_t)g * R * src_pitch;
  uint16_t* d = dst + (int64_t)g * K * dst_pitch;
  for (int i = threadIdx.y; i < 32; i += 8) {
    const int r = r0 + i, k = k0 + threadIdx.x;
    tile[i][threadIdx.x] = (r < R && k < K) ? s[(int64_t)r * src_pitch + k] : 0;
  }
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += 8) {
    const int k = k0 + i, r = r0 + threadIdx.x;
    if (k < K && r < R) d[(int64_t)k * dst_pitch + r] = tile[threadIdx.x][i];
  }
}

cudaError_t to_mp(const double* src, int64_t ld, int rows, int cols, const int32_t* shift, int axis,
                  uint64_t* limbs, int32_t* exps, int8_t* signs, cudaStream_t s) {
  const int64_t n = (int64_t)rows * cols;
  const int blocks = (int)std::min<int64_t>((n + 255) / 256, 148 * 32);
  k_f64_to_mp<<<blocks, 256, 0, s>>>(src, ld, rows, cols, shift, axis, limbs, exps, signs);
  return cudaGetLastError();
}

cudaError_t transpose_planes(const uint16_t* src, int64_t src_pitch, int R, int K, int G, uint16_t* dst,
                             int64_t dst_pitch, cudaStream_t s) {
  dim3 grid((K + 31) / 32, (R + 31) / 32, G);
  k_transpose_planes<<<grid, dim3(32, 8), 0, s>>>(src, src_pitch, R, K, dst, dst_pitch);
  return cudaGetLastError();
}

size_t al(size_t x) { return (x + 255) / 256 * 256; }

// One-limb matrix buffers inside a device allocation.
struct MpBuf {
  uint64_t* limbs = nullptr;
  int32_t* exp = nullptr;
  int8_t* sign = nullptr;
  int rows = 0, cols = 0;
  static size_t bytes(int r, int c) { return al(8ull * r * c) + al(4ull * r * c) + al((size_t)r * c); }
  void place(uint8_t* base, int r, int c) {
    rows = r; cols = c;
    limbs = reinterpret_cast<uint64_t*>(base);
    exp = reinterpret_cast<int32_t*>(base + al(8ull * r * c));
    sign = reinterpret_cast<int8_t*>(base + al(8ull * r * c) + al(4ull * r * c));
  }
  ozaki2_mat mat() const {
    return ozaki2_mat{limbs, exp, sign, cols, (int64_t)rows * cols};
  }
};

}  // namespace

}  // namespace oz2

struct ozaki2_cache_s {
  int64_t M = 0, N = 0, K = 0;
  ozaki2_opts opts{};
  ozaki2_plan fwd = nullptr, bwd_a = nullptr, bwd_b = nullptr;
  oz2::PlanFacts ff{}, fa{}, fb{};
  void* mem = nullptr;          // fwd workspace + A/B conversions
  void* mem_bwd = nullptr;      // backward workspaces + dC conversion
  size_t bwd_bytes = 0;
  oz2::MpBuf a, b;
};

namespace oz2 {
namespace {

int cache_release(ozaki2_cache_s* c) {
  if (!c) return OZ2_EINVAL;
  if (c->mem || c->mem_bwd) cudaDeviceSynchronize();
  if (c->fwd) ozaki2_plan_destroy(c->fwd);
  if (c->bwd_a) ozaki2_plan_destroy(c->bwd_a);
  if (c->bwd_b) ozaki2_plan_destroy(c->bwd_b);
  if (c->mem) cudaFree(c->mem);
  if (c->mem_bwd) cudaFree(c->mem_bwd);
  delete c;
  return OZ2_OK;
}

int cache_build(int64_t M, int64_t N, int64_t K, const ozaki2_opts* opts, ozaki2_cache_s** out) {
  if (M <= 0 || N <= 0 || K <= 0) return OZ2_EINVAL;
  if (M > INT32_MAX / 2 || N > INT32_MAX / 2 || K > INT32_MAX / 2) return OZ2_ERANGE;
  auto* c = new (std::nothrow) ozaki2_cache_s();
  if (!c) return OZ2_ENOMEM;
  c->M = M; c->N = N; c->K = K;
  if (opts) c->opts = *opts;
  else ozaki2_opts_default(&c->opts);
  PlanExtra ex;
  ex.inner = std::max(M, std::max(N, K));
  ex.kind = 1;
  int rc = plan_create_ex(M, N, K, 53, &c->opts, ex, &c->fwd);
  if (!rc) rc = plan_query(c->fwd, &c->ff);
  if (rc) { cache_release(c); return rc; }
  const size_t bytes = al(c->ff.ws_bytes) + MpBuf::bytes((int)M, (int)K) + MpBuf::bytes((int)K, (int)N);
  if (cudaMalloc(&c->mem, bytes) != cudaSuccess) { c->mem = nullptr; cache_release(c); return OZ2_ENOMEM; }
  auto* base = static_cast<uint8_t*>(c->mem);
  c->a.place(base + al(c->ff.ws_bytes), (int)M, (int)K);
  c->b.place(base + al(c->ff.ws_bytes) + MpBuf::bytes((int)M, (int)K), (int)K, (int)N);
  *out = c;
  return OZ2_OK;
}

int run_fwd(ozaki2_cache_s* c, const double* A, int64_t lda, const double* B, int64_t ldb, double* Cd,
            int64_t ldc, cudaStream_t s) {
  if (!A || !B || !Cd || lda < c->K || ldb < c->N || ldc < c->N) return OZ2_EINVAL;
  if (to_mp(A, lda, (int)c->M, (int)c->K, nullptr, 0, c->a.limbs, c->a.exp, c->a.sign, s) != cudaSuccess ||
      to_mp(B, ldb, (int)c->K, (int)c->N, nullptr, 0, c->b.limbs, c->b.exp, c->b.sign, s) != cudaSuccess)
    return OZ2_ECUDA;
  ozaki2_problem q{};
  q.M = c->M; q.N = c->N; q.K = c->K; q.p = 53;
  q.A = c->a.mat();
  q.B = c->b.mat();
  q.C = ozaki2_mat{reinterpret_cast<uint64_t*>(Cd), nullptr, nullptr, ldc, 0};
  return plan_run(c->fwd, &q, c->mem, c->ff.ws_bytes, s);
}

int ensure_bwd(ozaki2_cache_s* c) {
  if (c->mem_bwd) return OZ2_OK;
  PlanExtra ea;
  ea.force_t = c->ff.t; ea.force_L = c->ff.L; ea.kind = 1; ea.skip_b = true;
  int rc = plan_create_ex(c->M, c->K, c->N, 53, &c->opts, ea, &c->bwd_a);   // dA = D1 (M x N) * B_hat^T
  if (!rc) rc = plan_query(c->bwd_a, &c->fa);
  PlanExtra eb;
  eb.force_t = c->ff.t; eb.force_L = c->ff.L; eb.kind = 1; eb.skip_a = true;
  if (!rc) rc = plan_create_ex(c->K, c->N, c->M, 53, &c->opts, eb, &c->bwd_b);   // dB = A_hat^T * D2 (M x N)
  if (!rc) rc = plan_query(c->bwd_b, &c->fb);
  if (rc) return rc;
  c->bwd_bytes = al(c->fa.ws_bytes) + al(c->fb.ws_bytes) + MpBuf::bytes((int)c->M, (int)c->N);
  if (cudaMalloc(&c->mem_bwd, c->bwd_bytes) != cudaSuccess) { c->mem_bwd = nullptr; return OZ2_ENOMEM; }
  return OZ2_OK;
}

int run_bwd(ozaki2_cache_s* c, const double* dC, int64_t lddc, double* dA, int64_t ldda, double* dB,
            int64_t lddb, cudaStream_t s) {
  if (!dC || lddc < c->N) return OZ2_EINVAL;
  if ((dA && ldda < c->K) || (dB && lddb < c->N)) return OZ2_EINVAL;
  int rc = ensure_bwd(c);
  if (rc) return rc;
  auto* fw = static_cast<uint8_t*>(c->mem);
  auto* bw = static_cast<uint8_t*>(c->mem_bwd);
  uint8_t* ws_a = bw;
  uint8_t* ws_b = bw + al(c->fa.ws_bytes);
  MpBuf d;
  d.place(bw + al(c->fa.ws_bytes) + al(c->fb.ws_bytes), (int)c->M, (int)c->N);
  const int32_t* e_fwd = reinterpret_cast<const int32_t*>(fw + c->ff.off_e);
  const int32_t* f_fwd = reinterpret_cast<const int32_t*>(fw + c->ff.off_f);
  const auto* pa_fwd = reinterpret_cast<const uint16_t*>(fw + c->ff.off_pa);
  const auto* pb_fwd = reinterpret_cast<const uint16_t*>(fw + c->ff.off_pb);
  const int M = (int)c->M, N = (int)c->N, K = (int)c->K, G = c->ff.G;
  if (dA) {
    // D1 = dC diag(2^f) ; B-side planes = B_hat planes [G][N][Kp] transposed to [G][K][Np]
    if (to_mp(dC, lddc, M, N, f_fwd, 1, d.limbs, d.exp, d.sign, s) != cudaSuccess) return OZ2_ECUDA;
    if (transpose_planes(pb_fwd, c->ff.Kp, N, K, G, reinterpret_cast<uint16_t*>(ws_a + c->fa.off_pb),
                         c->fa.Kp, s) != cudaSuccess)
      return OZ2_ECUDA;
    ozaki2_problem q{};
    q.M = c->M; q.N = c->K; q.K = c->N; q.p = 53;
    q.A = d.mat();
    q.C = ozaki2_mat{reinterpret_cast<uint64_t*>(dA), nullptr, nullptr, ldda, 0};
    rc = plan_run(c->bwd_a, &q, ws_a, c->fa.ws_bytes, s);
    if (rc) return rc;
  }
  if (dB) {
    // D2 = diag(2^e) dC ; A-side planes = A_hat planes [G][M][Kp] transposed to [G][K][Mp]
    if (to_mp(dC, lddc, M, N, e_fwd, 0, d.limbs, d.exp, d.sign, s) != cudaSuccess) return OZ2_ECUDA;
    if (transpose_planes(pa_fwd, c->ff.Kp, M, K, G, reinterpret_cast<uint16_t*>(ws_b + c->fb.off_pa),
                         c->fb.Kp, s) != cudaSuccess)
      return OZ2_ECUDA;
    ozaki2_problem q{};
    q.M = c->K; q.N = c->N; q.K = c->M; q.p = 53;
    q.B = d.mat();
    q.C = ozaki2_mat{reinterpret_cast<uint64_t*>(dB), nullptr, nullptr, lddb, 0};
    rc = plan_run(c->bwd_b, &q, ws_b, c->fb.ws_bytes, s);
    if (rc) return rc;
  }
  return OZ2_OK;
}

std::mutex g_mu;
std::map<std::vector<int64_t>, ozaki2_cache_s*> g_nocache;   // forwards without a cache handle

}  // namespace
}  // namespace oz2

using namespace oz2;

extern "C" {

int ozaki2_dgemm_fwd(int64_t M, int64_t N, int64_t K, const double* A, int64_t lda, const double* B,
                     int64_t ldb, double* Cd, int64_t ldc, const ozaki2_opts* opts, ozaki2_cache* cache_out,
                     void* stream) {
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  try {
    if (cache_out) {
      *cache_out = nullptr;
      ozaki2_cache_s* c = nullptr;
      int rc = cache_build(M, N, K, opts, &c);
      if (rc) return rc;
      rc = run_fwd(c, A, lda, B, ldb, Cd, ldc, s);
      if (rc) { cache_release(c); return rc; }
      *cache_out = c;
      return OZ2_OK;
    }
    ozaki2_opts o;
    if (opts) o = *opts;
    else ozaki2_opts_default(&o);
    int dev = -1;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(g_mu);
    const std::vector<int64_t> key{dev, M, N, K, o.guard_bits, o.t_bits, o.engine, o.k_chunk, o.grid, o.schedule,
                                    o.crt_engine, o.res_engine};
    auto it = g_nocache.find(key);
    if (it == g_nocache.end()) {
      ozaki2_cache_s* c = nullptr;
      const int rc = cache_build(M, N, K, &o, &c);
      if (rc) return rc;
      it = g_nocache.emplace(key, c).first;
    }
    return run_fwd(it->second, A, lda, B, ldb, Cd, ldc, s);
  } catch (const std::bad_alloc&) {
    return OZ2_ENOMEM;
  }
}

int ozaki2_dgemm_bwd(ozaki2_cache cache, const double* dC, int64_t lddc, double* dA, int64_t ldda, double* dB,
                     int64_t lddb, void* stream) {
  if (!cache) return OZ2_EINVAL;
  try {
    return run_bwd(cache, dC, lddc, dA, ldda, dB, lddb, static_cast<cudaStream_t>(stream));
  } catch (const std::bad_alloc&) {
    return OZ2_ENOMEM;
  }
}

int ozaki2_cache_destroy(ozaki2_cache cache) { return cache_release(cache); }

}  // extern "C"
