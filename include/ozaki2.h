/*
 * ozaki2.h -- C ABI of the GB300 Ozaki-scheme-II multiple-precision GEMM.
 *
 * The library computes C = A * B for p-bit floating-point matrices
 * (p = 2 .. 2048) with the Ozaki scheme II of "Ozaki Scheme II Is Fast on CPUs
 * Too" (Kouya, 2026): shared-exponent integerization (Sec. 4.2, Eq. 1-3),
 * centered residues over the pairwise-coprime modulus set of Sec. 4.3 (54
 * one-limb moduli <= 255, then two-limb primes <= 16191 split in balanced base
 * 128 with the 3-GEMM Karatsuba combine of Eq. 4-5), one exact integer GEMM
 * per plane on the sm_103a tensor cores, mod-reduction of each product, the
 * direct CRT of Sec. 4.4 and one final round-to-nearest-even to p bits.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Every call returns an int status (OZ2_OK = 0 or one of the OZ2_E* codes
 *   below); nothing aborts and no C++ exception crosses this boundary.
 * - Device work is enqueued on the given stream (a cudaStream_t; NULL is the
 *   legacy default stream) and runs asynchronously.  Argument errors are
 *   reported before anything is enqueued.  Errors detected on the device
 *   (a range check of the CRT failing, a wait that timed out) set a status
 *   word that ozaki2_check() reads after synchronising the stream.
 * - All matrix pointers are device pointers owned by the caller; the library
 *   never frees them.  Plans, caches and graphs are owned by the library and
 *   released by their destroy calls.
 * - A plan may be executed many times but not concurrently from two host
 *   threads or on two streams at once.
 *
 * Matrix storage (ozaki2_mat), row-major, struct of arrays:
 *   element (i, j) has nl = ceil(p/64) limbs, limb q at
 *       limbs[q * plane_stride + i * ld + j]           (uint64, least significant first)
 *   and exponent exp[i * ld + j], sign sign[i * ld + j] (0 = +, 1 = -).
 *   Value = (-1)^sign * (sum_q limb_q 2^(64 q)) * 2^(exp - 64 nl), the MPFR
 *   convention |x| in [2^(exp-1), 2^exp).  A nonzero significand has bit 63 of
 *   its top limb set (MSB-normalised); an element whose top limb is zero is
 *   zero (its other limbs, exp and sign are ignored).  Inf/NaN are not
 *   representable (the paper treats them as 0, Sec. 10).  |exp| <= 2^28.
 *   Outputs are written MSB-normalised with the 64 nl - p low bits zero;
 *   a zero output has all limbs 0, exp 0 and sign 0.
 */
#ifndef OZAKI2_H
#define OZAKI2_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define OZ2_API __attribute__((visibility("default")))
#else
#define OZ2_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. */
enum {
  OZ2_OK = 0,
  OZ2_EINVAL = 1,    /* null pointer, size <= 0, p < 2, bad option, workspace too small */
  OZ2_ERANGE = 2,    /* K > 133000 (int32 exactness cap, Sec. 4.3(a)), p > 2048, or the
                        modulus table cannot reach the CRT bound (Eq. crtcond) */
  OZ2_ENOMEM = 3,    /* a library-owned allocation failed */
  OZ2_ECUDA = 4,     /* a CUDA runtime/driver call failed */
  OZ2_EINTERNAL = 5, /* a device-side consistency check failed (status word set) */
  OZ2_ETIMEOUT = 6,  /* a bounded device-side wait gave up (status word set) */
  OZ2_ENODEV = 7     /* no usable sm_103 device */
};

/* GEMM engines for the per-plane products. */
enum {
  OZ2_ENGINE_TC = 0,   /* tcgen05 kind::f16 tensor-core kernel (TMA + TMEM), default */
  OZ2_ENGINE_SIMT = 1, /* CUDA-core int32 kernel: slow cross-check engine */
  OZ2_ENGINE_S8 = 2    /* INT8 x INT8 -> INT32 on the warp-level tensor-core instruction
                          mma.sync m16n8k32 (sm_103a has no tcgen05 INT8 form): the second
                          engine, for comparison at equal accuracy; bf16 planes converted to
                          int8 while staged in shared memory */
};

/* Plane schedules. */
enum {
  OZ2_SCHED_GROUPED = 0, /* all planes of all problems in one persistent launch */
  OZ2_SCHED_PLAIN = 1    /* one GEMM launch per modulus per problem */
};

typedef struct {
  uint64_t* limbs;
  int32_t* exp;
  int8_t* sign;
  int64_t ld;           /* row stride in elements (>= number of columns) */
  int64_t plane_stride; /* elements between limb planes (>= rows * ld) */
} ozaki2_mat;

typedef struct {
  int guard_bits; /* g of Eq. 3, default 16 */
  int t_bits;     /* 0: t = p + g + ceil(log2 K) (Eq. 3); > 0 forces t */
  int engine;     /* OZ2_ENGINE_* */
  int k_chunk;    /* K per exact fp32 accumulation chunk: multiple of 64, <= 1024;
                     0 = 1024 (127^2 * 1024 + 16191 < 2^24 keeps every partial sum exact) */
  int grid;       /* persistent CTAs of the grouped GEMM; 0 = one per SM */
  int schedule;   /* OZ2_SCHED_* */
  int timing;     /* nonzero: record per-stage CUDA events (ozaki2_last_timings) */
  int crt_engine; /* 0: automatic (default): engine 2 where the CRT accumulator needs more than
                     20 32-bit digits (p above about 240), CUDA cores otherwise; 1: CRT column sums as an exact bf16
                     GEMM on the tensor cores where 2L <= 256, the accumulator has <= 40 digits
                     and the tables fit in shared memory (CUDA cores otherwise); 2: the column
                     sums of any length as an exact bf16 GEMM on the tensor cores, written as
                     group sums to the workspace and finished on the CUDA cores, where
                     32 <= L <= 448 and M N >= 128 (CUDA cores otherwise);
                     3: the CRT on the CUDA cores only */
  int res_engine; /* 0: automatic (default): engine 2 for integers of more than 72 bytes
                     (p above about 550), CUDA cores otherwise; 1: residues as an exact bf16
                     GEMM of the bytes of a_hat with a table of centered 2^(8b) mod m on the
                     tensor cores where the table has <= 256 rows and <= 256 bytes (CUDA cores
                     otherwise); 2: the same GEMM, warp-specialised (bytes in tensor memory, table
                     streamed), for integers of up to 448 bytes; 3: CUDA cores only */
  int plane_group; /* residue planes streamed through the workspace in groups of consecutive
                     moduli (single-product plans with the tensor-core engine and the grouped
                     schedule; batched plans ignore it): 0 automatic (default): one group while
                     the bf16 plane stacks of A and B fit in 32 GiB, else groups of at most that
                     size; -1: never (one group); >= 3: at most this many planes per group.
                     Each group computes its moduli's residues and plane products before the next
                     starts; the CRT runs once over all moduli.  Bits are identical either way. */
  int gemm_tile;  /* output tile of the tensor-core plane GEMMs: 0 automatic (default); 1: 128 x 256
                     tiles, one SM each; 2: 256 x 256 tiles on CTA pairs (clusters of two SMs,
                     tcgen05 cta_group::2), each SM holding its 128 rows of A and half of B.  The
                     SIMT engine uses 1.  Bits are identical either way. */
} ozaki2_opts;

/* Facts about a plan (all computed on the host at plan creation). */
typedef struct {
  int count;        /* problems in the plan (1 for a single GEMM) */
  int t;            /* internal width of problem 0 (Eq. 3) */
  int L;            /* moduli of problem 0 */
  int L1;           /* one-limb moduli among them */
  int G;            /* int8 planes (GEMMs) of problem 0: L1 + 3 (L - L1) */
  int crt_digits;   /* 32-bit digits of the CRT accumulator: ceil(bits(P)/32) + 2 */
  int units;        /* (modulus, output tile) work units over all problems */
  int jobs;         /* tensor-core accumulation jobs over all problems */
  size_t workspace_bytes;
  int crt_mode;     /* CRT path of problem 0: 0 CUDA cores, 1 tensor-core column sums in one
                       kernel, 2 tensor-core sums of any length plus the finish (see crt_engine) */
  int res_mode;     /* residue path of problem 0: 0 CUDA cores, 1 or 2 tensor cores (res_engine) */
  int plane_groups; /* modulus groups the planes of problem 0 are streamed in (1: not streamed) */
  int group_planes; /* planes of the largest group (= G when not streamed) */
  int gemm_tile;    /* plane GEMM tile in use: 1 (128 x 256, one SM) or 2 (256 x 256, CTA pairs) */
  int crt_skip_groups; /* crt_mode 2 with the long finish: groups of 32 column sums (7-bit pieces
                       of P) below the ones the finish's fast form reads, not formed (0: none) */
} ozaki2_info;

typedef struct {
  int64_t M, N, K;
  int p;
  ozaki2_mat A; /* M x K */
  ozaki2_mat B; /* K x N */
  ozaki2_mat C; /* M x N (written) */
} ozaki2_problem;

typedef struct ozaki2_plan_s* ozaki2_plan;
typedef struct ozaki2_cache_s* ozaki2_cache;
typedef struct ozaki2_graph_s* ozaki2_graph;

/* Fill *o with the defaults (g = 16, auto t, tensor-core engine, k_chunk 1024,
   one CTA per SM, grouped schedule, no timing).  Host only. */
OZ2_API int ozaki2_opts_default(ozaki2_opts* o);

/* Human-readable text of a status code (static storage). */
OZ2_API const char* ozaki2_strerror(int status);

/* Create a plan for one M x N x K product at p bits (Sec. 4.1 flow).  Host
   only: chooses t (Eq. 3) and the shortest modulus prefix with
   log2 P > 2t + log2 K + 2 (Sec. 4.3), builds the CRT tables (Sec. 4.4) and
   the tile schedule.  Device tables are uploaded lazily by the first execute
   on the device that is current then.  opts may be NULL (defaults). */
OZ2_API int ozaki2_plan_create(int64_t M, int64_t N, int64_t K, int p, const ozaki2_opts* opts,
                       ozaki2_plan* out);

/* Plan for `count` independent products (only M, N, K, p of each problem are
   read).  All of them run in one grouped persistent launch per stage. */
OZ2_API int ozaki2_plan_create_batched(int count, const ozaki2_problem* shapes, const ozaki2_opts* opts,
                               ozaki2_plan* out);

/* The same with per-problem choices (an autotuner's per-class table):
   per_problem[i] supplies problem i's guard_bits, t_bits, k_chunk,
   crt_engine and res_engine (its other fields are ignored); the launch-wide
   options (engine, grid, schedule, timing, plane GEMM tile) come from opts.
   per_problem may be NULL (= ozaki2_plan_create_batched). */
OZ2_API int ozaki2_plan_create_batched_ex(int count, const ozaki2_problem* shapes, const ozaki2_opts* opts,
                                          const ozaki2_opts* per_problem, ozaki2_plan* out);

OZ2_API int ozaki2_plan_destroy(ozaki2_plan plan);

/* Host-side facts; see ozaki2_info. */
OZ2_API int ozaki2_plan_info(ozaki2_plan plan, ozaki2_info* out);

/* Copy the moduli of problem `prob` (in plane order) into out[0..cap). Host only. */
OZ2_API int ozaki2_plan_moduli(ozaki2_plan plan, int prob, int32_t* out, int cap);

/* Host copies of problem `prob`'s CRT tables (Sec. 4.4): P as crt_digits
   little-endian 32-bit digits, M_l = P / m_l as L x crt_digits digits
   (row l), and M_l^{-1} mod m_l.  Any output may be NULL.  Host only. */
OZ2_API int ozaki2_plan_crt_tables(ozaki2_plan plan, int prob, uint32_t* P_digits, uint32_t* M_digits,
                           uint32_t* Minv);

/* Byte offsets of the workspace regions of problem `prob` (for inspection of
   intermediates after an execute; when the planes are streamed in groups the
   plane regions hold the last group's planes, group_planes of them):
     off[0] row exponents e   int32 [M]
     off[1] column exponents f int32 [N]
     off[2] A planes  bf16 [G][M][Kp]   (Kp = K rounded up to 8; K-major)
     off[3] B planes  bf16 [G][N][Kp]   (transposed: column j of B is row j)
     off[4] reduced products v  uint16 [L][MNp], MNp = M*N rounded up to a multiple of 8
            (row-major (i, j) within each modulus row): v_l = u_l M_l^{-1} mod m_l,
            u_l = c mod m_l the reduced product, M_l = P / m_l (the CRT's first step)
   and *kp = Kp.  Plane order: one-limb moduli in plane order, then for each
   two-limb modulus the planes r0, r1, r0 + r1 (balanced base-128 split). */
OZ2_API int ozaki2_plan_layout(ozaki2_plan plan, int prob, size_t off[5], int64_t* kp);

/* Number of kernel launches of this library per execute of the plan (the
   workspace memsets are not counted).  Known once the plan has run
   (OZ2_EINVAL before the first execute). */
OZ2_API int ozaki2_plan_launches(ozaki2_plan plan, int* n);

/* Debugging aid: when dev_buf is not NULL, later executes also write the
   CRT integer c_hat of every output of problem `prob` to dev_buf (device,
   uint32 [M*N][crt_digits + 1]: word 0 = 1 for a negative c_hat, then
   |c_hat| as crt_digits little-endian digits), row-major over (i, j). */
OZ2_API int ozaki2_plan_set_debug_chat(ozaki2_plan plan, int prob, uint32_t* dev_buf);

/* Fault injection and failure detection (debugging aids; the paper has none).
   Every failure is made on the host; no GPU fault is involved. */

/* The number of polls of every bounded device-side wait (mbarrier waits of
   the tensor-core kernels) in later executes of this plan; 0 restores the
   default (2^26).  A wait that runs out sets the device status word
   (ozaki2_check then returns OZ2_ETIMEOUT), the kernel drains the copies and
   MMAs it has in flight, frees its tensor memory and returns; the product's
   output is then undefined.  Host only. */
OZ2_API int ozaki2_plan_set_wait_limit(ozaki2_plan plan, uint32_t polls);

/* Corrupt problem `prob`'s CRT tables on the host before they are uploaded
   (OZ2_EINVAL after the plan's first execute): the top 32-bit digit of
   M_0 = P / m_0 (and its top 7-bit piece in the tensor-core table) has one
   bit flipped, so the direct CRT's range check (x0 < P, Sec. 4.4) fails on
   the device and ozaki2_check returns OZ2_EINTERNAL.  Host only. */
OZ2_API int ozaki2_plan_debug_corrupt_crt(ozaki2_plan plan, int prob);

/* Make the next `count` library allocations (host plan construction, the
   device tables of a plan's first execute, launch images) fail with
   OZ2_ENOMEM without allocating; 0 cancels.  Nothing half-made is kept: a
   later call with the same arguments starts over. */
OZ2_API int ozaki2_debug_inject_alloc_failure(int count);

/* Debugging aid: when dev_buf is not NULL, later executes of the tensor-core
   engine also write the exact sum of every plane product before any
   reduction, C_g[i][j] = sum_k r_a[g][i][k] r_b[g][k][j] (Sec. 2.4: the
   integer GEMM output of plane g), to dev_buf (device, int32 [G][M][N],
   plane order as in ozaki2_plan_layout).  Only for problems whose K fits in
   one exact accumulation chunk (K <= k_chunk); OZ2_EINVAL otherwise. */
OZ2_API int ozaki2_plan_set_debug_prods(ozaki2_plan plan, int prob, int32_t* dev_buf);

/* Run the plan: C = A * B rounded to p bits, via workspace `ws` (device,
   >= info.workspace_bytes, 256-byte aligned, caller-owned, contents need not
   be initialised and are clobbered).  Single-problem plans only. */
OZ2_API int ozaki2_execute(ozaki2_plan plan, const ozaki2_mat* A, const ozaki2_mat* B, ozaki2_mat* C,
                   void* ws, size_t ws_bytes, void* stream);

/* Run a batched plan on `count` problems with the planned shapes. */
OZ2_API int ozaki2_execute_batched(ozaki2_plan plan, int count, const ozaki2_problem* probs, void* ws,
                           size_t ws_bytes, void* stream);

/* Operand reuse (the paper's Sec. 11 names reusing the residues of one
   operand across products as future work): C = A X (keep = 0) or C = X B
   (keep = 1) with the plan's shape, keeping the row exponents and residue
   planes of A (keep = 0) or the column exponents and planes of B (keep = 1)
   that the previous execute of this single-problem plan left in the same
   workspace `ws`; only X is scanned, integerized and reduced.  X has the shape
   of the replaced operand (K x N for keep = 0, M x K for keep = 1).  The
   workspace must not have been used by anything else in between (the library
   checks only that the pointer is the same).  OZ2_EINVAL without a previous
   execute with this workspace, for batched plans, for plans whose planes are
   streamed in modulus groups (only the last group's planes stay), and for the
   binary64 mode's internal plans.  The result is bit-identical to a full
   execute with the same operands. */
OZ2_API int ozaki2_execute_reuse(ozaki2_plan plan, int keep, const ozaki2_mat* X, ozaki2_mat* C, void* ws,
                                 size_t ws_bytes, void* stream);

/* Capture one execute of a (batched or single) plan with fixed pointers into
   a CUDA graph; ozaki2_graph_launch replays it on any stream. */
OZ2_API int ozaki2_graph_create(ozaki2_plan plan, int count, const ozaki2_problem* probs, void* ws,
                        size_t ws_bytes, void* stream, ozaki2_graph* out);
OZ2_API int ozaki2_graph_launch(ozaki2_graph g, void* stream);
OZ2_API int ozaki2_graph_destroy(ozaki2_graph g);

/* Convenience single call: C = A * B at p bits with a plan and workspace
   cached by the library (library-owned device memory, kept until
   ozaki2_release_cache()). */
OZ2_API int ozaki2_gemm(int64_t M, int64_t N, int64_t K, int p, const ozaki2_mat* A, const ozaki2_mat* B,
                ozaki2_mat* C, const ozaki2_opts* opts, void* stream);

/* C = A * B at p bits, like ozaki2_gemm, for callers that cannot allocate
   device memory (a memory-capped or custom-allocator setting, or a thread
   that must not call cudaMalloc/cudaFree because they synchronise the
   device).  The paper has no counterpart: this is a deployment variant.
   Nothing is allocated on the device: the intermediates (exponents, residue
   planes, reduced products) live in a fixed 64 MiB array and the tables,
   schedule, problem descriptor and TMA descriptors in a fixed 4 MiB array,
   both static device memory of this library that every GPU loading the
   library holds until the process exits.  Products whose intermediates need
   more (ozaki2_info.workspace_bytes of the same shape above 64 MiB, e.g.
   1024^3 at p = 256) are rejected with OZ2_ERANGE before any device work.
   The first call on a device looks up the arrays' device addresses (once per
   device, with that device current).  Each call writes its tables into the
   array with small kernels on `stream` (their parameters carry the bytes), so
   it does not wait on the host for earlier work on the stream.  Every call
   shares the arrays and rewrites them: calls that overlap on the GPU
   (different streams, or concurrent host threads) race, so order them on one
   stream.  Default options.  The device status word of the most recent call on the current
   device (cleared at the start of each call) is read by ozaki2_noalloc_check. */
OZ2_API int ozaki2_gemm_noalloc(int64_t M, int64_t N, int64_t K, int p, const ozaki2_mat* A,
                                const ozaki2_mat* B, ozaki2_mat* C, void* stream);

/* Synchronise `stream` and read (then clear) the device status word of the
   last ozaki2_gemm_noalloc call on the current device: OZ2_OK, OZ2_EINTERNAL
   (a device-side consistency check failed) or OZ2_ETIMEOUT (a bounded wait
   gave up).  Allocates nothing. */
OZ2_API int ozaki2_noalloc_check(void* stream);

/* ---------------------------------------------------------------------------
 * Complex products in 3M form in the residue domain (the paper names complex
 * 3M/4M products as future work, Sec. 11): C = (Ar + i Ai)(Br + i Bi) for
 * p-bit parts.  Rows of Ar and Ai share one exponent, columns of Br and Bi
 * one, so that Cr_hat = sum ar br - ai bi and Ci_hat = sum ar bi + ai br are
 * exact integers below 2K 2^(2t) (t and the moduli chosen for inner length
 * 2K); per modulus three plane products, T1 = ar br, T2 = ai bi and
 * T3 = (ar + ai)(br + bi) (the sums' residue planes formed from the parts'),
 * then u_r = T1 - T2 and u_i = T3 - T1 - T2 mod m, the direct CRT of each and
 * one rounding of each part to p bits.
 * ------------------------------------------------------------------------- */

/* A plan of three real products (Ar Br, Ai Bi and the sums' product) sharing
   the exponents; ozaki2_plan_info reports count 3.  Host only. */
OZ2_API int ozaki2_plan_create_complex(int64_t M, int64_t N, int64_t K, int p, const ozaki2_opts* opts,
                                       ozaki2_plan* out);

/* Run a complex plan (workspace as for ozaki2_execute).  Cr and Ci are M x N
   p-bit matrices written with the real and imaginary parts. */
OZ2_API int ozaki2_execute_complex(ozaki2_plan plan, const ozaki2_mat* Ar, const ozaki2_mat* Ai,
                                   const ozaki2_mat* Br, const ozaki2_mat* Bi, ozaki2_mat* Cr, ozaki2_mat* Ci,
                                   void* ws, size_t ws_bytes, void* stream);

/* Convenience call with a library-owned plan and workspace (as ozaki2_gemm). */
OZ2_API int ozaki2_zgemm(int64_t M, int64_t N, int64_t K, int p, const ozaki2_mat* Ar, const ozaki2_mat* Ai,
                         const ozaki2_mat* Br, const ozaki2_mat* Bi, ozaki2_mat* Cr, ozaki2_mat* Ci,
                         const ozaki2_opts* opts, void* stream);

/* Convenience batched call (library-owned plan and workspace). */
OZ2_API int ozaki2_gemm_batched(int count, const ozaki2_problem* probs, const ozaki2_opts* opts,
                        void* stream);

/* Free the plans and workspaces cached by ozaki2_gemm / ozaki2_gemm_batched. */
OZ2_API int ozaki2_release_cache(void);

/* Synchronise `stream` and read the plan's device status word:
   OZ2_OK, OZ2_EINTERNAL or OZ2_ETIMEOUT.  Clears the word. */
OZ2_API int ozaki2_check(ozaki2_plan plan, void* stream);

/* Per-stage device times of the plan's last execute with opts.timing set, in
   milliseconds: [0] exponent scan, [1] residues (integerize + centered
   residues + plane writes), [2] plane GEMMs with fused mod-reduce, [3] CRT and
   rounding, [4] total.  Synchronises on the recorded events. */
OZ2_API int ozaki2_last_timings(ozaki2_plan plan, float ms[5]);

/* The CRT stage of the same execute split in two, in milliseconds: [0] the
   column sums on the tensor cores (crt_engine 2; about 0 where none ran),
   [1] the rest (the finish from the group sums, or the whole CUDA-core CRT).
   Synchronises on the recorded events. */
OZ2_API int ozaki2_last_crt_split(ozaki2_plan plan, float ms[2]);

/* ---------------------------------------------------------------------------
 * binary64 mode (p = 53): C = A B for row-major double matrices, computed
 * through the same exact path, with a cache of the forward's int8 residue
 * planes for the backward.  Readings for the backward (the paper has none):
 * dA = dC B^T reuses the cached planes of B (scaled per column j by 2^f_j),
 * with dC scaled by 2^f_j per column and integerized per row; dB = A^T dC
 * reuses the cached planes of A, with dC scaled by 2^e_i per row and
 * integerized per column.  The forward's modulus set is chosen to cover all
 * three products.  Results are rounded to nearest-even binary64.
 * ------------------------------------------------------------------------- */

/* Forward.  cache_out may be NULL (no backward); else *cache_out receives a
   library-owned cache (device memory) to pass to ozaki2_dgemm_bwd. */
OZ2_API int ozaki2_dgemm_fwd(int64_t M, int64_t N, int64_t K, const double* A, int64_t lda,
                     const double* B, int64_t ldb, double* C, int64_t ldc,
                     const ozaki2_opts* opts, ozaki2_cache* cache_out, void* stream);

/* Backward: dA = dC B^T (M x K) and dB = A^T dC (K x N); either output may be
   NULL.  dC is M x N. */
OZ2_API int ozaki2_dgemm_bwd(ozaki2_cache cache, const double* dC, int64_t lddc, double* dA,
                     int64_t ldda, double* dB, int64_t lddb, void* stream);

OZ2_API int ozaki2_cache_destroy(ozaki2_cache cache);

/* ---------------------------------------------------------------------------
 * Measurement aid (no counterpart in the paper): the throughput of the
 * warp-level INT8 tensor-core instruction mma.sync m16n8k32 (s8 x s8 -> s32),
 * the only INT8 tensor path sm_103a exposes (tcgen05.mma kind::i8 is not
 * available for this target).  It states the INT8 peak against which the
 * plane GEMMs' exact-integer rate is reported.
 * ------------------------------------------------------------------------- */

/* Launch `blocks` blocks of 8 warps, each warp issuing 8 x iters independent
   MMAs on register operands, time the launch with CUDA events on `stream`
   (after one warm-up launch) and store the rate in tera integer operations
   per second (2 per multiply-add) in *tops.  `sink` is a device int that is
   written only in a practically impossible case (it keeps the compiler from
   removing the MMAs).  Synchronises `stream`. */
OZ2_API int ozaki2_probe_mma_s8(int blocks, int iters, int* sink, double* tops, void* stream);

/* Library version string (static storage). */
OZ2_API const char* ozaki2_version(void);

#ifdef __cplusplus
}
#endif

#endif /* OZAKI2_H */
