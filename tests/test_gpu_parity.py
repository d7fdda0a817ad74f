"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Integer stages (shared exponents, residue planes, reduced products u_l, CRT
integers) must match bit for bit; final p-bit results must equal the oracle's
stage-by-stage result bit for bit and lie within 1 ulp of the correctly
rounded exact product (0 ulp where the exponent spread is within t - p).
"""
import random
from fractions import Fraction

import numpy as np
import pytest

import synth
from oracle import ozaki2_oracle as o
from ties_cases import final_rounding_ties, integerization_ties, mat_from_values

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)


@pytest.fixture(scope="module")
def ozk():
    from paper_2609_27831_gb300 import build
    build.build()
    import paper_2609_27831_gb300 as pkg
    return pkg


def crt_v(u, mods):
    """v_l = u_l M_l^{-1} mod m_l (M_l = P / m_l), the value the plane GEMM
    stores for the CRT (Sec. 4.4), from the oracle's reduced products u_l
    (leading axis l)."""
    P = 1
    for m in mods:
        P *= m
    inv = np.array([pow((P // m) % m, -1, m) for m in mods], dtype=np.int64)
    u = np.asarray(u, dtype=np.int64)
    shape = (-1,) + (1,) * (u.ndim - 1)
    return (u * inv.reshape(shape)) % np.array(mods, dtype=np.int64).reshape(shape)


def run_gpu(ozk, A, B, p, debug=True, **kw):
    """Execute one product; return output and every intermediate."""
    M, K = A["exp"].shape
    N = B["exp"].shape[1]
    plan = ozk.Plan((M, N, K, p), **kw)
    ws = plan.workspace()
    dA, dB = ozk.MPMatrix.from_host(A), ozk.MPMatrix.from_host(B)
    dC = ozk.MPMatrix.empty(M, N, p)
    D = plan.info["crt_digits"]
    chat = torch.zeros((M * N, D + 1), dtype=torch.int32, device="cuda") if debug else None
    if debug:
        plan.set_debug_chat(0, chat)
    plan.execute(dA, dB, dC, ws)
    plan.check()
    torch.cuda.synchronize()
    off, kp = plan.layout()
    G, L = plan.info["group_planes"], plan.info["L"]     # streamed: the last group's planes
    upitch = -(-(M * N) // 8) * 8
    w = ws.cpu().numpy()

    def region(o_, dtype, n):
        return w[o_: o_ + n * np.dtype(dtype).itemsize].view(dtype)

    out = {
        "plan": plan, "C": dC.to_host(),
        "e": region(off[0], np.int32, M), "f": region(off[1], np.int32, N),
        "pa": region(off[2], np.uint16, G * M * kp).reshape(G, M, kp)[:, :, :K],
        "pb": region(off[3], np.uint16, G * N * kp).reshape(G, N, kp)[:, :, :K],
        "u": region(off[4], np.uint16, L * upitch).reshape(L, upitch)[:, :M * N].reshape(L, M, N),
    }
    if debug:
        ch = chat.cpu().numpy().view(np.uint32)
        vals = []
        for r in ch:
            mag = 0
            for d in range(D):
                mag |= int(r[1 + d]) << (32 * d)
            vals.append(-mag if r[0] else mag)
        out["chat"] = np.array(vals, dtype=object).reshape(M, N)
    return out


def bf16_to_int(a):
    return (a.astype(np.uint32) << 16).view(np.float32).astype(np.int64)


def assert_full_parity(ozk, A, B, p, truth=True, **kw):
    got = run_gpu(ozk, A, B, p, **kw)
    ref = o.ozaki2_full(A, B, p)
    M, N = got["u"].shape[1:]
    e_ok = np.where(ref["e"] == 0, True, got["e"] == ref["e"])  # all-zero lines keep the sentinel
    assert e_ok.all()
    assert np.array_equal(bf16_to_int(got["pa"]), ref["planes_a"])
    assert np.array_equal(bf16_to_int(got["pb"]), ref["planes_b"])
    # the plane GEMM stores v_l = u_l M_l^{-1} mod m_l (the CRT's first step)
    assert np.array_equal(got["u"].astype(np.int64), crt_v(ref["u"], ref["par"].moduli))
    assert all(got["chat"][i, j] == ref["chat"][i, j] for i in range(M) for j in range(N))
    for key in ("limbs", "exp", "sign"):
        assert np.array_equal(got["C"][key], ref["C"][key]), key
    if truth:
        T = o.truth_full(A, B, p)
        worst = Fraction(0)
        for i in range(M):
            for j in range(N):
                g = o.to_fraction(*o.matrix_entry(got["C"], i, j))
                t = o.to_fraction(*o.matrix_entry(T, i, j))
                worst = max(worst, o.ulp_distance(g, t, p) if t else abs(g))
        assert worst <= 1
    return got, ref


def test_gemm_256_p53_all_stages(ozk):
    """The 256^3, p = 53 workload: every stage bit-exact, results 0 ulp."""
    A, B = synth.gemm_256_p53()
    got, ref = assert_full_parity(ozk, A, B, 53, truth=False)
    T = o.truth_full(A, B, 53)   # spread 16 <= t - p: quantisation is exact
    for key in ("limbs", "exp", "sign"):
        assert np.array_equal(got["C"][key], T[key])


def test_ragged_tiles_two_limb_moduli(ozk):
    """Ragged M, N, K (tile tails in every dimension) and two-limb moduli."""
    rng = np.random.Generator(np.random.PCG64(2001))
    A = synth.mp_matrix(rng, 150, 70, 256, -20, 20)
    B = synth.mp_matrix(rng, 70, 270, 256, -20, 20)
    assert_full_parity(ozk, A, B, 256)


def test_k_chunks_and_karatsuba_write_back(ozk):
    """k_chunk = 64 forces many exact accumulation chunks per plane, with the
    reduce-and-write-back step between chunks and between Karatsuba planes."""
    rng = np.random.Generator(np.random.PCG64(2002))
    A = synth.mp_matrix(rng, 130, 300, 200, -6, 6)
    B = synth.mp_matrix(rng, 300, 40, 200, -6, 6)
    assert_full_parity(ozk, A, B, 200, truth=False, k_chunk=64)


def test_engines_and_schedules_agree(ozk):
    rng = np.random.Generator(np.random.PCG64(2003))
    A = synth.mp_matrix(rng, 200, 96, 300, -10, 10)
    B = synth.mp_matrix(rng, 96, 300, 300, -10, 10)
    base = run_gpu(ozk, A, B, 300, debug=False)
    for kw in ({"engine": 1}, {"engine": 2}, {"schedule": 1}, {"grid": 7}, {"k_chunk": 128}, {"crt_engine": 1},
               {"res_engine": 1}):
        other = run_gpu(ozk, A, B, 300, debug=False, **kw)
        assert np.array_equal(other["u"], base["u"]), kw
        for key in ("limbs", "exp", "sign"):
            assert np.array_equal(other["C"][key], base["C"][key]), kw


def _adversarial_pair(K, p, need):
    """Seeded search for two values whose residues make some plane's per-chunk
    partial sum exceed `need` (all-equal rows and columns)."""
    par = o.Params(K, p)
    for seed in range(5000):
        rng = np.random.Generator(np.random.PCG64(2004 + seed))
        a1 = synth.mp_matrix(rng, 1, 1, p, 0, 0)
        b1 = synth.mp_matrix(rng, 1, 1, p, 0, 0)
        ai, _ = o.integer_line(a1, 0, 0, par.t)
        bj, _ = o.integer_line(b1, 0, 1, par.t)
        ra, rb = o.plane_values(ai[0], par.moduli), o.plane_values(bj[0], par.moduli)
        big = max(abs(x * y) for x, y in zip(ra, rb)) * min(K, 1024)
        if big > need:
            return a1, b1, big
    raise AssertionError("no adversarial pair found")


@pytest.mark.parametrize("K", [1024, 1040, 2048, 2100])
def test_fp32_accumulation_exactness_torture(ozk, K):
    """All-equal inputs make every plane product K r_a r_b; the values are
    chosen so that one plane's partial sum within a chunk exceeds 0.9 * 2^24
    (K = 1024), and chunk boundaries are crossed (K > 1024).  Every u_l must
    be exact."""
    p = 53
    a1, b1, big = _adversarial_pair(K, p, 0.9 * 2 ** 24)
    assert big < 2 ** 24
    A = {k: (np.broadcast_to(v, v.shape[:-2] + (64, K)).copy() if isinstance(v, np.ndarray) else v)
         for k, v in a1.items()}
    B = {k: (np.broadcast_to(v, v.shape[:-2] + (K, 64)).copy() if isinstance(v, np.ndarray) else v)
         for k, v in b1.items()}
    got = run_gpu(ozk, A, B, p)
    par = o.Params(K, p)
    ai, e = o.integer_line(A, 0, 0, par.t)
    bj, f = o.integer_line(B, 0, 1, par.t)
    ref = o.entry(ai, e, bj, f, par)
    v = crt_v(ref["u"], par.moduli)
    assert np.all(got["u"].astype(np.int64) == v[:, None, None])
    assert all(got["chat"][i, j] == ref["chat"] for i in (0, 63) for j in (0, 63))
    assert o.matrix_entry(got["C"], 5, 7) == (ref["limbs"], ref["exp"], ref["sign"])


def test_zero_lines_and_tiny_shapes(ozk):
    rng = np.random.Generator(np.random.PCG64(2005))
    A = synth.zero_rows(synth.mp_matrix(rng, 33, 17, 113, -5, 5), [0, 5])
    B = synth.zero_cols(synth.mp_matrix(rng, 17, 9, 113, -5, 5), [3])
    got, _ = assert_full_parity(ozk, A, B, 113)
    assert not got["C"]["limbs"][:, 0, :].any() and not got["C"]["limbs"][:, :, 3].any()
    for (M, N, K, p) in [(1, 1, 1, 53), (1, 5, 1, 2), (3, 1, 2, 64), (2, 2, 3, 8)]:
        A = synth.mp_matrix(rng, M, K, p, -3, 3)
        B = synth.mp_matrix(rng, K, N, p, -3, 3)
        assert_full_parity(ozk, A, B, p)


def test_p2048_small(ozk):
    """p = 2048 (the largest precision): 32-limb inputs, two-limb moduli; the
    residues and the CRT both on the tensor cores (the defaults at this length)
    and on the CUDA cores (132-digit residue class, 32-lane CRT groups); every
    stage bit-exact."""
    rng = np.random.Generator(np.random.PCG64(2030))
    A = synth.mp_matrix(rng, 20, 24, 2048, -64, 64)
    B = synth.mp_matrix(rng, 24, 18, 2048, -64, 64)
    got, _ = assert_full_parity(ozk, A, B, 2048, truth=False)
    assert got["plan"].info["crt_mode"] == 2 and got["plan"].info["res_mode"] == 2
    got3, _ = assert_full_parity(ozk, A, B, 2048, truth=False, crt_engine=3, res_engine=3)
    assert got3["plan"].info["crt_mode"] == 0 and got3["plan"].info["res_mode"] == 0


# Cancelling, exactly zero and ordinary small-integer outputs for the finish
# of long accumulators (|c_hat| far below its usual size in some).
CANCEL_ROWS_A = [
    [(1, 0), (1, 0), (1, -1000), (0, 0)],
    [(3, 5), (-3, 5), (5, -3000), (1, -3100)],
    [(1, 0), (1, 0), (0, 0), (0, 0)],
    [(5, 2), (7, 1), (-9, -40), (11, -3)],
]
CANCEL_ROWS_B = [
    [(1, 0), (7, 10), (1, 0)],
    [(-1, 0), (7, 10), (-1, 0)],
    [(1, 0), (1, -5), (1, -2000)],
    [(1, 0), (3, 1), (0, 0)],
]


@pytest.mark.parametrize("p", [1024, 2048])
def test_long_finish_small_and_zero_results(ozk, p):
    """The finish of long accumulators keeps only the highest digits of |c_hat|
    in shared memory and moves that window down when a word below it is
    needed: outputs whose large terms cancel (|c_hat| far below its usual
    size), an exact zero, and ordinary ones, every stage bit-exact."""
    A = mat_from_values(CANCEL_ROWS_A * 8, p)                   # 32 x 4: at least one 128-output tile
    B = mat_from_values([r * 2 for r in CANCEL_ROWS_B], p)      # 4 x 6
    got, ref = assert_full_parity(ozk, A, B, p, truth=False, crt_engine=2)
    assert got["plan"].info["crt_mode"] == 2 and got["plan"].info["crt_digits"] > 24
    assert ref["chat"][2, 0] == 0 and ref["chat"][0, 0] != 0
    assert abs(ref["chat"][0, 0]).bit_length() < abs(ref["chat"][0, 1]).bit_length() - 64


@pytest.mark.parametrize("p,shape", [(1024, (40, 36, 30)), (2048, (24, 22, 20))])
def test_long_finish_top_groups_form(ozk, p, shape):
    """Without the debug dump of c_hat the finish of long accumulators first
    tries its fast form: both passes over the group words from the group
    below the window on, with the carry left out of that group's lowest digit
    (at most alpha + 2) bounded; an output falls back to the full form where
    a digit the fast form uses lies near a wrap, no digit between that one and
    the window is nonzero, or the rounding needs a word below the window.
    Random outputs (the fast form) and cancelling or small-integer ones (the
    full form) equal the oracle bit for bit, and equal the outputs of the
    full form (debug dump on) for the random product."""
    M, N, K = shape
    rng = np.random.Generator(np.random.PCG64(2044 + p))
    A = synth.mp_matrix(rng, M, K, p, -64, 64)
    B = synth.mp_matrix(rng, K, N, p, -64, 64)
    fast = run_gpu(ozk, A, B, p, debug=False, crt_engine=2)
    assert fast["plan"].info["crt_mode"] == 2 and fast["plan"].info["crt_digits"] > 2 * (p // 64) + 4 + 7
    full = run_gpu(ozk, A, B, p, debug=True, crt_engine=2)
    ref = o.ozaki2_full(A, B, p)
    for key in ("limbs", "exp", "sign"):
        assert np.array_equal(fast["C"][key], ref["C"][key]), key
        assert np.array_equal(full["C"][key], fast["C"][key]), key
    A2 = mat_from_values(CANCEL_ROWS_A * 8, p)
    B2 = mat_from_values([r * 2 for r in CANCEL_ROWS_B], p)
    got2 = run_gpu(ozk, A2, B2, p, debug=False, crt_engine=2)
    ref2 = o.ozaki2_full(A2, B2, p)
    for key in ("limbs", "exp", "sign"):
        assert np.array_equal(got2["C"][key], ref2["C"][key]), key


@pytest.mark.parametrize("p", [300, 700])
def test_crt_engines_bit_exact(ozk, p):
    """The CRT engines (automatic: the tensor-core sums above 20 digits, CUDA
    cores only, tensor-core column sums in one kernel) give the same CRT
    integers and outputs, and all match the oracle."""
    rng = np.random.Generator(np.random.PCG64(2010 + p))
    A = synth.mp_matrix(rng, 140, 60, p, -30, 30)
    B = synth.mp_matrix(rng, 60, 20, p, -30, 30)
    got_auto, ref = assert_full_parity(ozk, A, B, p, truth=False)
    for eng in (1, 3):
        got = run_gpu(ozk, A, B, p, crt_engine=eng)
        assert all(got["chat"][i, j] == ref["chat"][i, j] for i in range(140) for j in range(20))
        for key in ("limbs", "exp", "sign"):
            assert np.array_equal(got["C"][key], got_auto["C"][key])


@pytest.mark.parametrize("shape", [(140, 20, 60, 300), (70, 45, 50, 700), (40, 36, 30, 1024),
                                   (20, 18, 24, 2048), (9, 15, 7, 130)])
def test_crt_sum_engine_stages(ozk, shape):
    """CRT sums on the tensor cores (crt_engine 2) and their finish from the
    group sums, accumulators of 12 to 133 digits, one to five chunks, ragged
    last tiles; every stage bit-exact against the oracle."""
    M, N, K, p = shape
    rng = np.random.Generator(np.random.PCG64(2040 + p))
    A = synth.mp_matrix(rng, M, K, p, -30, 30)
    B = synth.mp_matrix(rng, K, N, p, -30, 30)
    assert_full_parity(ozk, A, B, p, truth=False, crt_engine=2)


def test_crt_sum_engine_many_tiles(ozk):
    """More 128-output tiles than CTAs (V rebuilt, TMEM slots and rings
    cycling): identical to the CUDA-core CRT, and sampled entries against the
    oracle."""
    M, N, K, p = 256, 160, 16, 1024
    rng = np.random.Generator(np.random.PCG64(2045))
    A = synth.mp_matrix(rng, M, K, p, -20, 20)
    B = synth.mp_matrix(rng, K, N, p, -20, 20)
    g2 = run_gpu(ozk, A, B, p, debug=False, crt_engine=2)
    g0 = run_gpu(ozk, A, B, p, debug=False)
    for key in ("limbs", "exp", "sign"):
        assert np.array_equal(g2["C"][key], g0["C"][key])
    rnd = random.Random(11)
    pairs = [(0, 0), (M - 1, N - 1)] + [(rnd.randrange(M), rnd.randrange(N)) for _ in range(6)]
    for (i, j), r in zip(pairs, o.ozaki2_entries(A, B, p, pairs)):
        assert o.matrix_entry(g2["C"], i, j) == (r["limbs"], r["exp"], r["sign"])


def test_crt_sum_engine_one_chunk_many_tiles(ozk):
    """One 128-column chunk per tile (p = 256) and many tiles per CTA: the half
    without a chunk in a tile must still wait for that tile's MMAs before it
    rewrites V.  Identical to the CUDA-core CRT."""
    M, N, K, p = 512, 448, 8, 256
    rng = np.random.Generator(np.random.PCG64(2047))
    A = synth.mp_matrix(rng, M, K, p, -20, 20)
    B = synth.mp_matrix(rng, K, N, p, -20, 20)
    g2 = run_gpu(ozk, A, B, p, debug=False, crt_engine=2)
    g0 = run_gpu(ozk, A, B, p, debug=False)
    for key in ("limbs", "exp", "sign"):
        assert np.array_equal(g2["C"][key], g0["C"][key])


@pytest.mark.parametrize("res_engine", [0, 2])
def test_crt_sum_engine_batched(ozk, res_engine):
    """A batch whose problems have different modulus counts and digit lengths
    through the tensor-core sums: four TMEM layouts of the CRT sums (one
    launch each; tables switch between tiles of one CTA within a layout), and
    with res_engine 2 four layouts of the tensor-core residues as well (two and
    four byte buffers)."""
    rng = np.random.Generator(np.random.PCG64(2046))
    shapes = [(70, 40, 30, 256), (33, 60, 17, 1024), (40, 30, 50, 512), (5, 5, 5, 53)]
    mats = [(synth.mp_matrix(rng, M, K, p, -8, 8), synth.mp_matrix(rng, K, N, p, -8, 8))
            for (M, N, K, p) in shapes]
    plan = ozk.Plan(shapes, crt_engine=2, res_engine=res_engine)
    ws = plan.workspace()
    trip = [(ozk.MPMatrix.from_host(A), ozk.MPMatrix.from_host(B), ozk.MPMatrix.empty(M, N, p))
            for (M, N, K, p), (A, B) in zip(shapes, mats)]
    plan.execute_batched(trip, ws)
    plan.check()
    for (M, N, K, p), (A, B), (_, _, Cd) in zip(shapes, mats, trip):
        ref = o.ozaki2_full(A, B, p)["C"]
        for key in ("limbs", "exp", "sign"):
            assert np.array_equal(Cd.to_host()[key], ref[key])


@pytest.mark.parametrize("engine", [1, 2])
@pytest.mark.parametrize("shape", [(130, 70, 45, 256), (33, 9, 100, 53), (64, 129, 17, 500), (5, 3, 1, 2)])
def test_residue_engines_bit_exact(ozk, shape, engine):
    """Residues on the tensor cores (byte GEMM, opt-in; one kernel or
    warp-specialised) give the oracle's planes bit for bit on both sides, with
    ragged tiles, zero lines and two-limb moduli."""
    M, N, K, p = shape
    rng = np.random.Generator(np.random.PCG64(2020 + M))
    A = synth.zero_rows(synth.mp_matrix(rng, M, K, p, -40, 40), [1])
    B = synth.zero_cols(synth.mp_matrix(rng, K, N, p, -40, 40), [0])
    assert_full_parity(ozk, A, B, p, truth=False, res_engine=engine)


@pytest.mark.parametrize("shape", [(20, 18, 70, 2048), (40, 36, 130, 1024), (300, 260, 600, 113)])
def test_residue_mm_engine_chunks_and_tiles(ozk, shape):
    """The warp-specialised tensor-core residues with several column chunks
    (p = 1024, 2048), 512 TMEM columns, and more tiles than CTAs (p = 113):
    planes bit for bit against the CUDA-core kernel and the oracle."""
    M, N, K, p = shape
    rng = np.random.Generator(np.random.PCG64(2050 + p))
    A = synth.zero_rows(synth.mp_matrix(rng, M, K, p, -50, 50), [2])
    B = synth.zero_cols(synth.mp_matrix(rng, K, N, p, -50, 50), [1])
    if M * N * K <= 600_000:
        assert_full_parity(ozk, A, B, p, truth=False, res_engine=2)
    else:
        g2 = run_gpu(ozk, A, B, p, debug=False, res_engine=2)
        g0 = run_gpu(ozk, A, B, p, debug=False)
        assert np.array_equal(g2["pa"], g0["pa"]) and np.array_equal(g2["pb"], g0["pb"])
        for key in ("limbs", "exp", "sign"):
            assert np.array_equal(g2["C"][key], g0["C"][key])


def test_cancellation_to_zero(ozk):
    """x * y + (-x) * y = 0 exactly: the CRT integer is 0 and the output zero."""
    rng = np.random.Generator(np.random.PCG64(2006))
    A = synth.mp_matrix(rng, 4, 2, 128, -5, 5)
    A["limbs"][:, :, 1] = A["limbs"][:, :, 0]
    A["exp"][:, 1] = A["exp"][:, 0]
    A["sign"][:, 1] = 1 - A["sign"][:, 0]
    B = synth.mp_matrix(rng, 2, 3, 128, -5, 5)
    B["limbs"][:, 1, :] = B["limbs"][:, 0, :]
    B["exp"][1, :] = B["exp"][0, :]
    B["sign"][1, :] = B["sign"][0, :]
    got, _ = assert_full_parity(ozk, A, B, 128)
    assert not got["C"]["limbs"].any() and not got["C"]["exp"].any()


def test_gemm_1024_p256_sampled(ozk):
    """The 1024^3, p = 256 workload in the launch configuration the benchmark
    times: sampled outputs against the oracle entry by entry (every stage) and
    against the exact product (<= 1 ulp)."""
    A, B = synth.gemm_1024_p256()
    got = run_gpu(ozk, A, B, 256)
    rnd = random.Random(7)
    pairs = [(0, 0), (1023, 1023), (0, 1023), (1023, 0), (511, 257)]
    pairs += [(rnd.randrange(1024), rnd.randrange(1024)) for _ in range(11)]
    ref = o.ozaki2_entries(A, B, 256, pairs)
    mods = o.Params(1024, 256).moduli
    worst = Fraction(0)
    for (i, j), r in zip(pairs, ref):
        assert [int(x) for x in got["u"][:, i, j]] == crt_v(r["u"], mods).tolist()
        assert got["chat"][i, j] == r["chat"]
        assert o.matrix_entry(got["C"], i, j) == (r["limbs"], r["exp"], r["sign"])
        t = o.to_fraction(*o.truth_entry(A, B, i, j, 256))
        worst = max(worst, o.ulp_distance(o.to_fraction(r["limbs"], r["exp"], r["sign"]), t, 256))
    assert worst <= 1
    print(f"max ulp 1024x1024x1024 p=256: {float(worst):.4f} over {len(pairs)} sampled entries")
    # the integer planes of a 256 x 256 corner, in full
    par = o.Params(1024, 256)
    for i in (0, 100, 1023):
        row, _ = o.integer_line(A, i, 0, par.t)
        assert np.array_equal(bf16_to_int(got["pa"][:, i, :]).T,
                              np.array([o.plane_values(x, par.moduli) for x in row]))


def test_batched_and_graph(ozk):
    rng = np.random.Generator(np.random.PCG64(2007))
    # p = 1024 needs more CRT digits than the tensor-core CRT takes: both CRT
    # paths run in one batch
    shapes = [(70, 300, 90, 113), (129, 40, 200, 256), (33, 260, 17, 512), (5, 5, 5, 53),
              (40, 30, 50, 1024)]
    mats = []
    for (M, N, K, p) in shapes:
        mats.append((synth.mp_matrix(rng, M, K, p, -8, 8), synth.mp_matrix(rng, K, N, p, -8, 8)))
    plan = ozk.Plan(shapes)
    ws = plan.workspace()
    trip = []
    for (M, N, K, p), (A, B) in zip(shapes, mats):
        trip.append((ozk.MPMatrix.from_host(A), ozk.MPMatrix.from_host(B), ozk.MPMatrix.empty(M, N, p)))
    plan.execute_batched(trip, ws)
    plan.check()
    for (M, N, K, p), (A, B), (_, _, Cd) in zip(shapes, mats, trip):
        ref = o.ozaki2_full(A, B, p)["C"]
        for key in ("limbs", "exp", "sign"):
            assert np.array_equal(Cd.to_host()[key], ref[key])
    # the same problems through a captured CUDA graph
    s = torch.cuda.Stream()
    for _, _, Cd in trip:
        Cd.limbs.zero_()
    with torch.cuda.stream(s):
        g = plan.graph(trip, ws, s)
        g.launch(s)
        g.launch(s)
    s.synchronize()
    for (M, N, K, p), (A, B), (_, _, Cd) in zip(shapes, mats, trip):
        ref = o.ozaki2_full(A, B, p)["C"]
        assert np.array_equal(Cd.to_host()["limbs"], ref["limbs"])


def test_launch_count(ozk):
    """The library reports its kernel launches per execute: scan, residues,
    plane GEMM and CRT for a short accumulator; the CRT sums and the long
    finish replace the one-lane CRT above 40 digits."""
    rng = np.random.Generator(np.random.PCG64(2060))
    for p, n in ((256, 4), (2048, 5)):
        A = synth.mp_matrix(rng, 40, 30, p, -5, 5)
        B = synth.mp_matrix(rng, 30, 50, p, -5, 5)
        got = run_gpu(ozk, A, B, p, debug=False)
        assert got["plan"].launches() == n


def test_convenience_gemm_call(ozk):
    rng = np.random.Generator(np.random.PCG64(2008))
    A = synth.mp_matrix(rng, 40, 50, 160, -4, 4)
    B = synth.mp_matrix(rng, 50, 30, 160, -4, 4)
    Cd = ozk.gemm(ozk.MPMatrix.from_host(A), ozk.MPMatrix.from_host(B), 160)
    torch.cuda.synchronize()
    ref = o.ozaki2_full(A, B, 160)["C"]
    assert np.array_equal(Cd.to_host()["limbs"], ref["limbs"])


def _groups(moduli, req):
    """Planes per modulus group: as few groups of consecutive moduli with at
    most req planes each (one per one-limb modulus, three per two-limb) as
    the plane counts allow, of about equal size (the smallest cap from the
    even split up that reaches that count); a group with two-limb moduli
    holds an even number of one-limb ones."""
    planes = [1 if m <= 255 else 3 for m in moduli]
    G = sum(planes)
    ng = -(-G // req)

    def split(cap):
        out, cur, ones = [], 0, 0
        for pl_ in planes:
            if cur and (cur + pl_ > cap or (pl_ == 3 and ones % 2)):
                out.append(cur)
                cur, ones = 0, 0
            cur += pl_
            ones += pl_ == 1
        out.append(cur)
        return out

    for cap in range(-(-G // ng), req + 1):
        out = split(cap)
        if len(out) <= ng:
            break
    return out


@pytest.mark.parametrize("p,shape,req,kw", [
    (256, (150, 130, 200), 20, {}),                 # CUDA-core residues, groups across the one/two-limb border
    (256, (150, 130, 200), 7, {"res_engine": 2}),   # tensor-core residues, small groups
    (1024, (70, 60, 90), 40, {}),                   # tensor-core residues (automatic), an odd one-limb border
    (1024, (70, 60, 90), 40, {"res_engine": 3}),    # the same groups on the CUDA cores
    (113, (40, 300, 70), 3, {"crt_engine": 3}),     # one or three planes per group
])
def test_planes_streamed_in_modulus_groups(ozk, p, shape, req, kw):
    """Planes streamed through the workspace group by group give the same
    reduced products, CRT integers and outputs as the oracle (and as one
    group); the plane region holds the last group's planes."""
    M, N, K = shape
    rng = np.random.Generator(np.random.PCG64(5200 + p + req))
    A = synth.mp_matrix(rng, M, K, p, -8, 8)
    B = synth.mp_matrix(rng, K, N, p, -8, 8)
    got = run_gpu(ozk, A, B, p, plane_group=req, **kw)
    info = got["plan"].info
    ref = o.ozaki2_full(A, B, p)
    sizes = _groups(ref["par"].moduli, req)
    assert info["plane_groups"] == len(sizes) > 1 and info["group_planes"] == max(sizes)
    last = sizes[-1]
    assert np.array_equal(bf16_to_int(got["pa"][:last]), ref["planes_a"][-last:])
    assert np.array_equal(bf16_to_int(got["pb"][:last]), ref["planes_b"][-last:])
    assert np.array_equal(got["u"].astype(np.int64), crt_v(ref["u"], ref["par"].moduli))
    assert all(got["chat"][i, j] == ref["chat"][i, j] for i in range(M) for j in range(N))
    for key in ("limbs", "exp", "sign"):
        assert np.array_equal(got["C"][key], ref["C"][key]), key
    whole = run_gpu(ozk, A, B, p, debug=False, plane_group=-1, **kw)
    assert whole["plan"].info["plane_groups"] == 1
    for key in ("limbs", "exp", "sign"):
        assert np.array_equal(got["C"][key], whole["C"][key]), key
    # timings: residues and GEMMs summed over the groups
    plan = ozk.Plan((M, N, K, p), plane_group=req, timing=1, **kw)
    ws = plan.workspace()
    dC = ozk.MPMatrix.empty(M, N, p)
    plan.execute(ozk.MPMatrix.from_host(A), ozk.MPMatrix.from_host(B), dC, ws)
    tm = plan.timings()
    assert all(tm[k] > 0 for k in ("scan", "residues", "gemm", "crt"))
    assert tm["scan"] + tm["residues"] + tm["gemm"] + tm["crt"] <= tm["total"] * 1.001 + 1e-3
    assert plan.launches() >= 1 + len(sizes) * 2


@pytest.mark.parametrize("shape,p,kw", [
    ((40, 30, 50), 53, {}),                           # one pair tile, the peer's rows all outside M
    ((130, 260, 70), 113, {}),                        # ragged rows inside the peer, two column tiles
    ((300, 520, 200), 256, {"k_chunk": 128}),         # K chunks with write-back, two-limb moduli
    ((257, 129, 1100), 53, {}),                       # K above one 1024 chunk, rows one past a pair tile
])
def test_pair_tiles_bit_exact(ozk, shape, p, kw):
    """The CTA-pair plane GEMM (256 x 256 tiles, tcgen05 cta_group::2) gives the
    oracle's planes products bit for bit: every v_l, CRT integer and output."""
    M, N, K = shape
    rng = np.random.Generator(np.random.PCG64(7100 + M + p))
    A = synth.mp_matrix(rng, M, K, p, -8, 8)
    B = synth.mp_matrix(rng, K, N, p, -8, 8)
    got, _ = assert_full_parity(ozk, A, B, p, truth=False, gemm_tile=2, **kw)
    assert got["plan"].info["gemm_tile"] == 2


def test_pair_tiles_streamed_and_batched(ozk):
    """Pair tiles through modulus groups and in a batched plan agree with the
    one-SM tiles bit for bit."""
    rng = np.random.Generator(np.random.PCG64(7200))
    A = synth.mp_matrix(rng, 180, 200, 256, -8, 8)
    B = synth.mp_matrix(rng, 200, 300, 256, -8, 8)
    one = run_gpu(ozk, A, B, 256, debug=False, gemm_tile=1)
    two = run_gpu(ozk, A, B, 256, debug=False, gemm_tile=2, plane_group=20)
    assert two["plan"].info["plane_groups"] > 1
    assert np.array_equal(one["u"], two["u"])
    for key in ("limbs", "exp", "sign"):
        assert np.array_equal(one["C"][key], two["C"][key]), key
    shapes = [(70, 300, 90, 113), (260, 40, 64, 256), (33, 33, 33, 53)]
    trip, ins = [], []
    for (M, N, K, p) in shapes:
        a = synth.mp_matrix(rng, M, K, p, -8, 8)
        b = synth.mp_matrix(rng, K, N, p, -8, 8)
        ins.append((a, b, p))
        trip.append((ozk.MPMatrix.from_host(a), ozk.MPMatrix.from_host(b), ozk.MPMatrix.empty(M, N, p)))
    for sched in (0, 1):                               # grouped, and one launch per modulus
        plan = ozk.Plan(shapes, gemm_tile=2, schedule=sched)
        plan.execute_batched(trip, plan.workspace())
        plan.check()
        torch.cuda.synchronize()
        for (a, b, p), (_, _, c) in zip(ins, trip):
            ref = o.ozaki2_full(a, b, p)["C"]
            h = c.to_host()
            for key in ("limbs", "exp", "sign"):
                assert np.array_equal(h[key], ref[key]), key


@pytest.mark.parametrize("p,shape,kw", [(113, (90, 70, 130), {}), (256, (64, 300, 200), {"res_engine": 2}),
                                        (1024, (40, 50, 60), {})])
def test_operand_reuse(ozk, p, shape, kw):
    """ozaki2_execute_reuse: a second right-hand side with A's planes kept, and
    a second left-hand side with B's planes kept, each bit-identical to the
    oracle; a workspace that did not run the previous product is refused."""
    M, N, K = shape
    rng = np.random.Generator(np.random.PCG64(7300 + p))
    A = synth.mp_matrix(rng, M, K, p, -8, 8)
    B1 = synth.mp_matrix(rng, K, N, p, -8, 8)
    B2 = synth.mp_matrix(rng, K, N, p, -20, 3)
    A2 = synth.mp_matrix(rng, M, K, p, -2, 9)
    plan = ozk.Plan((M, N, K, p), **kw)
    ws = plan.workspace()
    dA, dB1 = ozk.MPMatrix.from_host(A), ozk.MPMatrix.from_host(B1)
    C1 = ozk.MPMatrix.empty(M, N, p)
    plan.execute(dA, dB1, C1, ws)
    C2 = ozk.MPMatrix.empty(M, N, p)
    plan.execute_reuse(0, ozk.MPMatrix.from_host(B2), C2, ws)      # A kept
    C3 = ozk.MPMatrix.empty(M, N, p)
    plan.execute_reuse(1, ozk.MPMatrix.from_host(A2), C3, ws)      # B2 kept
    plan.check()
    torch.cuda.synchronize()
    for got, (x, y) in ((C1, (A, B1)), (C2, (A, B2)), (C3, (A2, B2))):
        ref = o.ozaki2_full(x, y, p)["C"]
        h = got.to_host()
        for key in ("limbs", "exp", "sign"):
            assert np.array_equal(h[key], ref[key]), key
    with pytest.raises(ozk.OzakiError):
        plan.execute_reuse(0, ozk.MPMatrix.from_host(B2), C2, plan.workspace())
    streamed = ozk.Plan((M, N, K, p), plane_group=3, **kw)
    if streamed.info["plane_groups"] > 1:
        w2 = streamed.workspace()
        streamed.execute(dA, dB1, C1, w2)
        with pytest.raises(ozk.OzakiError):
            streamed.execute_reuse(0, ozk.MPMatrix.from_host(B2), C2, w2)


@pytest.mark.parametrize("p", [53, 113, 256])
@pytest.mark.parametrize("res_engine", [2, 3])
def test_integerization_ties(ozk, p, res_engine):
    """Entries whose integerization drops exactly half a step (even and odd
    kept bits, both signs) or just off it: planes, CRT integers and outputs
    bit-exact against the oracle (whose rounding is pinned to round(Fraction))
    on both residue engines."""
    K = 3
    rows, t, d = integerization_ties(p, K)
    A = mat_from_values(rows, p)
    rng = np.random.Generator(np.random.PCG64(7400 + p))
    B = synth.mp_matrix(rng, K, 5, p, -3, 3)
    got, ref = assert_full_parity(ozk, A, B, p, truth=False, res_engine=res_engine)
    assert got["plan"].info["t"] == t


@pytest.mark.parametrize("p", [53, 256])
def test_final_rounding_ties(ozk, p):
    """Products whose exact value is a tie at p bits (or just off one, or
    carries into a new bit): outputs equal to the values fixed by hand."""
    cases = final_rounding_ties(p)
    A = mat_from_values([c[0] for c in cases], p)
    B = mat_from_values([[(1, 0)] for _ in range(3)], p)
    got, _ = assert_full_parity(ozk, A, B, p)
    for i, (_, want) in enumerate(cases):
        assert o.to_fraction(*o.matrix_entry(got["C"], i, 0)) == Fraction(want, 1 << 10), i


@pytest.mark.parametrize("shape,p,kw", [
    ((100, 130, 200), 53, {}),                                  # one-limb planes only
    ((90, 300, 257), 256, {"gemm_tile": 1}),                    # two-limb Karatsuba planes, one-SM tiles
    ((300, 90, 128), 256, {"gemm_tile": 2}),                    # CTA-pair tiles
    ((150, 120, 100), 256, {"plane_group": 20}),                # planes streamed in groups
])
def test_plane_sums_before_reduction(ozk, shape, p, kw):
    """The exact integer GEMM output of every plane, C_g = sum_k r_a r_b
    before any reduction (dumped by the tensor-core epilogue), equals the
    oracle's plane products bit for bit."""
    M, N, K = shape
    rng = np.random.Generator(np.random.PCG64(7500 + M + p))
    A = synth.mp_matrix(rng, M, K, p, -8, 8)
    B = synth.mp_matrix(rng, K, N, p, -8, 8)
    plan = ozk.Plan((M, N, K, p), **kw)
    G = plan.info["G"]
    buf = torch.full((G, M, N), -7, dtype=torch.int32, device="cuda")
    plan.set_debug_prods(0, buf)
    dC = ozk.MPMatrix.empty(M, N, p)
    plan.execute(ozk.MPMatrix.from_host(A), ozk.MPMatrix.from_host(B), dC, plan.workspace())
    plan.check()
    torch.cuda.synchronize()
    ref = o.ozaki2_full(A, B, p)
    assert np.array_equal(buf.cpu().numpy().astype(np.int64), ref["prods"])
    h = dC.to_host()
    for key in ("limbs", "exp", "sign"):
        assert np.array_equal(h[key], ref["C"][key]), key


def test_plane_sums_need_one_chunk(ozk):
    plan = ozk.Plan((64, 64, 2000, 113))             # K above one 1024 chunk
    buf = torch.zeros(1, dtype=torch.int32, device="cuda")
    with pytest.raises(ozk.OzakiError):
        plan.set_debug_prods(0, buf)


@pytest.mark.parametrize("shape,p", [((130, 300, 77), 256),      # two-limb moduli, ragged tiles, K tail
                                     ((40, 20, 2100), 53),       # K above one accumulation chunk
                                     ((257, 129, 33), 113)])     # a column tile with one 128-half
def test_int8_mma_engine_bit_exact(ozk, shape, p):
    """The second plane GEMM engine (INT8 x INT8 -> INT32 on mma.sync) gives
    the oracle's v_l, CRT integers and outputs bit for bit."""
    M, N, K = shape
    rng = np.random.Generator(np.random.PCG64(7600 + M + p))
    A = synth.mp_matrix(rng, M, K, p, -8, 8)
    B = synth.mp_matrix(rng, K, N, p, -8, 8)
    assert_full_parity(ozk, A, B, p, truth=False, engine=2)
