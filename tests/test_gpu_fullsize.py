"""Parity at the workloads' full sizes, on sampled outputs.

The oracle cannot compute these products whole, so each test runs the full
product on the GPU and checks sampled entries stage by stage against the
oracle (the reduced products of every modulus, times M_l^{-1} mod m_l as the
plane GEMM stores them, the output limbs, exponent and sign bit for bit) and against the exact product rounded once (<= 1 ulp):
  4096^3 at p = 2048 (exponents in [-64, 64]; planes streamed in two groups
  of moduli; the CRT as tensor-core sums), 16 entries,
  8192^3 at p = 53 (exponents in [-8, 8]), 16 entries, both with the
  benchmark's inputs,
  the 64-problem batch (M, N, K log-uniform in [128, 2048], p in {113, 256, 512}),
  2 entries in each of 8 problems,
  the binary64 forward and backward at 4096^2, 16 entries of each of C, dA, dB.
"""
from fractions import Fraction

import numpy as np
import pytest

import synth
from oracle import ozaki2_oracle as o

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


def _oracle_entries(A, B, p, pairs):
    """ozaki2_entries at the sampled pairs, one spawn-pool process per entry
    (each task receives only its row of A and column of B)."""
    import multiprocessing as mp
    import os
    tasks = []
    for i, j in pairs:
        a = {"p": A["p"], "limbs": A["limbs"][:, i:i + 1, :].copy(), "exp": A["exp"][i:i + 1, :].copy(),
             "sign": A["sign"][i:i + 1, :].copy()}
        b = {"p": B["p"], "limbs": B["limbs"][:, :, j:j + 1].copy(), "exp": B["exp"][:, j:j + 1].copy(),
             "sign": B["sign"][:, j:j + 1].copy()}
        tasks.append((a, b, p, [(0, 0)]))
    with mp.get_context("spawn").Pool(min(len(tasks), os.cpu_count() or 1)) as pool:
        return [r[0] for r in pool.starmap(o.ozaki2_entries, tasks, chunksize=1)]


def _pairs(M, N, n, seed):
    """n sampled entries: the four corners, then seeded random ones."""
    rnd = np.random.Generator(np.random.PCG64(seed))
    out = [(0, 0), (M - 1, N - 1), (0, N - 1), (M - 1, 0)]
    while len(out) < n:
        out.append((int(rnd.integers(M)), int(rnd.integers(N))))
    return out[:n]


def _sampled(ozk, plan, ws, dC, M, N, K, p, pairs, A, B, off=None):
    """Compare sampled entries of an executed product with the oracle."""
    off = off if off is not None else plan.layout()[0][4]
    L = plan.info["L"]
    upitch = -(-(M * N) // 8) * 8
    u16 = ws[off: off + 2 * L * upitch].view(torch.int16)
    ref = _oracle_entries(A, B, p, pairs)
    par = o.Params(K, p)
    P = 1
    for m in par.moduli:
        P *= m
    worst = Fraction(0)
    for (i, j), r in zip(pairs, ref):
        got_u = (u16[torch.arange(L, device=u16.device) * upitch + i * N + j].cpu().numpy().astype(np.int64)
                 & 0xFFFF)
        # the plane GEMM stores v_l = u_l M_l^{-1} mod m_l (the CRT's first step)
        want = np.array([(x * pow((P // m) % m, -1, m)) % m for x, m in zip(r["u"], par.moduli)])
        assert np.array_equal(got_u, want), (i, j)
        limbs = [int(x) & ((1 << 64) - 1) for x in dC.limbs[:, i, j].cpu().tolist()]
        got = (limbs, int(dC.exp[i, j].item()), int(dC.sign[i, j].item()))
        assert got == (r["limbs"], r["exp"], r["sign"]), (i, j)
        t = o.to_fraction(*o.truth_entry(A, B, i, j, p))
        u = o.ulp_distance(o.to_fraction(*got), t, p)
        assert u <= 1, (i, j)
        worst = max(worst, u)
    print(f"max ulp {M}x{N}x{K} p={p}: {float(worst):.4f} over {len(pairs)} sampled entries")


def _single(ozk, A, B, p, pairs):
    M, K = A["exp"].shape
    N = B["exp"].shape[1]
    plan = ozk.Plan((M, N, K, p))
    ws = plan.workspace()
    dA, dB = ozk.MPMatrix.from_host(A), ozk.MPMatrix.from_host(B)
    dC = ozk.MPMatrix.empty(M, N, p)
    plan.execute(dA, dB, dC, ws)
    plan.check()
    torch.cuda.synchronize()
    _sampled(ozk, plan, ws, dC, M, N, K, p, pairs, A, B)
    return plan


def test_gemm_4096_p2048_sampled(ozk):
    """The benchmark's product, planes streamed in two groups of moduli."""
    A, B = synth.workload_single(4096, 4096, 4096, 2048, -64, 64, 1004)
    plan = _single(ozk, A, B, 2048, _pairs(4096, 4096, 16, 11))
    assert plan.info["L"] == 329 and plan.info["G"] == 879 and plan.info["crt_mode"] == 2
    assert plan.info["plane_groups"] == 2


def test_gemm_8192_p53_sampled(ozk):
    A, B = synth.workload_single(8192, 8192, 8192, 53, -8, 8, 1004)
    plan = _single(ozk, A, B, 53, _pairs(8192, 8192, 16, 12))
    assert plan.info["G"] == 24


def test_batched64_sampled(ozk):
    probs = synth.batched_problems(64, 1002)
    shapes = [(M, N, K, p) for (M, N, K, p, _, _) in probs]
    plan = ozk.Plan(shapes)
    ws = plan.workspace()
    trip = [(ozk.MPMatrix.from_host(A), ozk.MPMatrix.from_host(B), ozk.MPMatrix.empty(M, N, p))
            for (M, N, K, p, A, B) in probs]
    plan.execute_batched(trip, ws)
    plan.check()
    torch.cuda.synchronize()
    rnd = np.random.Generator(np.random.PCG64(12))
    for q in (0, 9, 17, 25, 33, 40, 51, 63):
        M, N, K, p, A, B = probs[q]
        pairs = [(int(rnd.integers(M)), int(rnd.integers(N))) for _ in range(2)]
        ref = o.ozaki2_entries(A, B, p, pairs)
        Cd = trip[q][2]
        for (i, j), r in zip(pairs, ref):
            limbs = [int(x) & ((1 << 64) - 1) for x in Cd.limbs[:, i, j].cpu().tolist()]
            assert (limbs, int(Cd.exp[i, j].item()), int(Cd.sign[i, j].item())) == \
                (r["limbs"], r["exp"], r["sign"]), (q, i, j)


def test_dgemm_4096_autograd_sampled(ozk):
    from paper_2609_27831_gb300 import autograd as ag
    X, Y, G = synth.fp64_workload(4096, 1003)
    xa = torch.tensor(X, device="cuda", requires_grad=True)
    ya = torch.tensor(Y, device="cuda", requires_grad=True)
    out = ag.ozaki_matmul(xa, ya)
    out.backward(torch.tensor(G, device="cuda"))
    torch.cuda.synchronize()
    n = 4096
    par = o.dgemm_params(n, n, n)
    e, f = o.f64_exponents(X, 1), o.f64_exponents(Y, 0)
    rnd = np.random.Generator(np.random.PCG64(13))
    worst = Fraction(0)
    for _ in range(16):
        i, j, k = (int(rnd.integers(n)) for _ in range(3))
        c, da, db = out[i, j].item(), xa.grad[i, k].item(), ya.grad[k, j].item()
        assert c == o.dgemm_fwd_entry(X, Y, i, j, par, e, f)
        assert da == o.dgemm_dA_entry(Y, G, i, k, par, f)
        assert db == o.dgemm_dB_entry(X, G, k, j, par, e)
        for got, xs, ys in ((c, X[i, :], Y[:, j]), (da, G[i, :], Y[k, :]), (db, X[:, k], G[:, j])):
            ref = o.exact_dot_double(xs, ys)
            u = o.ulp_distance(Fraction(got), Fraction(ref), 53) if ref else abs(got)
            assert u <= 1
            worst = max(worst, u)
    print(f"max ulp binary64 4096^2 forward + backward: {float(worst):.4f} over 48 sampled entries")
