"""Complex products (3M form in the residue domain) on the GPU against the
oracle's complex method: the CRT integers of both parts and both rounded
outputs bit for bit, and against the exact complex product (<= 1 ulp)."""
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


def _chat(buf, D, M, N):
    ch = buf.cpu().numpy().view(np.uint32)
    vals = []
    for r in ch:
        mag = 0
        for d in range(D):
            mag |= int(r[1 + d]) << (32 * d)
        vals.append(-mag if r[0] else mag)
    return np.array(vals, dtype=object).reshape(M, N)


@pytest.mark.parametrize("shape,p,kw", [
    ((40, 30, 50), 53, {}),
    ((130, 70, 90), 256, {}),                       # two-limb moduli, tensor-core CRT sums
    ((33, 260, 20), 113, {"gemm_tile": 2}),         # CTA-pair plane GEMMs
    ((20, 24, 30), 1024, {}),                       # tensor-core residues
])
def test_complex_3m_against_oracle(ozk, shape, p, kw):
    M, N, K = shape
    rng = np.random.Generator(np.random.PCG64(8100 + p + M))
    Ar, Ai = synth.mp_matrix(rng, M, K, p, -8, 8), synth.mp_matrix(rng, M, K, p, -8, 8)
    Br, Bi = synth.mp_matrix(rng, K, N, p, -8, 8), synth.mp_matrix(rng, K, N, p, -8, 8)
    Ai = synth.zero_rows(Ai, [1])                    # a row that is real only
    plan = ozk.ComplexPlan((M, N, K, p), **kw)
    D = plan.info["crt_digits"]
    bufs = [torch.zeros((M * N, D + 1), dtype=torch.int32, device="cuda") for _ in range(2)]
    for i, b in enumerate(bufs):
        plan.set_debug_chat(i, b)
    d = [ozk.MPMatrix.from_host(x) for x in (Ar, Ai, Br, Bi)]
    Cr, Ci = ozk.MPMatrix.empty(M, N, p), ozk.MPMatrix.empty(M, N, p)
    plan.execute_complex(*d, Cr, Ci, plan.workspace())
    plan.check()
    torch.cuda.synchronize()
    ref = o.complex_full(Ar, Ai, Br, Bi, p)
    assert plan.info["t"] == ref["par"].t and plan.info["L"] == ref["par"].L
    chr_, chi = _chat(bufs[0], D, M, N), _chat(bufs[1], D, M, N)
    assert all(chr_[i, j] == ref["chat_r"][i, j] and chi[i, j] == ref["chat_i"][i, j]
               for i in range(M) for j in range(N))
    for got, part in ((Cr.to_host(), "Cr"), (Ci.to_host(), "Ci")):
        for key in ("limbs", "exp", "sign"):
            assert np.array_equal(got[key], ref[part][key]), (part, key)
    # and against the exact complex product at a few entries
    for (i, j) in ((0, 0), (M - 1, N - 1), (1, 2)):
        tr = o.complex_truth_entry(Ar, Ai, Br, Bi, i, j, p)
        for got, t in ((Cr, tr[0]), (Ci, tr[1])):
            h = got.to_host()
            g = o.to_fraction(*o.matrix_entry(h, i, j))
            tv = o.to_fraction(*t)
            assert (o.ulp_distance(g, tv, p) if tv else abs(g)) <= 1


def test_zgemm_convenience_matches_the_plan(ozk):
    M, N, K, p = 50, 40, 70, 200
    rng = np.random.Generator(np.random.PCG64(8200))
    mats = [synth.mp_matrix(rng, *s, p, -6, 6) for s in ((M, K), (M, K), (K, N), (K, N))]
    d = [ozk.MPMatrix.from_host(x) for x in mats]
    Cr, Ci = ozk.zgemm(*d, p)
    plan = ozk.ComplexPlan((M, N, K, p))
    Pr, Pi = ozk.MPMatrix.empty(M, N, p), ozk.MPMatrix.empty(M, N, p)
    plan.execute_complex(*d, Pr, Pi, plan.workspace())
    plan.check()
    torch.cuda.synchronize()
    for a, b in ((Cr, Pr), (Ci, Pi)):
        for key in ("limbs", "exp", "sign"):
            assert torch.equal(getattr(a, key), getattr(b, key))
