"""Failure detection on the GPU, with every failure made on the host (no
GPU fault, trap or endless wait is involved):

* a bounded device-side wait that runs out (the plan's wait limit lowered to
  one poll) sets the device status word, ozaki2_check reports OZ2_ETIMEOUT,
  and the same context then computes the next product correctly;
* CRT tables corrupted on the host before upload make the direct CRT's range
  check (x0 < P, Sec. 4.4) fail: OZ2_EINTERNAL;
* an injected device allocation failure is reported as OZ2_ENOMEM and the
  next execute of the same plan succeeds.
"""
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


def _inputs(M, N, K, p, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    return synth.mp_matrix(rng, M, K, p, -8, 8), synth.mp_matrix(rng, K, N, p, -8, 8)


def _run(ozk, plan, A, B, p):
    M, K = A["exp"].shape
    N = B["exp"].shape[1]
    dC = ozk.MPMatrix.empty(M, N, p)
    plan.execute(ozk.MPMatrix.from_host(A), ozk.MPMatrix.from_host(B), dC, plan.workspace())
    return dC


def _equal_to_oracle(got, A, B, p):
    ref = o.ozaki2_full(A, B, p)["C"]
    h = got.to_host()
    return all(np.array_equal(h[k], ref[k]) for k in ("limbs", "exp", "sign"))


@pytest.mark.parametrize("shape,p,kw", [((64, 64, 64), 53, {}),                    # plane GEMM waits
                                        ((64, 64, 64), 256, {"res_engine": 2})])    # + tensor-core residues and CRT
def test_bounded_wait_runs_out(ozk, shape, p, kw):
    M, N, K = shape
    A, B = _inputs(M, N, K, p, 6100 + p)
    plan = ozk.Plan((M, N, K, p), **kw)
    assert ozk.lib().ozaki2_plan_set_wait_limit(plan._h, 1) == 0
    _run(ozk, plan, A, B, p)
    with pytest.raises(ozk.OzakiError) as ei:
        plan.check()
    assert ei.value.status == ozk._lib.OZ2_ETIMEOUT
    plan.check()                                     # the word was cleared by the read
    # the context is still usable: the default limit gives the oracle's bits
    assert ozk.lib().ozaki2_plan_set_wait_limit(plan._h, 0) == 0
    got = _run(ozk, plan, A, B, p)
    plan.check()
    torch.cuda.synchronize()
    assert _equal_to_oracle(got, A, B, p)


@pytest.mark.parametrize("p,crt_engine,crt_mode", [(113, 0, 0), (256, 2, 2)])
def test_corrupted_crt_table_trips_the_range_check(ozk, p, crt_engine, crt_mode):
    M = N = K = 64
    A, B = _inputs(M, N, K, p, 6200 + p)
    plan = ozk.Plan((M, N, K, p), crt_engine=crt_engine)
    assert plan.info["crt_mode"] == crt_mode
    assert ozk.lib().ozaki2_plan_debug_corrupt_crt(plan._h, 0) == 0
    _run(ozk, plan, A, B, p)
    with pytest.raises(ozk.OzakiError) as ei:
        plan.check()
    assert ei.value.status == ozk._lib.OZ2_EINTERNAL
    # an intact plan on the same inputs passes its check
    good = ozk.Plan((M, N, K, p), crt_engine=crt_engine)
    got = _run(ozk, good, A, B, p)
    good.check()
    assert _equal_to_oracle(got, A, B, p)


def test_injected_device_allocation_failure(ozk):
    M = N = K = 48
    p = 113
    A, B = _inputs(M, N, K, p, 6300)
    plan = ozk.Plan((M, N, K, p))
    # the device tables of the first execute
    assert ozk.lib().ozaki2_debug_inject_alloc_failure(1) == 0
    with pytest.raises(ozk.OzakiError) as ei:
        _run(ozk, plan, A, B, p)
    assert ei.value.status == ozk._lib.OZ2_ENOMEM
    got = _run(ozk, plan, A, B, p)
    plan.check()
    torch.cuda.synchronize()
    assert _equal_to_oracle(got, A, B, p)
    # the launch image of a captured graph (the plan's tables exist by now)
    dA, dB = ozk.MPMatrix.from_host(A), ozk.MPMatrix.from_host(B)
    dC = ozk.MPMatrix.empty(M, N, p)
    ws = plan.workspace()
    s = torch.cuda.Stream()
    assert ozk.lib().ozaki2_debug_inject_alloc_failure(1) == 0
    with torch.cuda.stream(s):
        with pytest.raises(ozk.OzakiError) as ei:
            plan.graph([(dA, dB, dC)], ws, s)
        assert ei.value.status == ozk._lib.OZ2_ENOMEM
        g = plan.graph([(dA, dB, dC)], ws, s)
    g.launch(torch.cuda.current_stream())
    plan.check()
    torch.cuda.synchronize()
    assert _equal_to_oracle(dC, A, B, p)
