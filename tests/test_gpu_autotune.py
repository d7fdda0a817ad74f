"""The autotuner on the GPU: a small class and a small batch tuned for real,
and the chosen options give the same bits as the automatic ones."""
import numpy as np
import pytest

import synth

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


def test_tune_small_class_and_same_bits(ozk, tmp_path):
    from paper_2609_27831_gb300 import autotune as at
    shape = (256, 256, 256, 300)
    path = str(tmp_path / "tune.json")
    best = at.tune(shape, path, reps=1)
    assert set(best) == {"gemm_tile", "k_chunk", "res_engine", "crt_engine"}
    assert at.options_for(shape, path) == best
    rng = np.random.Generator(np.random.PCG64(2077))
    A = synth.mp_matrix(rng, 256, 256, 300, -8, 8)
    B = synth.mp_matrix(rng, 256, 256, 300, -8, 8)
    dA, dB = ozk.MPMatrix.from_host(A), ozk.MPMatrix.from_host(B)
    outs = []
    for kw in ({}, best):
        plan = ozk.Plan(shape, **kw)
        ws = plan.workspace()
        C = ozk.MPMatrix.empty(256, 256, 300)
        plan.execute(dA, dB, C, ws)
        plan.check()
        outs.append(C.to_host())
    for key in ("limbs", "exp", "sign"):
        assert np.array_equal(outs[0][key], outs[1][key])


def test_tune_small_batch_and_same_bits(ozk, tmp_path):
    from paper_2609_27831_gb300 import autotune as at
    shapes = [(200, 130, 150, 256), (64, 300, 90, 113), (150, 150, 150, 512)]
    path = str(tmp_path / "tune.json")
    got = at.tune_batched(shapes, path, reps=1)
    assert got["opts"] in at.PLAN_STAGE and len(got["per_problem"]) == 3
    rng = np.random.Generator(np.random.PCG64(2078))
    trips = []
    for (M, N, K, p) in shapes:
        A = ozk.MPMatrix.from_host(synth.mp_matrix(rng, M, K, p, -8, 8))
        B = ozk.MPMatrix.from_host(synth.mp_matrix(rng, K, N, p, -8, 8))
        trips.append((A, B))
    outs = []
    for kw in ({}, dict(got["opts"], per_problem=got["per_problem"])):
        plan = ozk.Plan(shapes, **kw)
        trip = [(A, B, ozk.MPMatrix.empty(M, N, p)) for (A, B), (M, N, K, p) in zip(trips, shapes)]
        plan.execute_batched(trip, plan.workspace())
        plan.check()
        outs.append([c.to_host() for (_, _, c) in trip])
    for a, b in zip(*outs):
        for key in ("limbs", "exp", "sign"):
            assert np.array_equal(a[key], b[key])
