"""The autotuner on the GPU: a small class tuned for real, and the chosen
options give the same bits as the automatic ones."""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)


def test_tune_small_class_and_same_bits(tmp_path):
    from paper_2609_27831_gb300 import build
    build.build()
    import paper_2609_27831_gb300 as ozk
    from paper_2609_27831_gb300 import autotune as at
    shape = (256, 256, 256, 300)
    path = str(tmp_path / "tune.json")
    best = at.tune(shape, path, reps=1)
    assert best in at.CANDIDATES
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
