"""Host logic of the autotuner (CPU, with fake timers)."""
import json

import pytest

from paper_2609_27831_gb300 import autotune as at


def test_problem_class_rounds_up_to_powers_of_two():
    assert at.problem_class(1000, 1024, 1025, 256) == "1024x1024x2048:p256"
    assert at.problem_class(1, 2, 3, 53) == "1x2x4:p53"


def _cost(shape, opts, reps):
    if opts.get("res_engine") == 2 and opts.get("crt_engine") == 3:
        raise RuntimeError("unsupported here")
    return (1.0 + 0.1 * opts.get("res_engine", 0) + (0.5 if opts.get("crt_engine", 0) == 0 else 0.0)
            + opts.get("k_chunk", 0) / 1e4 + (0.01 if opts.get("crt_engine") == 3 else 0.0)
            - (0.2 if opts.get("gemm_tile") == 2 else 0.0))


def test_tune_searches_stage_by_stage_and_caches(tmp_path):
    path = str(tmp_path / "tune.json")
    seen = []

    def fake(shape, opts, reps):
        seen.append(dict(opts))
        return _cost(shape, opts, reps)

    best = at.tune((100, 200, 300, 256), path, measure=fake, reps=1)
    # stage 1 picks the pair tile with the whole K chunk; stage 2 the engines on top of it
    assert best == {"gemm_tile": 2, "k_chunk": 0, "res_engine": 0, "crt_engine": 2}
    assert len(seen) == len(at.STAGES[0]) + len(at.STAGES[1])
    assert all(s["gemm_tile"] == 2 and s["k_chunk"] == 0 for s in seen[len(at.STAGES[0]):])
    entry = json.load(open(path))["128x256x512:p256"]
    assert entry["ms"] == pytest.approx(0.8)
    assert sum("error" in t for t in entry["tried"]) == 1          # the rejected candidate is recorded
    # the same class comes from the cache without measuring
    assert at.tune((128, 256, 512, 256), path, measure=lambda *a: pytest.fail("measured")) == best
    assert at.options_for((120, 250, 500, 256), path) == best
    assert at.options_for((64, 64, 64, 53), path) == {}
    # force re-measures
    again = at.tune((100, 200, 300, 256), path, measure=fake, force=True)
    assert again == best and len(seen) == 2 * (len(at.STAGES[0]) + len(at.STAGES[1]))


def test_tune_fails_when_nothing_runs(tmp_path):
    def bad(shape, opts, reps):
        raise RuntimeError("no")
    with pytest.raises(RuntimeError):
        at.tune((8, 8, 8, 53), str(tmp_path / "t.json"), measure=bad)


def test_unreadable_cache_is_empty(tmp_path):
    p = tmp_path / "bad.json"
    p.write_text("not json")
    assert at.load_cache(str(p)) == {}
    assert at.options_for((8, 8, 8, 53), str(p)) == {}


def test_tune_batched_per_problem_then_launch_wide_tile(tmp_path):
    """Each problem class is tuned for its K chunk and engines (no tile), and
    the launch-wide tile is measured on the whole batch with those choices."""
    path = str(tmp_path / "tune.json")
    shapes = [(100, 200, 300, 256), (64, 64, 64, 53), (100, 200, 300, 256)]

    def per_class(shape, opts, reps):
        assert "gemm_tile" not in opts                   # the tile is chosen for the batch
        c = _cost(shape, opts, reps)
        return c + (0.3 if shape[3] == 53 and opts.get("res_engine") == 0 else 0.0)

    batches = []

    def batch(shapes_, opts, per_problem, reps):
        batches.append((dict(opts), [dict(d) for d in per_problem]))
        return 5.0 if opts["gemm_tile"] == 1 else 4.0

    got = at.tune_batched(shapes, path, measure=per_class, measure_batch=batch, reps=1)
    assert got["opts"] == {"gemm_tile": 2}
    assert got["per_problem"][0] == {"k_chunk": 0, "res_engine": 0, "crt_engine": 2}
    assert got["per_problem"][1]["res_engine"] != 0
    assert got["per_problem"][2] == got["per_problem"][0]
    assert [b[0] for b in batches] == at.PLAN_STAGE
    assert all(b[1] == got["per_problem"] for b in batches)
    # cached as a whole
    again = at.tune_batched(shapes, path, measure=lambda *a: pytest.fail("measured"),
                            measure_batch=lambda *a: pytest.fail("measured"))
    assert again == got
    assert at.batch_key(shapes) != at.batch_key(shapes[:2])
