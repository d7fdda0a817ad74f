"""Host logic of the autotuner (CPU, with a fake timer)."""
import json

import pytest

from paper_2609_27831_gb300 import autotune as at


def test_problem_class_rounds_up_to_powers_of_two():
    assert at.problem_class(1000, 1024, 1025, 256) == "1024x1024x2048:p256"
    assert at.problem_class(1, 2, 3, 53) == "1x2x4:p53"


def _cost(shape, opts, reps):
    if opts["res_engine"] == 2 and opts["crt_engine"] == 3:
        raise RuntimeError("unsupported here")
    return (1.0 + 0.1 * opts["res_engine"] + (0.5 if opts["crt_engine"] == 0 else 0.0)
            + opts["k_chunk"] / 1e4 + opts["grid"] / 1e4 + (0.01 if opts["crt_engine"] == 3 else 0.0))


def test_tune_picks_the_fastest_and_caches(tmp_path):
    path = str(tmp_path / "tune.json")
    seen = []

    def fake(shape, opts, reps):
        seen.append(dict(opts))
        return _cost(shape, opts, reps)

    best = at.tune((100, 200, 300, 256), path, measure=fake, reps=1)
    assert best == {"res_engine": 0, "crt_engine": 2, "k_chunk": 0, "grid": 0}
    assert len(seen) == len(at.CANDIDATES)
    entry = json.load(open(path))["128x256x512:p256"]
    assert entry["ms"] == pytest.approx(1.0)
    assert sum("error" in t for t in entry["tried"]) == 1          # the rejected candidate is recorded
    # the same class comes from the cache without measuring
    assert at.tune((128, 256, 512, 256), path, measure=lambda *a: pytest.fail("measured")) == best
    assert at.options_for((120, 250, 500, 256), path) == best
    assert at.options_for((64, 64, 64, 53), path) == {}
    # force re-measures
    again = at.tune((100, 200, 300, 256), path, measure=fake, force=True)
    assert again == best and len(seen) == 2 * len(at.CANDIDATES)


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
