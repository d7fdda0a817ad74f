"""Autotuner of the launch options for a problem class and for batches (one GPU).

The library's automatic choices are fixed thresholds measured on one GB300:
the tensor-core residues above 72-byte integers, the tensor-core CRT sums
above 20 accumulator digits, K chunks of 1024, CTA-pair plane GEMM tiles
(256 x 256) for products below 1e13 plane flops.  ``tune`` measures instead.
For a problem class it searches the options stage by stage (the plane GEMM
tile and K chunk first, then the residue and CRT engines with the best of
those), each candidate run on seeded random inputs of that shape, taking the
median of a few timed executions (the library's own stage events on the
launch stream), and stores the choice in a JSON cache keyed by the class.  A
class is the shape with M, N and K rounded up to powers of two, and p.

``tune_batched`` gives a batch per-problem choices (each problem's class
tuned for its K chunk and engines) and one launch-wide plane GEMM tile,
measured on the whole batch; ``Plan(shapes, per_problem=..., **opts)`` takes
them.  ``options_for`` returns the cached choice for a shape ({} when the
class has not been tuned: the automatic choice), ready to pass to ``Plan`` or
``gemm``.  Every option set computes the same bits; only the time differs.
"""
from __future__ import annotations

import json
import os
import statistics

# the search, stage by stage: each stage's candidates are tried on top of the
# best choice so far (an empty dict = the automatic choice)
PLAN_STAGE = [{"gemm_tile": g} for g in (1, 2)]
CHUNK_STAGE = [{"k_chunk": k} for k in (0, 512)]
ENGINE_STAGE = [{"res_engine": r, "crt_engine": c} for r in (0, 2, 3) for c in (0, 2, 3)]
STAGES = [[dict(a, **b) for a in PLAN_STAGE for b in CHUNK_STAGE], ENGINE_STAGE]
# the options a batched plan takes per problem
PER_PROBLEM_KEYS = ("k_chunk", "res_engine", "crt_engine")

DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "ozaki2_gb300_tune.json")


def _pow2(x: int) -> int:
    return 1 << max(0, int(x) - 1).bit_length()


def problem_class(M: int, N: int, K: int, p: int) -> str:
    """Cache key of a shape: M, N, K rounded up to powers of two, and p."""
    return f"{_pow2(M)}x{_pow2(N)}x{_pow2(K)}:p{int(p)}"


def load_cache(path: str) -> dict:
    try:
        with open(path) as fh:
            data = json.load(fh)
        return data if isinstance(data, dict) else {}
    except (OSError, ValueError):
        return {}


def save_cache(path: str, cache: dict) -> None:
    os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
    tmp = path + ".tmp"
    with open(tmp, "w") as fh:
        json.dump(cache, fh, indent=1, sort_keys=True)
    os.replace(tmp, path)


def _random_operand(rng, rows: int, cols: int, p: int) -> dict:
    """Seeded random p-bit matrix in the storage format (MSB-normalised
    significands, exponents in [-8, 8], random signs)."""
    import numpy as np
    nl = (p + 63) // 64
    limbs = rng.integers(0, np.iinfo(np.uint64).max, size=(nl, rows, cols), dtype=np.uint64, endpoint=True)
    low = 64 * nl - p
    if low:
        limbs[0] &= np.uint64(int(np.iinfo(np.uint64).max) ^ ((1 << low) - 1))
    limbs[nl - 1] |= np.uint64(1) << np.uint64(63)
    exp = rng.integers(-8, 8, size=(rows, cols), endpoint=True).astype(np.int32)
    sign = rng.integers(0, 1, size=(rows, cols), dtype=np.int8, endpoint=True)
    return {"p": p, "limbs": limbs, "exp": exp, "sign": sign}


def measure_gpu(shape, opts: dict, reps: int = 3, warmup: int = 2, seed: int = 1234) -> float:
    """Median device time (ms) of one execute of ``shape`` with ``opts``."""
    import numpy as np
    import torch
    from . import MPMatrix, Plan
    M, N, K, p = shape
    rng = np.random.Generator(np.random.PCG64(seed))
    A = MPMatrix.from_host(_random_operand(rng, M, K, p))
    B = MPMatrix.from_host(_random_operand(rng, K, N, p))
    C = MPMatrix.empty(M, N, p)
    plan = Plan((M, N, K, p), timing=1, **opts)
    ws = plan.workspace()
    for _ in range(warmup):
        plan.execute(A, B, C, ws)
    times = []
    for _ in range(max(1, reps)):
        plan.execute(A, B, C, ws)
        times.append(plan.timings()["total"])
    plan.check()
    torch.cuda.synchronize()
    return statistics.median(times)


def tune(shape, cache_path: str | None = None, stages=None, reps: int = 3, measure=None,
         force: bool = False) -> dict:
    """The fastest option set for the class of ``shape`` (cached).

    ``stages`` (default STAGES) is a list of candidate lists, searched in
    order: every candidate of a stage is measured on top of the best options
    of the stages before, and the fastest is kept (ties go to the earlier
    candidate).  ``measure(shape, opts, reps) -> ms`` defaults to
    ``measure_gpu``; a candidate it rejects (an exception: options the shape
    does not support) is skipped.  The cache entry records every candidate's
    time."""
    path = cache_path or DEFAULT_CACHE
    key = problem_class(*shape)
    cache = load_cache(path)
    if not force and key in cache:
        return dict(cache[key]["opts"])
    measure = measure or measure_gpu
    best: dict = {}
    best_ms = None
    tried = []
    for stage in (stages or STAGES):
        stage_best, stage_ms = None, None
        for cand in stage:
            opts = dict(best, **cand)
            try:
                ms = float(measure(tuple(shape), dict(opts), reps))
            except Exception as exc:      # unsupported for this shape: skip it
                tried.append({"opts": opts, "error": f"{type(exc).__name__}: {exc}"})
                continue
            tried.append({"opts": opts, "ms": ms})
            if stage_ms is None or ms < stage_ms:
                stage_best, stage_ms = opts, ms
        if stage_best is not None:
            best, best_ms = stage_best, stage_ms
    if best_ms is None:
        raise RuntimeError(f"no candidate ran for {key}")
    cache[key] = {"opts": best, "ms": best_ms, "shape": list(shape), "tried": tried}
    save_cache(path, cache)
    return dict(best)


def options_for(shape, cache_path: str | None = None) -> dict:
    """The cached choice for the class of ``shape``, or {} (automatic)."""
    entry = load_cache(cache_path or DEFAULT_CACHE).get(problem_class(*shape))
    return dict(entry["opts"]) if entry else {}


def batch_key(shapes) -> str:
    """Cache key of a batch: its problem classes in order."""
    import hashlib
    text = ";".join(problem_class(*s) for s in shapes)
    return "batch:" + hashlib.sha1(text.encode()).hexdigest()[:16]


def measure_batch_gpu(shapes, opts: dict, per_problem, reps: int = 3, warmup: int = 2, seed: int = 4321) -> float:
    """Median device time (ms) of one batched execute of ``shapes``."""
    import numpy as np
    import torch
    from . import MPMatrix, Plan
    rng = np.random.Generator(np.random.PCG64(seed))
    trip = []
    for (M, N, K, p) in shapes:
        trip.append((MPMatrix.from_host(_random_operand(rng, M, K, p)),
                     MPMatrix.from_host(_random_operand(rng, K, N, p)), MPMatrix.empty(M, N, p)))
    plan = Plan(list(shapes), per_problem=per_problem, timing=1, **opts)
    ws = plan.workspace()
    for _ in range(warmup):
        plan.execute_batched(trip, ws)
    times = []
    for _ in range(max(1, reps)):
        plan.execute_batched(trip, ws)
        times.append(plan.timings()["total"])
    plan.check()
    torch.cuda.synchronize()
    return statistics.median(times)


def tune_batched(shapes, cache_path: str | None = None, reps: int = 3, measure=None, measure_batch=None,
                 force: bool = False) -> dict:
    """Options for a batch: {"opts": launch-wide options, "per_problem": [...]}.

    Each problem's class is tuned for its K chunk and engines (the stages
    without the plane GEMM tile, cached per class as by ``tune``); the tile,
    which one grouped launch shares, is then measured on the whole batch with
    those per-problem choices (``measure_batch(shapes, opts, per_problem,
    reps) -> ms``, default ``measure_batch_gpu``)."""
    path = cache_path or DEFAULT_CACHE
    key = batch_key(shapes)
    cache = load_cache(path)
    if not force and key in cache:
        e = cache[key]
        return {"opts": dict(e["opts"]), "per_problem": [dict(d) for d in e["per_problem"]]}
    problem_stages = [CHUNK_STAGE, ENGINE_STAGE]
    per_problem = []
    for s_ in shapes:
        best = tune(s_, path, stages=problem_stages, reps=reps, measure=measure, force=force)
        per_problem.append({k: v for k, v in best.items() if k in PER_PROBLEM_KEYS})
    measure_batch = measure_batch or measure_batch_gpu
    tried = []
    for cand in PLAN_STAGE:
        try:
            ms = float(measure_batch(list(shapes), dict(cand), per_problem, reps))
        except Exception as exc:
            tried.append({"opts": dict(cand), "error": f"{type(exc).__name__}: {exc}"})
            continue
        tried.append({"opts": dict(cand), "ms": ms})
    timed = [t for t in tried if "ms" in t]
    if not timed:
        raise RuntimeError(f"no launch-wide candidate ran for {key}")
    best = min(timed, key=lambda t: t["ms"])
    cache = load_cache(path)
    cache[key] = {"opts": best["opts"], "ms": best["ms"], "per_problem": per_problem, "tried": tried,
                  "shapes": [list(s_) for s_ in shapes]}
    save_cache(path, cache)
    return {"opts": dict(best["opts"]), "per_problem": per_problem}
