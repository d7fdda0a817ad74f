"""Autotuner of the launch options for a problem class (one GPU).

The library's automatic choices are fixed thresholds measured on one GB300:
the tensor-core residues above 72-byte integers, the tensor-core CRT sums
above 20 accumulator digits, K chunks of 1024, one persistent GEMM CTA per
SM.  ``tune`` measures instead.  For a problem class it runs every candidate
option set on seeded random inputs of that shape, takes the median of a few
timed executions (the library's own stage events on the launch stream), keeps
the fastest, and stores the choice in a JSON cache keyed by the class.  A
class is the shape with M, N and K rounded up to powers of two, and p.

``options_for`` returns the cached choice for a shape ({} when the class has
not been tuned: the automatic choice), ready to pass to ``Plan`` or ``gemm``.
Every option set computes the same bits; only the time differs.
"""
from __future__ import annotations

import json
import os
import statistics

# engine and tile choices: residues (0 automatic, 2 tensor cores, 3 CUDA
# cores), CRT (0 automatic, 2 tensor-core sums, 3 CUDA cores), the K chunk of
# the plane GEMMs' exact accumulation (0 = 1024); the persistent grid stays
# one CTA per SM (grid 0)
CANDIDATES = [
    {"res_engine": r, "crt_engine": c, "k_chunk": 0, "grid": 0} for r in (0, 2, 3) for c in (0, 2, 3)
] + [
    {"res_engine": 0, "crt_engine": 0, "k_chunk": 512, "grid": 0},
]

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


def tune(shape, cache_path: str | None = None, candidates=None, reps: int = 3, measure=None,
         force: bool = False) -> dict:
    """The fastest option set for the class of ``shape`` (cached).

    ``measure(shape, opts, reps) -> ms`` defaults to ``measure_gpu``; a
    candidate it rejects (an exception: options the shape does not support)
    is skipped.  The cache entry records every candidate's time."""
    path = cache_path or DEFAULT_CACHE
    key = problem_class(*shape)
    cache = load_cache(path)
    if not force and key in cache:
        return dict(cache[key]["opts"])
    measure = measure or measure_gpu
    tried = []
    for cand in (candidates or CANDIDATES):
        try:
            ms = float(measure(tuple(shape), dict(cand), reps))
        except Exception as exc:          # unsupported for this shape: skip it
            tried.append({"opts": dict(cand), "error": f"{type(exc).__name__}: {exc}"})
            continue
        tried.append({"opts": dict(cand), "ms": ms})
    timed = [t for t in tried if "ms" in t]
    if not timed:
        raise RuntimeError(f"no candidate ran for {key}")
    best = min(timed, key=lambda t: t["ms"])
    cache[key] = {"opts": best["opts"], "ms": best["ms"], "shape": list(shape), "tried": tried}
    save_cache(path, cache)
    return dict(best["opts"])


def options_for(shape, cache_path: str | None = None) -> dict:
    """The cached choice for the class of ``shape``, or {} (automatic)."""
    entry = load_cache(cache_path or DEFAULT_CACHE).get(problem_class(*shape))
    return dict(entry["opts"]) if entry else {}
