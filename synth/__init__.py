"""Seeded synthetic inputs for the Ozaki-II multiple-precision GEMM.

This module only draws random numbers and packs them into the storage format;
it holds none of the method's arithmetic, so both the CUDA path and the CPU
oracle can take their inputs from it.

Storage format of a p-bit matrix with R rows and C columns (row-major):

* ``limbs``: uint64 array ``[nl, R, C]`` (``nl = ceil(p/64)``), limb plane
  ``q`` holds limb ``q`` of every element, least-significant limb first.
  A nonzero significand is MSB-normalised: bit 63 of limb ``nl-1`` is set and
  the ``64*nl - p`` lowest bits are zero.
* ``exp``: int32 ``[R, C]``, MPFR convention ``|x| in [2^(exp-1), 2^exp)``.
* ``sign``: int8 ``[R, C]``, 0 for +, 1 for -.

Value of an element: ``(-1)^sign * sum_q limb_q 2^(64 q) * 2^(exp - 64 nl)``.
Zero is all limbs 0 (exp and sign are then ignored).

Workload shapes follow the paper's sweeps (uniform random significands with a
random sign and a spread of exponents, Sec. 6): the generators below state each
recipe; every array comes from a numpy PCG64 stream seeded by the caller.
"""
from __future__ import annotations

import math

import numpy as np

U64_MAX = np.iinfo(np.uint64).max


def nlimbs(p: int) -> int:
    return (p + 63) // 64


def mp_matrix(rng: np.random.Generator, rows: int, cols: int, p: int,
              exp_lo: int, exp_hi: int, zero_frac: float = 0.0,
              row_spread: int = 0, col_spread: int = 0) -> dict:
    """Random p-bit matrix: p uniform random significand bits with the top bit
    set, uniform random sign, exponent uniform in [exp_lo, exp_hi] per entry.

    ``row_spread``/``col_spread`` add a per-row / per-column integer offset drawn
    uniformly from [-spread, spread] (stresses the shared-exponent scaling).
    ``zero_frac`` sets that fraction of entries to exact zero.
    """
    nl = nlimbs(p)
    limbs = rng.integers(0, U64_MAX, size=(nl, rows, cols), dtype=np.uint64,
                         endpoint=True)
    low = 64 * nl - p  # 0 <= low < 64: bits below the p-bit significand are zero
    if low:
        limbs[0] &= np.uint64(int(U64_MAX) ^ ((1 << low) - 1))
    limbs[nl - 1] |= np.uint64(1) << np.uint64(63)
    exp = rng.integers(exp_lo, exp_hi, size=(rows, cols), endpoint=True).astype(np.int32)
    if row_spread:
        exp += rng.integers(-row_spread, row_spread, size=(rows, 1), endpoint=True).astype(np.int32)
    if col_spread:
        exp += rng.integers(-col_spread, col_spread, size=(1, cols), endpoint=True).astype(np.int32)
    sign = rng.integers(0, 1, size=(rows, cols), dtype=np.int8, endpoint=True)
    if zero_frac > 0:
        z = rng.random(size=(rows, cols)) < zero_frac
        limbs[:, z] = 0
        exp[z] = 0
        sign[z] = 0
    return {"p": p, "limbs": limbs, "exp": exp, "sign": sign}


def zero_rows(m: dict, rows) -> dict:
    """Return a copy with the given rows set to exact zero."""
    out = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in m.items()}
    out["limbs"][:, rows, :] = 0
    out["exp"][rows, :] = 0
    out["sign"][rows, :] = 0
    return out


def zero_cols(m: dict, cols) -> dict:
    out = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in m.items()}
    out["limbs"][:, :, cols] = 0
    out["exp"][:, cols] = 0
    out["sign"][:, cols] = 0
    return out


def fp64_matrix(rng: np.random.Generator, rows: int, cols: int, u_lo: int = -20,
                u_hi: int = 20) -> np.ndarray:
    """binary64 matrix with entries normal(0,1) * 2^u, u uniform integer."""
    x = rng.standard_normal(size=(rows, cols))
    u = rng.integers(u_lo, u_hi, size=(rows, cols), endpoint=True)
    return np.ldexp(x, u)


def fp64_normal(rng: np.random.Generator, rows: int, cols: int) -> np.ndarray:
    return rng.standard_normal(size=(rows, cols))


# ---------------------------------------------------------------------------
# Named workloads (seed = 1000 + workload index)
# ---------------------------------------------------------------------------

def workload_single(M: int, N: int, K: int, p: int, exp_lo: int, exp_hi: int,
                    seed: int) -> tuple[dict, dict]:
    rng = np.random.Generator(np.random.PCG64(seed))
    A = mp_matrix(rng, M, K, p, exp_lo, exp_hi)
    B = mp_matrix(rng, K, N, p, exp_lo, exp_hi)
    return A, B


def gemm_256_p53(seed: int = 1000):
    """M=N=K=256, p=53: 53-bit significands in [2^52, 2^53), exponent in [-8, 8]."""
    return workload_single(256, 256, 256, 53, -8, 8, seed)


def gemm_1024_p256(seed: int = 1001):
    """M=N=K=1024, p=256: 256 random bits (top set), exponent i.i.d. in [-32, 32]."""
    return workload_single(1024, 1024, 1024, 256, -32, 32, seed)


def batched_problem_shapes(count: int = 64, seed: int = 1002):
    """Shapes of the batched workload: M, N, K log-uniform in [128, 2048]
    independently, p uniform in {113, 256, 512}."""
    rng = np.random.Generator(np.random.PCG64(seed))
    lo, hi = math.log(128), math.log(2048)
    shapes = []
    for _ in range(count):
        M, N, K = (int(round(math.exp(rng.uniform(lo, hi)))) for _ in range(3))
        p = int(rng.choice([113, 256, 512]))
        shapes.append((M, N, K, p))
    return shapes


def batched_problems(count: int = 64, seed: int = 1002):
    """The batched workload's inputs (as the 256^3 p=53 workload, at width p)."""
    shapes = batched_problem_shapes(count, seed)
    probs = []
    for idx, (M, N, K, p) in enumerate(shapes):
        rng = np.random.Generator(np.random.PCG64(seed * 1000 + idx))
        A = mp_matrix(rng, M, K, p, -8, 8)
        B = mp_matrix(rng, K, N, p, -8, 8)
        probs.append((M, N, K, p, A, B))
    return probs


def fp64_workload(n: int = 4096, seed: int = 1003):
    """binary64 differentiation workload: A, B = normal(0,1)*2^u with u uniform
    integer in [-20, 20]; dC normal(0,1)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    A = fp64_matrix(rng, n, n)
    B = fp64_matrix(rng, n, n)
    dC = fp64_normal(rng, n, n)
    return A, B, dC
