"""Constructed inputs whose integerization (Eq. 1) or final rounding to p bits
lands exactly on a round-half-even tie, with the results fixed by hand.

Shared by the oracle pins (CPU) and the GPU parity tests; no method
arithmetic lives here, only the construction of inputs in the storage format
and the expected values stated as integers.
"""
from __future__ import annotations

import numpy as np


def mat_from_values(rows, p: int) -> dict:
    """A p-bit matrix (storage format) from rows of exact dyadic values given
    as (numerator, power) pairs, value = numerator * 2^power, |numerator| < 2^p."""
    R, C = len(rows), len(rows[0])
    nl = (p + 63) // 64
    limbs = np.zeros((nl, R, C), dtype=np.uint64)
    exp = np.zeros((R, C), dtype=np.int32)
    sign = np.zeros((R, C), dtype=np.int8)
    for r, row in enumerate(rows):
        for c, (num, pw) in enumerate(row):
            if num == 0:
                continue
            a = abs(num)
            assert a < (1 << p)
            e = a.bit_length() + pw                       # |x| in [2^(e-1), 2^e)
            sig = a << (64 * nl - a.bit_length())         # MSB-normalised
            for q in range(nl):
                limbs[q, r, c] = (sig >> (64 * q)) & ((1 << 64) - 1)
            exp[r, c] = e
            sign[r, c] = 1 if num < 0 else 0
    return {"p": p, "limbs": limbs, "exp": exp, "sign": sign}


def final_rounding_ties(p: int):
    """Rows of A (with B a column of ones) whose exact product is a tie (or just
    off one) at p bits, and the correctly rounded results by hand, each as an
    integer times 2^-10.

    T = 2^p: T + 1 needs p + 1 bits, so the last bit is dropped."""
    T = 1 << p                                            # written (1, p): its numerator is 1
    eps = (1, -10)                                        # 2^-10: exact after integerization
    cases = [
        # (row of A as (numerator, power) pairs, expected value as an integer times 2^-10)
        ([(1, p), (1, 0), (0, 0)], T << 10),                        # T + 1: tie, kept LSB even -> T
        ([(1, p), (3, 0), (0, 0)], (T + 4) << 10),                  # T + 3: tie, kept LSB odd -> T + 4
        ([(1, p), (5, 0), (0, 0)], (T + 4) << 10),                  # T + 5: tie, even -> T + 4
        ([(-1, p), (-1, 0), (0, 0)], -(T << 10)),                   # negative tie
        ([(T - 1, 1), (1, 0), (0, 0)], (2 * T) << 10),              # 2T - 1: odd kept, carry out -> 2T
        ([(1, p), (1, 0), eps], (T + 2) << 10),                     # just above the tie -> up
        ([(1, p), (1, 0), (-1, -10)], T << 10),                     # just below the tie -> down
        ([(1, p), (-1, 0), (0, 0)], (T - 1) << 10),                 # T - 1 fits in p bits: exact
    ]
    return cases


def integerization_ties(p: int, K: int):
    """Rows of A with one entry at 2^(E-1) (setting the shared exponent E) and
    entries d bits lower whose dropped bits are exactly half an integer step
    of the scaled integer, with even and odd kept bits, and entries just off
    the tie.  Returns the rows as (numerator, power) pairs and d; the scaled
    integer of entry x is round(x 2^(t - E)) with t = p + 16 + ceil(log2 K)."""
    t = p + 16 + (K - 1).bit_length()
    E = 0                                                 # the large entry is 2^(E-1) = 1/2
    d = t - p + 20                                        # the small entries drop 20 bits of their p
    # small entry = n 2^(E - d - p): scaled by 2^(t - E) it is n 2^(t - d - p) = n 2^-20
    base = (1 << (p - 1))                                 # p-bit numerators with the top bit set
    half = 1 << 19                                        # the dropped 20 bits = 100...0
    nums = [base | half,                                  # kept part even, tie -> stays
            base | (1 << 20) | half,                      # kept part odd, tie -> up
            -(base | half),                               # negative ties
            -(base | (1 << 20) | half),
            base | half | 1,                              # just above the tie -> up
            base | (half - 1)]                            # just below -> down
    rows = []
    for n in nums:
        row = [(1, E - 1)] + [(n, E - d - p)] + [(0, 0)] * (K - 2)
        rows.append(row)
    return rows, t, d
