"""Oracle pins on constructed round-half-even ties (CPU).

Integerization (Eq. 1): entries whose dropped bits are exactly half a step
of the scaled integer, with even and odd kept bits and entries just off the
tie, against Python's round(Fraction), which rounds half to even.  Final
rounding to p bits (Sec. 4.1, stage 5): products whose exact value is a tie
at p bits (or just off one, or rounds up with a carry into a new bit), against
values fixed by hand; the method's stage-by-stage result (O) and the
correctly rounded exact product (T) both give them."""
from fractions import Fraction

import numpy as np
import pytest

from oracle import ozaki2_oracle as o
from ties_cases import final_rounding_ties, integerization_ties, mat_from_values


@pytest.mark.parametrize("p", [53, 113, 256])
def test_integerization_ties_round_half_even(p):
    K = 3
    rows, t, d = integerization_ties(p, K)
    A = mat_from_values(rows, p)
    for r, row in enumerate(rows):
        ints, e = o.integer_line(A, r, 0, t)
        assert e == 0
        n, pw = row[1]
        want = round(Fraction(n) * Fraction(2) ** (pw + t - e))     # round half to even
        assert ints[1] == want
        # the construction: half a step dropped exactly, or just off it
        frac = Fraction(n) * Fraction(2) ** (pw + t) - int(Fraction(n) * Fraction(2) ** (pw + t))
        assert abs(frac) in (Fraction(1, 2),) or r >= 4
    kept = [o.integer_line(A, r, 0, t)[0][1] for r in range(len(rows))]
    # even kept part stays, odd kept part goes up (away from zero for negative entries)
    assert kept[0] % 2 == 0 and kept[1] % 2 == 0 and kept[0] > 0 and kept[1] > 0
    assert kept[2] == -kept[0] and kept[3] == -kept[1]


@pytest.mark.parametrize("p", [53, 256])
def test_final_rounding_ties_by_hand(p):
    cases = final_rounding_ties(p)
    A = mat_from_values([c[0] for c in cases], p)
    B = mat_from_values([[(1, 0)] for _ in range(3)], p)
    res = o.ozaki2_full(A, B, p)
    T = o.truth_full(A, B, p)
    for i, (_, want) in enumerate(cases):
        want_v = Fraction(want, 1 << 10)
        got = o.to_fraction(*o.matrix_entry(res["C"], i, 0))
        tru = o.to_fraction(*o.matrix_entry(T, i, 0))
        assert got == want_v, i
        assert tru == want_v, i
