"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

Each test ties the oracle to something other than itself: values printed in
the paper (worked example, moduli table, modulus facts), library routines with
independent implementations (``round`` on ``Fraction``, ``float(Fraction)``,
mpmath), closed forms and invariants, and brute force on tiny inputs.
"""
import json
import math
import os
import random
from fractions import Fraction

import numpy as np
import pytest

import synth
from oracle import ozaki2_oracle as o

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _gold(name):
    with open(os.path.join(GOLD, name)) as fh:
        return json.load(fh)


# ---------------------------------------------------------------------------
# Worked example (Sec. 2.3)
# ---------------------------------------------------------------------------

def test_worked_example_residues_and_crt():
    g = _gold("worked_example.json")
    ms, a, b = g["moduli"], g["a"], g["b"]
    for m in ms:
        assert [o.cen(x, m) for x in a] == g["residues_a"][str(m)]
        assert [o.cen(x, m) for x in b] == g["residues_b"][str(m)]
        ip = sum(o.cen(x, m) * o.cen(y, m) for x, y in zip(a, b))
        assert ip == g["residue_inner_products"][str(m)]
    u = [g["residue_inner_products"][str(m)] % m for m in ms]
    assert u == g["reduced"]
    tab = o.CrtTables(ms)
    assert tab.P == g["P"] and tab.P // 2 == g["half_range"]
    assert o.crt_signed(u, tab) == g["result"] == sum(x * y for x, y in zip(a, b))


# ---------------------------------------------------------------------------
# Modulus set and the moduli table (Sec. 4.3)
# ---------------------------------------------------------------------------

def test_moduli_table_reproduced():
    g = _gold("moduli_table.json")
    K = g["K"]
    for row in g["rows"]:
        t = o.internal_width(row["p"], K)
        assert t == row["t"]
        ms = o.select_moduli(t, t, K)
        assert len(ms) == row["L"]
        assert o.gemm_count(ms) == row["gemms"]
        assert math.ceil(math.log2(o.product(ms))) == row["log2P"]


def test_moduli_table_rejects_ascending_order():
    """The descending reading is the one that reproduces the table: the
    ascending order would need more moduli at p = 53."""
    K, t = 4096, o.internal_width(53, 4096)
    asc = sorted(o.one_limb_moduli())
    P, n = 1, 0
    while P <= K << (2 * t + 2):
        P *= asc[n]
        n += 1
    assert n != _gold("moduli_table.json")["rows"][0]["L"]


def test_modulus_facts():
    g = _gold("modulus_facts.json")
    one = o.one_limb_moduli()
    assert len(one) == g["one_limb_count"]
    for i in range(len(one)):
        for j in range(i + 1, len(one)):
            assert math.gcd(one[i], one[j]) == 1
    lp = math.log2(o.product(one))
    assert round(lp, 1) == g["one_limb_log2_product"]
    assert round(math.log2(one[0]), 2) == g["top_bits"]
    assert round(lp / len(one), 2) == g["average_bits"]
    two = o.two_limb_moduli()
    assert round(math.log2(two[0]), 2) == g["two_limb_bits"]
    assert round(math.log2(two[0]) / 3, 2) == g["two_limb_bits_per_gemm"]
    # every two-limb modulus is coprime to every one-limb modulus and to each other
    P1 = o.product(one)
    for m in two[:200]:
        assert math.gcd(m, P1) == 1
    # balanced base-128 split keeps every plane in int8 (|r0| <= 64, |r1| <= 63)
    for m in (two[0], two[-1]):
        for r in range(-(m // 2), m // 2 + 1):
            r0, r1 = o.split128(r)
            assert abs(r0) <= 64 and abs(r1) <= 63 and abs(r0 + r1) <= 127


def test_int32_exactness_bound():
    """K * 127^2 < 2^31 holds exactly up to K = 133144 (the printed 133146 is
    two too high); the implementation cap 133000 is inside it."""
    assert 127 ** 2 * 133144 < 2 ** 31 <= 127 ** 2 * 133145
    assert o.K_CAP <= 133144


def test_select_moduli_is_shortest_prefix():
    for t, K in [(40, 1), (77, 256), (282, 1024), (600, 3000)]:
        ms = o.select_moduli(t, t, K)
        assert o.product(ms) > K * 2 ** (2 * t + 2)
        assert o.product(ms[:-1]) <= K * 2 ** (2 * t + 2)


# ---------------------------------------------------------------------------
# Rounding and integerization against independent library routines
# ---------------------------------------------------------------------------

def test_round_to_p53_matches_float():
    rng = random.Random(5)
    for _ in range(3000):
        num = rng.getrandbits(rng.randint(1, 200)) * rng.choice((-1, 1))
        scale = rng.randint(-300, 100)
        if num == 0:
            continue
        sg, S, e = o.round_to_p(num, scale, 53)
        got = (-1) ** sg * S * Fraction(2) ** (e - 53)
        ref = Fraction(float(Fraction(num) * Fraction(2) ** scale))
        assert got == ref


def test_round_to_p_matches_mpmath():
    mpmath = pytest.importorskip("mpmath")
    rng = random.Random(6)
    for p in (2, 8, 64, 113, 256, 512):
        for _ in range(300):
            num = rng.getrandbits(rng.randint(1, 3 * p + 10)) * rng.choice((-1, 1))
            if num == 0:
                continue
            scale = rng.randint(-200, 200)
            sg, S, e = o.round_to_p(num, scale, p)
            got = (-1) ** sg * S * Fraction(2) ** (e - p)
            with mpmath.workprec(p):
                x = mpmath.ldexp(mpmath.mpf(num, rounding="n"), scale)
                neg, man, ex, _ = x._mpf_
            assert got == (-1) ** neg * Fraction(int(man)) * Fraction(2) ** int(ex)
            assert 2 ** (p - 1) <= S < 2 ** p


def test_rne_shift_matches_round_fraction():
    rng = random.Random(7)
    for _ in range(5000):
        n = rng.randint(-10 ** 12, 10 ** 12)
        s = rng.randint(-45, 5)
        assert o.rne_shift(n, s) == round(Fraction(n) * Fraction(2) ** s)
    for n in (1, 3, 5, 7, -1, -3, -5, 6, -6):   # exact ties
        assert o.rne_shift(n, -1) == round(Fraction(n, 2))


def test_integerize_exact_when_spread_small():
    """With every exponent in a line within t - p of the line maximum the
    scaling loses nothing: a_hat * 2^(e - t) == a exactly (Sec. 4.2)."""
    rng = np.random.Generator(np.random.PCG64(11))
    p, K = 53, 64
    t = o.internal_width(p, K)
    A = synth.mp_matrix(rng, 3, K, p, -8, 8)
    for i in range(3):
        line, e = o.integer_line(A, i, 0, t)
        for k in range(K):
            assert Fraction(line[k]) * Fraction(2) ** (e - t) == o.value(A, i, k)
            assert abs(line[k]) <= 2 ** t


def test_integerize_matches_round_fraction_with_wide_spread():
    rng = np.random.Generator(np.random.PCG64(12))
    p, K = 64, 32
    t = o.internal_width(p, K)
    A = synth.mp_matrix(rng, 2, K, p, -80, 80)
    for i in range(2):
        line, e = o.integer_line(A, i, 0, t)
        assert e == max(int(x) for x in A["exp"][i])
        for k in range(K):
            ref = round(o.value(A, i, k) * Fraction(2) ** (t - e))
            assert line[k] == ref and abs(line[k]) <= 2 ** t


def test_mpfr_exponent_convention():
    for x in (Fraction(1), Fraction(3, 4), Fraction(1, 2), Fraction(-5), Fraction(1, 3)):
        e = o.mpfr_exp(x)
        assert Fraction(2) ** (e - 1) <= abs(x) < Fraction(2) ** e
    assert o.from_double(1.0) == (1 << 63, 1, 1)
    assert o.from_double(-0.75) == (-(3 << 62), 0, 1)


# ---------------------------------------------------------------------------
# CRT (Sec. 4.4): round trip sweep, alpha bound, signed range
# ---------------------------------------------------------------------------

def test_crt_roundtrip_sweep():
    """t = 40..1120 in steps of 8 (the paper's CRT sweep, Sec. 7.1): random
    exact integers |z| < P/2 survive residues -> direct CRT unchanged."""
    rng = random.Random(13)
    for t in range(40, 1121, 8):
        ms = o.select_moduli(t, t, 4096)
        tab = o.CrtTables(ms)
        half = tab.P // 2
        cases = [0, 1, -1, half, -(half - 1) if tab.P % 2 == 0 else -half, half - 1]
        cases += [rng.randint(-(half - 1), half) for _ in range(6)]
        for z in cases:
            u = [z % m for m in ms]
            assert o.crt_signed(u, tab) == z


def test_crt_alpha_bound_and_headroom():
    """alpha = floor(S / P) < L and S < L * P; a 32-bit digit count of
    ceil(bits(P)/32) + 2 always holds S (Sec. 5.4 digit headroom)."""
    rng = random.Random(14)
    ml = o.modulus_list()
    for L in range(2, 400, 7):
        ms = ml[:L]
        tab = o.CrtTables(ms)
        for _ in range(3):
            u = [rng.randrange(m) for m in ms]
            u_max = [m - 1 for m in ms]
            for uu in (u, u_max):
                v = [(x * inv) % m for x, inv, m in zip(uu, tab.Minv, ms)]
                S = sum(a * b for a, b in zip(v, tab.M))
                assert S // tab.P < L
                D = -(-tab.P.bit_length() // 32) + 2
                assert S < 2 ** (32 * D)
                _, alpha = o.crt_alpha_route(uu, tab)
                assert alpha == S // tab.P


def test_karatsuba_combine_identity():
    """Eq. 4: sum r^a r^b = P0 + 128 (Ps - P0 - P2) + 16384 P2 on split residues."""
    rng = random.Random(15)
    for m in (16189, 257, 8191):
        for _ in range(200):
            ra = [o.cen(rng.randrange(10 ** 9), m) for _ in range(20)]
            rb = [o.cen(rng.randrange(10 ** 9), m) for _ in range(20)]
            sa = [o.split128(x) for x in ra]
            sb = [o.split128(x) for x in rb]
            P0 = sum(x[0] * y[0] for x, y in zip(sa, sb))
            P2 = sum(x[1] * y[1] for x, y in zip(sa, sb))
            Ps = sum((x[0] + x[1]) * (y[0] + y[1]) for x, y in zip(sa, sb))
            assert P0 + 128 * (Ps - P0 - P2) + 16384 * P2 == sum(x * y for x, y in zip(ra, rb))


# ---------------------------------------------------------------------------
# Whole method vs the exact product (brute force on tiny inputs)
# ---------------------------------------------------------------------------

def _direct_chat(A, B, par, i, j):
    ai, _ = o.integer_line(A, i, 0, par.t)
    bj, _ = o.integer_line(B, j, 1, par.t)
    return sum(x * y for x, y in zip(ai, bj))


@pytest.mark.parametrize("p,spread", [(2, 0), (8, 0), (53, 0), (53, 40), (130, 3), (200, 300)])
def test_tiny_products_against_truth(p, spread):
    rng = np.random.Generator(np.random.PCG64(100 + p + spread))
    M, K, N = 3, 5, 4
    A = synth.mp_matrix(rng, M, K, p, -2 - spread, 2 + spread)
    B = synth.mp_matrix(rng, K, N, p, -2 - spread, 2 + spread)
    A = synth.zero_rows(A, [1]) if spread == 40 else A
    res = o.ozaki2_full(A, B, p)
    par = res["par"]
    T = o.truth_full(A, B, p)
    for i in range(M):
        for j in range(N):
            # invariants: u_l == chat_direct mod m_l and CRT(u) == chat_direct
            cd = _direct_chat(A, B, par, i, j)
            assert [int(x) for x in res["u"][:, i, j]] == [cd % m for m in par.moduli]
            assert res["chat"][i, j] == cd
            # exact product (independent: Fractions summed directly)
            ex = sum(o.value(A, i, k) * o.value(B, k, j) for k in range(K))
            ref = o.to_fraction(*o.matrix_entry(T, i, j))
            got = o.to_fraction(*o.matrix_entry(res["C"], i, j))
            if ex == 0:
                assert ref == 0 and got == 0
                continue
            assert o.ulp_distance(ref, ex, p) <= Fraction(1, 2)
            # closed-form bound: each scaled input is off by at most 1/2, so
            # |chat 2^(e+f-2t) - exact| <= K 2^(e+f-t) (1 + 2^-t); the final
            # rounding adds at most half an ulp of the result
            e_i, f_j = int(res["e"][i]), int(res["f"][j])
            quant = K * Fraction(2) ** (e_i + f_j - par.t) * (1 + Fraction(1, 2 ** par.t))
            half_ulp = Fraction(2) ** (o.mpfr_exp(got) - p - 1) if got else 0
            assert abs(got - ex) <= quant + half_ulp
            if spread <= par.t - p:
                assert got == ref            # no quantisation loss -> 0 ulp


def test_entries_match_full():
    rng = np.random.Generator(np.random.PCG64(21))
    A = synth.mp_matrix(rng, 6, 7, 100, -5, 5)
    B = synth.mp_matrix(rng, 7, 5, 100, -5, 5)
    full = o.ozaki2_full(A, B, 100)
    pairs = [(0, 0), (5, 4), (2, 3)]
    ent = o.ozaki2_entries(A, B, 100, pairs)
    for (i, j), e in zip(pairs, ent):
        assert e["chat"] == full["chat"][i, j]
        assert e["u"] == [int(x) for x in full["u"][:, i, j]]
        assert (e["limbs"], e["exp"], e["sign"]) == o.matrix_entry(full["C"], i, j)


def test_truth_entry_matches_truth_full():
    rng = np.random.Generator(np.random.PCG64(22))
    A = synth.mp_matrix(rng, 4, 9, 70, -30, 30)
    B = synth.mp_matrix(rng, 9, 3, 70, -30, 30)
    T = o.truth_full(A, B, 70)
    for i in range(4):
        for j in range(3):
            assert o.truth_entry(A, B, i, j, 70) == o.matrix_entry(T, i, j)


def test_fp64_mode_truth_is_correctly_rounded_double():
    rng = np.random.Generator(np.random.PCG64(23))
    X = synth.fp64_matrix(rng, 3, 6)
    Y = synth.fp64_matrix(rng, 6, 2)
    A, B = o.fp64_as_mat(X), o.fp64_as_mat(Y)
    T = o.truth_full(A, B, 53)
    for i in range(3):
        for j in range(2):
            ex = sum(Fraction(float(X[i, k])) * Fraction(float(Y[k, j])) for k in range(6))
            assert o.to_double(*o.matrix_entry(T, i, j)) == float(ex)


def test_accuracy_level_on_random_matrix():
    """The method's error stays under 1 ulp (the paper reports <= 0.95 ulp)."""
    g = _gold("modulus_facts.json")
    rng = np.random.Generator(np.random.PCG64(24))
    p = 113
    # exponent spread 30 > t - p = 22 so the scaling does round
    A = synth.mp_matrix(rng, 4, 40, p, -15, 15)
    B = synth.mp_matrix(rng, 40, 4, p, -15, 15)
    res = o.ozaki2_full(A, B, p)
    worst = Fraction(0)
    for i in range(4):
        for j in range(4):
            ex = sum(o.value(A, i, k) * o.value(B, k, j) for k in range(40))
            got = o.to_fraction(*o.matrix_entry(res["C"], i, j))
            worst = max(worst, o.ulp_distance(got, ex, p))
    assert worst < 1 and g["max_ulp_printed"] < 1
