"""Pins of the oracle's complex product (3M in the residue domain).

Against results that do not come from the 3M combination: the CRT integers
equal the direct integer sums ar br - ai bi and ar bi + ai br of the jointly
scaled integers (the 4M formulas); the outputs equal the exact complex product
rounded once per part when every joint line spreads within t - p, and lie
within the closed-form quantisation bound otherwise; a purely real product
reduces to the real one; and a planted sign slip in the imaginary
combination is caught."""
import math
from fractions import Fraction

import numpy as np
import pytest

import synth
from oracle import ozaki2_oracle as o


def _mats(seed, M, K, N, p, lo, hi, zero_imag=False):
    rng = np.random.Generator(np.random.PCG64(seed))
    Ar = synth.mp_matrix(rng, M, K, p, lo, hi)
    Ai = synth.mp_matrix(rng, M, K, p, lo, hi, zero_frac=1.0 if zero_imag else 0.0)
    Br = synth.mp_matrix(rng, K, N, p, lo, hi)
    Bi = synth.mp_matrix(rng, K, N, p, lo, hi, zero_frac=1.0 if zero_imag else 0.0)
    return Ar, Ai, Br, Bi


@pytest.mark.parametrize("p", [8, 53, 200])
def test_crt_integers_equal_the_direct_complex_sums(p):
    M, K, N = 3, 5, 4
    Ar, Ai, Br, Bi = _mats(90 + p, M, K, N, p, -3, 3)
    par = o.complex_params(K, p)
    assert par.t == p + 16 + math.ceil(math.log2(2 * K))
    res = o.complex_full(Ar, Ai, Br, Bi, p)
    for i in range(M):
        (ar, ai), e = o.joint_lines([Ar, Ai], i, 0, par.t)
        for j in range(N):
            (br, bi), f = o.joint_lines([Br, Bi], j, 1, par.t)
            re = sum(a * b - c * d for a, b, c, d in zip(ar, br, ai, bi))
            im = sum(a * d + c * b for a, b, c, d in zip(ar, br, ai, bi))
            assert res["chat_r"][i, j] == re and res["chat_i"][i, j] == im
            assert [int(x) for x in res["u_r"][:, i, j]] == [re % m for m in par.moduli]
            assert [int(x) for x in res["u_i"][:, i, j]] == [im % m for m in par.moduli]


@pytest.mark.parametrize("p,spread", [(53, 0), (113, 0), (53, 40)])
def test_outputs_against_the_exact_complex_product(p, spread):
    M, K, N = 3, 4, 3
    Ar, Ai, Br, Bi = _mats(95 + p + spread, M, K, N, p, -2 - spread, 2 + spread)
    res = o.complex_full(Ar, Ai, Br, Bi, p)
    par = res["par"]
    for i in range(M):
        e = o.joint_exponent([Ar, Ai], i, 0)
        for j in range(N):
            f = o.joint_exponent([Br, Bi], j, 1)
            truth = o.complex_truth_entry(Ar, Ai, Br, Bi, i, j, p)
            exact = [sum(o.value(Ar, i, k) * o.value(Br, k, j) - o.value(Ai, i, k) * o.value(Bi, k, j)
                         for k in range(K)),
                     sum(o.value(Ar, i, k) * o.value(Bi, k, j) + o.value(Ai, i, k) * o.value(Br, k, j)
                         for k in range(K))]
            for part, tr, ex in zip(("Cr", "Ci"), truth, exact):
                got = o.to_fraction(*o.matrix_entry(res[part], i, j))
                if spread <= par.t - p:
                    assert got == o.to_fraction(*tr)          # no quantisation loss: 0 ulp
                else:
                    # each of the 4 K scaled products off by at most 2^(e+f-t)(1 + 2^-t) in total per pair
                    half = Fraction(2) ** (o.mpfr_exp(got) - p - 1) if got else 0
                    bound = 2 * K * Fraction(2) ** (e + f - par.t) * (1 + Fraction(1, 2 ** par.t)) + half
                    assert abs(got - ex) <= bound


def test_real_inputs_reduce_to_the_real_product():
    p, M, K, N = 53, 3, 6, 4
    Ar, Ai, Br, Bi = _mats(97, M, K, N, p, -2, 2, zero_imag=True)
    res = o.complex_full(Ar, Ai, Br, Bi, p)
    T = o.truth_full(Ar, Br, p)
    for i in range(M):
        for j in range(N):
            assert o.matrix_entry(res["Cr"], i, j) == o.matrix_entry(T, i, j)
            assert o.to_fraction(*o.matrix_entry(res["Ci"], i, j)) == 0


def test_a_planted_sign_slip_is_caught():
    """u_i = T3 - T1 + T2 (a sign slip) does not reproduce ar bi + ai br."""
    p, K = 53, 4
    Ar, Ai, Br, Bi = _mats(98, 1, K, 1, p, -2, 2)
    par = o.complex_params(K, p)
    (ar, ai), e = o.joint_lines([Ar, Ai], 0, 0, par.t)
    (br, bi), f = o.joint_lines([Br, Bi], 0, 1, par.t)
    ent = o.complex_entry(ar, ai, e, br, bi, f, par)
    im = sum(a * d + c * b for a, b, c, d in zip(ar, br, ai, bi))
    assert ent["chat_i"] == im
    u1, u2, u3 = (o.reduce_planes(T, par.moduli) for T in (ent["T1"], ent["T2"], ent["T3"]))
    slip = [(c - a + b) % m for a, b, c, m in zip(u1, u2, u3, par.moduli)]
    assert o.crt_signed(slip, par.tab) != im
