"""Pins of the oracle's binary64 mode (forward and the backward reading).

The binary64 functions of the oracle (``f64_exponents``, ``dgemm_fwd_entry``,
``dgemm_dA_entry``, ``dgemm_dB_entry``) are checked here against results that
do not come from the oracle's own arithmetic:

* ``f64_exponents`` against ``math.frexp`` element by element (the MPFR
  exponent of x is the e of x = m 2^e, |m| in [0.5, 1));
* every entry against the exact rational inner product rounded once to
  binary64 (``float(Fraction)`` is correctly rounded): equal when every
  line's spread is at most t - 53 (then the shared-exponent integerization of
  Sec. 4.2 drops no bit and the method is exact), and within the closed-form
  quantisation bound of Eq. 1 on wide exponent spreads;
* the backward entries against the exact central difference of the bilinear
  loss <G, A B> (exact for any step h), for A and for B;
* lines of very different magnitude, which fail if an operand is
  integerized along the wrong axis (per column where the reading takes rows,
  or the reverse) or scaled by the wrong side's exponents.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

from oracle import ozaki2_oracle as o


def _bounded(rng, rows, cols, lo, hi):
    """Entries +-(1 + u) 2^k, u uniform in [0, 1), k uniform integer in [lo, hi]."""
    sig = 1.0 + rng.random(size=(rows, cols))
    k = rng.integers(lo, hi, size=(rows, cols), endpoint=True)
    sgn = np.where(rng.random(size=(rows, cols)) < 0.5, -1.0, 1.0)
    return sgn * np.ldexp(sig, k)


def _wide(rng, rows, cols):
    """The differentiation workload's recipe: normal(0, 1) 2^u, u in [-20, 20]."""
    return np.ldexp(rng.standard_normal(size=(rows, cols)),
                    rng.integers(-20, 20, size=(rows, cols), endpoint=True))


def _exact(xs, ys) -> Fraction:
    return sum((Fraction(float(a)) * Fraction(float(b)) for a, b in zip(xs, ys)), Fraction(0))


def _ulps(x: float, ref: Fraction) -> Fraction:
    return o.ulp_distance(Fraction(x), Fraction(float(ref)), 53) if ref else Fraction(abs(x))


def _fd(X, Y, G, side, r, c) -> Fraction:
    """Exact central difference of <G, X Y> in X[r, c] (side 'A') or Y[r, c]."""
    h = Fraction(1, 7)

    def shifted(delta):
        Xf = np.array([[Fraction(float(v)) for v in row] for row in X], dtype=object)
        Yf = np.array([[Fraction(float(v)) for v in row] for row in Y], dtype=object)
        (Xf if side == "A" else Yf)[r, c] += delta
        Gf = np.array([[Fraction(float(v)) for v in row] for row in G], dtype=object)
        return (Gf * Xf.dot(Yf)).sum()

    return (shifted(h) - shifted(-h)) / (2 * h)


def test_f64_exponents_against_frexp_with_zero_lines():
    rng = np.random.Generator(np.random.PCG64(71))
    X = _wide(rng, 5, 7)
    X[2, :] = 0.0
    X[:, 4] = 0.0
    X[0, 1] = -0.0
    for axis in (0, 1):
        got = o.f64_exponents(X, axis)
        n = X.shape[1 - axis]
        assert len(got) == n
        for line in range(n):
            vals = X[line, :] if axis == 1 else X[:, line]
            exps = [math.frexp(float(v))[1] for v in vals if v != 0.0]
            assert got[line] == (max(exps) if exps else None)
    # the exponent of x: 2^(e-1) <= |x| < 2^e
    for v in (1.0, 0.75, 2.0 ** -30, -3.0, 2.0 ** 40 - 1.0):
        e = o.f64_exponents(np.array([[v]]), 1)[0]
        assert 2.0 ** (e - 1) <= abs(v) < 2.0 ** e


@pytest.mark.parametrize("M,N,K,seed", [(5, 6, 7, 72), (3, 4, 40, 73)])
def test_entries_exact_when_spread_within_t_minus_53(M, N, K, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    X = _bounded(rng, M, K, -2, 2)
    Y = _bounded(rng, K, N, -2, 2)
    G = _bounded(rng, M, N, -2, 2)
    par = o.dgemm_params(M, N, K)
    assert par.t - 53 >= 16          # every line below spreads by at most 5 + 2 + 2 bits
    e, f = o.f64_exponents(X, 1), o.f64_exponents(Y, 0)
    for i in range(M):
        for j in range(N):
            assert o.dgemm_fwd_entry(X, Y, i, j, par, e, f) == float(_exact(X[i, :], Y[:, j]))
    for i in range(M):
        for k in range(K):
            assert o.dgemm_dA_entry(Y, G, i, k, par, f) == float(_exact(G[i, :], Y[k, :]))
    for k in range(K):
        for j in range(N):
            assert o.dgemm_dB_entry(X, G, k, j, par, e) == float(_exact(X[:, k], G[:, j]))


def _bound(inner: int, scale: int, t: int, got: float) -> Fraction:
    """Closed-form error bound of the method on one entry: every scaled input
    is off by at most 1/2 (Eq. 1), so the scaled sum is within
    inner 2^(scale - t) (1 + 2^-t) of the exact one, where scale is the sum of
    the two lines' shared exponents; the final rounding adds half an ulp."""
    half = Fraction(2) ** (math.frexp(got)[1] - 54) if got else Fraction(0)
    return inner * Fraction(2) ** (scale - t) * (1 + Fraction(1, 2 ** t)) + half


def _line_exp(vals) -> int | None:
    exps = [math.frexp(float(v))[1] for v in vals if v != 0.0]
    return max(exps) if exps else None


def test_entries_within_quantisation_bound_on_wide_spreads():
    """Spreads beyond t - 53 drop low bits of small entries (the paper's
    documented limit): each entry stays within the closed-form bound."""
    rng = np.random.Generator(np.random.PCG64(74))
    M, N, K = 5, 6, 7
    X, Y, G = _wide(rng, M, K), _wide(rng, K, N), rng.standard_normal(size=(M, N))
    X[3, :] = 0.0                    # a zero row of A
    Y[:, 2] = 0.0                    # a zero column of B
    par = o.dgemm_params(M, N, K)
    t = par.t
    e, f = o.f64_exponents(X, 1), o.f64_exponents(Y, 0)
    for i in range(M):
        for j in range(N):
            ref = _exact(X[i, :], Y[:, j])
            got = o.dgemm_fwd_entry(X, Y, i, j, par, e, f)
            if i == 3 or j == 2:
                assert got == 0.0
                continue
            assert abs(Fraction(got) - ref) <= _bound(K, _line_exp(X[i, :]) + _line_exp(Y[:, j]), t, got)
    for i in range(M):
        for k in range(K):
            ref = _exact(G[i, :], Y[k, :])
            got = o.dgemm_dA_entry(Y, G, i, k, par, f)
            # the row of dC 2^f_j that is integerized, and its shared exponent
            g_i = _line_exp([G[i, j] * 2.0 ** f[j] for j in range(N) if f[j] is not None])
            assert abs(Fraction(got) - ref) <= _bound(N, g_i, t, got)
    for k in range(K):
        for j in range(N):
            ref = _exact(X[:, k], G[:, j])
            got = o.dgemm_dB_entry(X, G, k, j, par, e)
            h_j = _line_exp([G[i, j] * 2.0 ** e[i] for i in range(M) if e[i] is not None])
            assert abs(Fraction(got) - ref) <= _bound(M, h_j, t, got)


def test_backward_entries_against_exact_central_difference():
    """Spreads within t - 53 (the backward is then exact): each gradient entry
    equals the exact central difference of <G, A B>, rounded once."""
    rng = np.random.Generator(np.random.PCG64(75))
    M, N, K = 5, 6, 7
    X, Y, G = _bounded(rng, M, K, -3, 3), _bounded(rng, K, N, -3, 3), _bounded(rng, M, N, -3, 3)
    par = o.dgemm_params(M, N, K)
    e, f = o.f64_exponents(X, 1), o.f64_exponents(Y, 0)
    for (i, k) in ((0, 0), (2, 5), (4, 6)):
        assert o.dgemm_dA_entry(Y, G, i, k, par, f) == float(_fd(X, Y, G, "A", i, k))
    for (k, j) in ((0, 0), (3, 2), (6, 5)):
        assert o.dgemm_dB_entry(X, G, k, j, par, e) == float(_fd(X, Y, G, "B", k, j))


def test_lines_of_very_different_magnitude():
    """A tiny line next to a huge one: integerizing along the wrong axis
    (one shared exponent for both lines) would round the tiny line to zero;
    scaling by the other side's exponents would be off by powers of two."""
    rng = np.random.Generator(np.random.PCG64(76))
    M, N, K = 3, 4, 5
    X = _bounded(rng, M, K, -1, 1)
    X[0, :] *= 2.0 ** -60            # tiny row of A
    X[1, :] *= 2.0 ** 60             # huge row of A
    Y = _bounded(rng, K, N, -1, 1)
    Y[:, 0] *= 2.0 ** -60            # tiny column of B
    Y[:, 1] *= 2.0 ** 60             # huge column of B
    G = _bounded(rng, M, N, -1, 1)
    G[0, :] *= 2.0 ** -70            # tiny row and huge row of dC (dA reads rows)
    G[1, :] *= 2.0 ** 70
    G2 = _bounded(rng, M, N, -1, 1)
    G2[:, 0] *= 2.0 ** -70           # tiny column and huge column of dC (dB reads columns)
    G2[:, 1] *= 2.0 ** 70
    par = o.dgemm_params(M, N, K)
    e, f = o.f64_exponents(X, 1), o.f64_exponents(Y, 0)
    for i in range(M):
        for j in range(N):
            assert o.dgemm_fwd_entry(X, Y, i, j, par, e, f) == float(_exact(X[i, :], Y[:, j]))
    for i in range(M):
        for k in range(K):
            ref = _exact(G[i, :], Y[k, :])
            assert _ulps(o.dgemm_dA_entry(Y, G, i, k, par, f), ref) <= 1
    for k in range(K):
        for j in range(N):
            ref = _exact(X[:, k], G2[:, j])
            assert _ulps(o.dgemm_dB_entry(X, G2, k, j, par, e), ref) <= 1


def test_a_planted_axis_slip_is_caught():
    """The lines test above detects the slip it is meant for: integerizing the
    dA operand per column of dC (shared over rows) loses the tiny row."""
    rng = np.random.Generator(np.random.PCG64(77))
    M, N, K = 3, 4, 5
    Y = _bounded(rng, K, N, -1, 1)
    G = _bounded(rng, M, N, -1, 1)
    G[0, :] *= 2.0 ** -70
    G[1, :] *= 2.0 ** 70
    par = o.dgemm_params(M, N, K)
    f = o.f64_exponents(Y, 0)

    def dA_per_column(i, k):
        # the slip: one shared exponent per column j of dC 2^f (over all rows)
        col_exp = [max(o.from_double(float(G[r, j]))[1] + f[j] for r in range(M)) for j in range(N)]
        g = max(col_exp)
        drow = [o._f64_int(float(G[i, j]), f[j], g, par.t) for j in range(N)]
        brow = [o._f64_int(float(Y[k, j]), 0, f[j], par.t) for j in range(N)]
        return o._round_double(o.entry(drow, g, brow, 0, par)["chat"], g - 2 * par.t)

    ref = _exact(G[0, :], Y[1, :])
    assert _ulps(o.dgemm_dA_entry(Y, G, 0, 1, par, f), ref) <= 1
    assert _ulps(dA_per_column(0, 1), ref) > 1
