"""The arithmetic behind the fast form of the long CRT finish, on the CPU.

The finish rebuilds R = (sum_g Q_g 2^(224 g) + alpha~ (2^(32 D) - P)) mod
2^(32 D) digit by digit from the group words (9 words per group of 32 column
sums, group g starting at digit 7 g).  Its fast form starts at digit
d0 = 7 g0 with no carry in and uses only the digits from d0 on; the kernel
relies on two facts checked here with exact integers:

1. the carry it leaves out is at most alpha~ + 2, whatever the words
   (every digit step adds at most two words and alpha~ times a digit);
2. where every digit-d0 quantity it uses (R's digit, R - P's, the sums of
   the comparisons, the range check and P - x0) lies at least alpha~ + 5 from
   both ends of its range, its decisions (R >= P, the sign, the range check)
   and every digit of |c_hat| above d0 equal those of the full R.

P is the product of the method's moduli at p = 2048 (Sec. 4.3).  For the
bound the words are any 32-bit values (all ones in a third of the trials) and
alpha~ any value up to L; for the decisions they hold a random S < L P (its
digits, part of each group's words 0 and 1 moved into words 7 and 8 of the
group before) with alpha~ = floor(S / P) or one less, so that R lies in
[0, 2P) as in the method, and half the trials put digit d0 next to a wrap.
"""
import random

from oracle import ozaki2_oracle as o

M32 = (1 << 32) - 1


def _digits_from(words, alpha, negP, D, gs):
    """Digits d >= 7 gs of R as the kernel forms them from group gs on, with
    no carry in (words 7 and 8 of group gs - 1 enter digits 7 gs and 7 gs + 1)."""
    carry = 0
    prev7, prev8 = (words[gs - 1][7], words[gs - 1][8]) if gs > 0 else (0, 0)
    out = {}
    g = gs
    while 7 * g < D:
        w = words[g] if g < len(words) else [0] * 9
        for k in range(7):
            d = 7 * g + k
            x = carry + alpha * (negP[d] if d < D else M32) + w[k]
            if k == 0:
                x += prev7
            if k == 1:
                x += prev8
            carry = x >> 32
            out[d] = x & M32 if d < D else 0
        prev7, prev8 = w[7], w[8]
        g += 1
    return out


def _num(digs, lo, hi):
    return sum(digs.get(d, 0) << (32 * (d - lo)) for d in range(lo, hi))


def _setup():
    par = o.Params(64, 2048)
    P = o.product(par.moduli)
    D = (P.bit_length() + 31) // 32 + 2
    ng = -(-D // 7) + 1
    DG = 7 * (-(-D // 7))
    negP_full = (1 << (32 * D)) - P
    negP = [(negP_full >> (32 * d)) & M32 for d in range(D)]
    return par, P, D, ng, DG, negP


def _valid_words(rng, P, L, ng):
    """Group words of a random S < L P as the sums kernel could leave them:
    the digits of S, with part of words 0 and 1 of every group moved into
    words 7 and 8 of the group before (the same digit positions)."""
    S = rng.randrange(L * P)
    words = [[(S >> (32 * (7 * g + k))) & M32 for k in range(7)] + [0, 0] for g in range(ng)]
    for g in range(1, ng):
        for k, kk in ((0, 7), (1, 8)):
            v = rng.randrange(words[g][k] + 1)
            words[g][k] -= v
            words[g - 1][kk] += v
    return words


def _words_sum(words):
    return sum(sum(w[k] << (32 * k) for k in range(9)) << (224 * g) for g, w in enumerate(words))


def _exact(words, alpha, P, D):
    S = _words_sum(words)
    R = (S + alpha * ((1 << (32 * D)) - P)) % (1 << (32 * D))
    ge = R >= P
    x0 = R - P if ge else R
    neg = x0 > P // 2
    mag = P - x0 if neg else x0
    return R, ge, neg, x0 >= P, mag


def _fast(digs, alpha, P, D, DG, d0):
    """The fast form's decisions and digits above d0, and whether every
    digit-d0 quantity it uses is safe."""
    n = DG - d0
    mod = 1 << (32 * n)
    wide = lambda x: (x >> (32 * d0)) | (((1 << (32 * DG)) - (1 << (32 * D))) >> (32 * d0))  # ones above D
    negP = wide((1 << (32 * D)) - P)
    negH1 = wide((1 << (32 * D)) - (P // 2 + 1))
    Pup = P >> (32 * d0)
    U = alpha + 5
    safe = lambda v: U <= (v & M32) <= M32 - U
    r = _num(digs, d0, DG)
    t1 = r + negP
    ge = t1 >= mod
    t1 %= mod
    c3 = r + negH1 >= mod
    c4 = t1 + negH1 >= mod
    neg = c4 if ge else c3
    x0 = t1 if ge else r
    bad = x0 + negP >= mod
    pm = (Pup - x0) % mod
    mag = pm if neg else x0
    ok = all(safe(v) for v in (r, t1, r + (negH1 & M32), t1 + (negH1 & M32), x0, x0 + (negP & M32),
                               (Pup & M32) - (x0 & M32)))
    return ok, ge, neg, bad, mag


def test_left_out_carry_is_at_most_alpha_plus_two():
    par, P, D, ng, DG, negP = _setup()
    rng = random.Random(2061)
    g0 = 9
    d0 = 7 * g0
    for trial in range(300):
        alpha = rng.randrange(par.L + 1)
        words = [[rng.getrandbits(32) if trial % 3 else M32 for _ in range(9)] for _ in range(ng)]
        full = _digits_from(words, alpha, negP, D, 0)
        up = _digits_from(words, alpha, negP, D, g0)
        c = (_num(full, d0, D) - _num(up, d0, D)) % (1 << (32 * (D - d0)))
        assert 0 <= c <= alpha + 2
        R = _exact(words, alpha, P, D)[0]
        assert _num(full, 0, D) == R                       # the digit-serial form is R itself


def test_fast_form_decisions_and_digits_when_safe():
    par, P, D, ng, DG, negP = _setup()
    rng = random.Random(2062)
    d0 = 7 * 9
    seen_safe = seen_unsafe = 0
    for trial in range(400):
        words = _valid_words(rng, P, par.L, ng)
        b = rng.randrange(2)                             # alpha~ = alpha or alpha - 1
        alpha = max(_words_sum(words) // P - b, 0)
        if trial % 2:
            # push digit d0 next to a wrap: choose word 0 of group 9 so that
            # the digit the fast form sees is 2^32 - delta, delta on either
            # side of the margin alpha~ + 5
            up = _digits_from(words, alpha, negP, D, 9)
            words[9][0] = (words[9][0] - up[d0] - rng.randrange(1, 2 * (alpha + 5))) & M32
            alpha = max(_words_sum(words) // P - b, 0)
        R, ge, neg, bad, mag = _exact(words, alpha, P, D)
        assert R < 2 * P and not bad                     # R = S - alpha~ P in [0, 2P)
        up = _digits_from(words, alpha, negP, D, 9)
        ok, fge, fneg, fbad, fmag = _fast(up, alpha, P, D, DG, d0)
        if not ok:
            seen_unsafe += 1
            continue
        seen_safe += 1
        assert (fge, fneg, fbad) == (ge, neg, bad)
        assert fmag >> 32 == mag >> (32 * (d0 + 1))        # every digit of |c_hat| above d0
    assert seen_safe > 150 and seen_unsafe > 60
