"""Ozaki scheme II oracle -- TEST INFRASTRUCTURE ONLY.

A plain, slow, exact CPU restatement of the multiple-precision GEMM of
"Ozaki Scheme II Is Fast on CPUs Too" (Kouya, 2026).  It is not part of the
product: only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU
baseline may import it.  It shares no code with the CUDA path and imports
nothing from the product package.

Two results are provided:

(T) ``truth_*``: the exact inner product sum_k a_ik b_kj of the dyadic inputs,
    computed with Python integers and rounded once to p bits (round to nearest,
    ties to even).  This is the definition of the correctly rounded product.

(O) ``stage_*`` / ``ozaki2_*``: the method step by step in the paper's order
    (Sec. 4.1 five-stage flow):
    1. shared-exponent integerization  (Sec. 4.2, Eq. 1-3)
    2. centered residues per modulus    (Sec. 2.3, Sec. 4.3 incl. the
                                          balanced base-128 split, Eq. 4-5)
    3. exact per-plane integer products (Sec. 2.4, Sec. 4.3)
    4. mod-reduction + Karatsuba combine (Eq. 4)
    5. direct CRT                       (Sec. 4.4)
    6. rescale and round to p bits      (Sec. 4.1 stage 5)
    Every intermediate is an integer, so a correct GPU path matches (O)
    bit for bit.

Readings of the paper where it is silent or loose (listed again in the design
notes): moduli are taken in descending order within each set; the CRT margin
is the implementation's "+2" (Sec. 4.3); ``round`` in Eq. 1 is round-half-even;
centered residues lie in (-m/2, m/2] (ties for even m go to +m/2); the final
rounding is round-half-even; two-limb moduli are the primes in (255, 16191].

Matrix format: see ``synth`` (limb planes [nl, R, C], exp [R, C], sign [R, C];
value = (-1)^sign * sig * 2^(exp - 64 nl)).

Every function is parity-pinned: the multiple-precision path by
``tests/test_oracle_pins.py``, the binary64 mode by
``tests/test_oracle_fp64_pins.py``.
"""
from __future__ import annotations

import math
from fractions import Fraction

import numpy as np

GUARD_BITS = 16          # g, Sec. 4.2 (default 16)
TWO_LIMB_MAX = 16191     # largest two-limb modulus bound, Sec. 4.3
ONE_LIMB_MAX = 255       # int8 centered residues, Sec. 2.4 / Sec. 4.3(a)
K_CAP = 133000           # implementation cap on K, Sec. 4.3(a) and Sec. 10


# ---------------------------------------------------------------------------
# Parameters: t and the modulus set (Sec. 4.2 Eq. 3, Sec. 4.3, Table "moduli")
# ---------------------------------------------------------------------------

def ceil_log2(k: int) -> int:
    """ceil(log2 k) for k >= 1 (0 for k = 1)."""
    assert k >= 1
    return (k - 1).bit_length()


def internal_width(p: int, K: int, g: int = GUARD_BITS) -> int:
    """t = p + g + ceil(log2 K)   (Sec. 4.2, Eq. 3)."""
    return p + g + ceil_log2(K)


def _is_prime(n: int) -> bool:
    if n < 2:
        return False
    d = 2
    while d * d <= n:
        if n % d == 0:
            return False
        d += 1
    return True


def one_limb_moduli() -> list[int]:
    """The pairwise-coprime moduli m <= 255 whose centered residues fit int8:
    for every prime q <= 255 the largest power q^k <= 255 (the 54 prime powers
    of Sec. 4.3(a)), in descending order."""
    out = []
    for q in range(2, ONE_LIMB_MAX + 1):
        if _is_prime(q):
            m = q
            while m * q <= ONE_LIMB_MAX:
                m *= q
            out.append(m)
    return sorted(out, reverse=True)


def two_limb_moduli() -> list[int]:
    """Moduli 255 < m <= 16191 added after the one-limb set; pairwise
    coprimality with the full prime-power set forces primes (Sec. 4.3(a)).
    Descending order."""
    return [m for m in range(TWO_LIMB_MAX, ONE_LIMB_MAX, -1) if _is_prime(m)]


def modulus_list() -> list[int]:
    """All one-limb moduli first, then two-limb ones (Sec. 4.3: the hybrid
    uses up all one-limb moduli before adding two-limb ones)."""
    return one_limb_moduli() + two_limb_moduli()


def select_moduli(bits_a: int, bits_b: int, inner: int) -> list[int]:
    """Shortest prefix of ``modulus_list()`` with
    log2 P > bits_a + bits_b + log2(inner) + 2, i.e. P > inner * 2^(bits_a+bits_b+2)
    (Sec. 4.3 Eq. crtcond with the implementation's +2 margin; for the forward
    product bits_a = bits_b = t and inner = K)."""
    bound = inner << (bits_a + bits_b + 2)
    P = 1
    chosen = []
    for m in modulus_list():
        chosen.append(m)
        P *= m
        if P > bound:
            return chosen
    raise ValueError("modulus table exhausted")


def gemm_count(moduli: list[int]) -> int:
    """Number of int8 GEMMs: one per one-limb modulus, three (Karatsuba) per
    two-limb modulus (Sec. 4.3, Eq. 4-5)."""
    return sum(1 if m <= ONE_LIMB_MAX else 3 for m in moduli)


def product(ms) -> int:
    P = 1
    for m in ms:
        P *= m
    return P


# ---------------------------------------------------------------------------
# Decoding the storage format
# ---------------------------------------------------------------------------

def decode(mat: dict, r: int, c: int) -> tuple[int, int, int]:
    """(signed significand, exp, nl): value = ssig * 2^(exp - 64 nl)."""
    limbs = mat["limbs"]
    nl = limbs.shape[0]
    sig = 0
    for q in range(nl):
        sig |= int(limbs[q, r, c]) << (64 * q)
    if sig == 0:
        return 0, 0, nl
    s = -1 if int(mat["sign"][r, c]) else 1
    return s * sig, int(mat["exp"][r, c]), nl


def value(mat: dict, r: int, c: int) -> Fraction:
    ssig, e, nl = decode(mat, r, c)
    return Fraction(ssig) * Fraction(2) ** (e - 64 * nl)


def mpfr_exp(x: Fraction) -> int:
    """MPFR exponent of a nonzero rational: |x| in [2^(e-1), 2^e)."""
    ax = abs(x)
    e = ax.numerator.bit_length() - ax.denominator.bit_length()
    # adjust so that 2^(e-1) <= ax < 2^e
    while ax >= Fraction(2) ** e:
        e += 1
    while ax < Fraction(2) ** (e - 1):
        e -= 1
    return e


# ---------------------------------------------------------------------------
# Rounding helpers (plain definitions)
# ---------------------------------------------------------------------------

def rne_shift(n: int, s: int) -> int:
    """Round-half-even of n * 2^s to an integer (n any integer)."""
    if s >= 0:
        return n << s
    sg = -1 if n < 0 else 1
    a = abs(n)
    d = 1 << (-s)
    q, r = divmod(a, d)
    half = d >> 1
    if r > half or (r == half and (q & 1)):
        q += 1
    return sg * q


def round_to_p(num: int, scale: int, p: int) -> tuple[int, int, int]:
    """Round the dyadic num * 2^scale to p bits (round-half-even).

    Returns (sign, p-bit significand S with 2^(p-1) <= S < 2^p, exp) so that
    the rounded value is (-1)^sign * S * 2^(exp - p); zero -> (0, 0, 0).
    """
    if num == 0:
        return 0, 0, 0
    sg = 1 if num < 0 else 0
    a = abs(num)
    n = a.bit_length()
    S = rne_shift(a, p - n)      # p-bit (or 2^p after carry)
    e = n + scale                # |x| in [2^(e-1), 2^e)
    if S == (1 << p):
        S >>= 1
        e += 1
    return sg, S, e


def encode_rounded(sg: int, S: int, e: int, p: int) -> tuple[list[int], int, int]:
    """Pack a rounded p-bit result into nl MSB-normalised 64-bit limbs."""
    nl = (p + 63) // 64
    if S == 0:
        return [0] * nl, 0, 0
    full = S << (64 * nl - p)
    limbs = [(full >> (64 * q)) & ((1 << 64) - 1) for q in range(nl)]
    return limbs, e, sg


# ---------------------------------------------------------------------------
# Stage 1: shared exponents and integerization (Sec. 4.2, Eq. 1)
# ---------------------------------------------------------------------------

def row_exponent(mat: dict, r: int, axis: int) -> int:
    """e = max exp over the nonzero entries of row r (axis=0: row of a
    row-major matrix) or column r (axis=1).  An all-zero line gives 0."""
    R, C = mat["exp"].shape
    best = None
    n = C if axis == 0 else R
    for k in range(n):
        rr, cc = (r, k) if axis == 0 else (k, r)
        ssig, e, _ = decode(mat, rr, cc)
        if ssig != 0 and (best is None or e > best):
            best = e
    return 0 if best is None else best


def integerize(ssig: int, e_elem: int, nl: int, e_line: int, t: int) -> int:
    """a_hat = round(a * 2^(t - e)) with round-half-even (Eq. 1)."""
    if ssig == 0:
        return 0
    return rne_shift(ssig, e_elem - 64 * nl + t - e_line)


def integer_line(mat: dict, r: int, axis: int, t: int) -> tuple[list[int], int]:
    """Integerized row (axis=0) or column (axis=1) and its shared exponent."""
    e = row_exponent(mat, r, axis)
    R, C = mat["exp"].shape
    n = C if axis == 0 else R
    out = []
    for k in range(n):
        rr, cc = (r, k) if axis == 0 else (k, r)
        ssig, ex, nl = decode(mat, rr, cc)
        out.append(integerize(ssig, ex, nl, e, t))
    return out, e


# ---------------------------------------------------------------------------
# Stage 2: centered residues (Sec. 2.3, Sec. 4.3)
# ---------------------------------------------------------------------------

def cen(x: int, m: int) -> int:
    """Centered representative of x mod m in (-m/2, m/2]."""
    r = x % m
    if 2 * r > m:
        r -= m
    return r


def split128(r: int) -> tuple[int, int]:
    """Balanced base-128 split r = r0 + 128 r1, r0 = cen(r mod 128) (Sec. 4.3)."""
    r0 = cen(r, 128)
    r1 = (r - r0) // 128
    assert r0 + 128 * r1 == r
    return r0, r1


def plane_values(x: int, moduli: list[int]) -> list[int]:
    """All int8 plane entries of one integer: one per one-limb modulus, and
    (r0, r1, r0 + r1) per two-limb modulus (Eq. 4-5)."""
    out = []
    for m in moduli:
        r = cen(x, m)
        if m <= ONE_LIMB_MAX:
            out.append(r)
        else:
            r0, r1 = split128(r)
            out.extend((r0, r1, r0 + r1))
    return out


# ---------------------------------------------------------------------------
# Stages 3-4: exact plane products and mod-reduction (Sec. 2.4, Eq. 4)
# ---------------------------------------------------------------------------

def reduce_planes(prods: list[int], moduli: list[int]) -> list[int]:
    """u_l = C mod m for one-limb moduli; for two-limb moduli
    u = (P0 + 128 (Ps - P0 - P2) + 16384 P2) mod m (Karatsuba, Eq. 4)."""
    u = []
    g = 0
    for m in moduli:
        if m <= ONE_LIMB_MAX:
            u.append(prods[g] % m)
            g += 1
        else:
            P0, P2, Ps = prods[g], prods[g + 1], prods[g + 2]
            u.append((P0 + 128 * (Ps - P0 - P2) + 16384 * P2) % m)
            g += 3
    return u


# ---------------------------------------------------------------------------
# Stage 5: direct CRT (Sec. 4.4)
# ---------------------------------------------------------------------------

class CrtTables:
    """P, M_l = P / m_l and M_l^{-1} mod m_l for one modulus set (Sec. 4.4)."""

    def __init__(self, moduli: list[int]):
        self.moduli = list(moduli)
        self.P = product(moduli)
        self.M = [self.P // m for m in moduli]
        self.Minv = [pow(Ml % m, -1, m) for Ml, m in zip(self.M, moduli)]


def crt_definition(u: list[int], tab: CrtTables) -> int:
    """x0 in [0, P) with x0 = u_l mod m_l: the plain CRT definition."""
    S = sum(((ul * inv) % m) * Ml for ul, inv, m, Ml in zip(u, tab.Minv, tab.moduli, tab.M))
    return S % tab.P


def crt_alpha_route(u: list[int], tab: CrtTables) -> tuple[int, int]:
    """Direct CRT of Sec. 4.4: v_l = u_l (M_l^{-1} mod m_l) mod m_l,
    S = sum v_l M_l, alpha = floor(sum v_l / m_l) in binary64, use alpha - 1,
    R = S - (alpha - 1) P in [0, 3P), at most two subtractions.
    Returns (x0, exact alpha)."""
    v = [(ul * inv) % m for ul, inv, m in zip(u, tab.Minv, tab.moduli)]
    S = sum(vl * Ml for vl, Ml in zip(v, tab.M))
    a_fp = 0.0
    for vl, m in zip(v, tab.moduli):
        a_fp += vl / m
    alpha_est = math.floor(a_fp)
    R = S - (alpha_est - 1) * tab.P
    assert 0 <= R < 3 * tab.P, "alpha estimate off by more than one"
    subs = 0
    while R >= tab.P:
        R -= tab.P
        subs += 1
    assert subs <= 2
    alpha = S // tab.P
    assert alpha < len(tab.moduli)   # alpha < L (Sec. 4.4)
    return R, alpha


def crt_signed(u: list[int], tab: CrtTables) -> int:
    """Signed representative: x0 if x0 <= floor(P/2) else x0 - P (Sec. 4.4).
    Both CRT routes are evaluated and must agree."""
    x0, _ = crt_alpha_route(u, tab)
    assert x0 == crt_definition(u, tab)
    return x0 if x0 <= tab.P // 2 else x0 - tab.P


# ---------------------------------------------------------------------------
# The whole method, per output entry and for whole (small) matrices
# ---------------------------------------------------------------------------

class Params:
    """t, the modulus set and its CRT tables for an M x N x K product at p bits.

    ``inner`` (binary64 mode) widens t and the CRT bound to cover inner
    lengths up to max(K, inner), so that one modulus set serves the forward
    and both backward products."""

    def __init__(self, K: int, p: int, g: int = GUARD_BITS, inner: int = 0):
        if K > K_CAP:
            raise ValueError("K above the int32 exactness cap")
        self.K, self.p = K, p
        q = max(K, inner)
        self.t = internal_width(p, q, g)
        self.moduli = select_moduli(self.t, self.t, q)
        self.L = len(self.moduli)
        self.L1 = sum(1 for m in self.moduli if m <= ONE_LIMB_MAX)
        self.G = gemm_count(self.moduli)
        self.tab = CrtTables(self.moduli)


def stage_lines(A: dict, B: dict, par: Params, rows, cols):
    """Integerized rows of A / columns of B and their shared exponents."""
    Ar = {i: integer_line(A, i, 0, par.t) for i in rows}
    Bc = {j: integer_line(B, j, 1, par.t) for j in cols}
    return Ar, Bc


def entry(ahat_row: list[int], e_i: int, bhat_col: list[int], f_j: int,
          par: Params) -> dict:
    """All stages for one output entry; returns every intermediate."""
    pa = [plane_values(x, par.moduli) for x in ahat_row]
    pb = [plane_values(x, par.moduli) for x in bhat_col]
    prods = [sum(pa[k][g] * pb[k][g] for k in range(len(ahat_row))) for g in range(par.G)]
    for c in prods:
        assert abs(c) < 2 ** 31          # int32 exactness (Sec. 2.4)
    u = reduce_planes(prods, par.moduli)
    chat = crt_signed(u, par.tab)
    sg, S, e = round_to_p(chat, e_i + f_j - 2 * par.t, par.p)
    limbs, eo, so = encode_rounded(sg, S, e, par.p)
    return {"prods": prods, "u": u, "chat": chat, "limbs": limbs, "exp": eo, "sign": so}


def ozaki2_entries(A: dict, B: dict, p: int, pairs, g: int = GUARD_BITS) -> list[dict]:
    """Method (O) evaluated at the listed (i, j) output entries only."""
    K = A["exp"].shape[1]
    par = Params(K, p, g)
    rows = sorted({i for i, _ in pairs})
    cols = sorted({j for _, j in pairs})
    Ar, Bc = stage_lines(A, B, par, rows, cols)
    return [entry(Ar[i][0], Ar[i][1], Bc[j][0], Bc[j][1], par) for i, j in pairs]


def ozaki2_full(A: dict, B: dict, p: int, g: int = GUARD_BITS) -> dict:
    """Method (O) for every entry of a small product, with numpy int64 plane
    products (exact: every |C_g| < 2^31 is asserted)."""
    M, K = A["exp"].shape
    N = B["exp"].shape[1]
    par = Params(K, p, g)
    Ar, Bc = stage_lines(A, B, par, range(M), range(N))
    e = np.array([Ar[i][1] for i in range(M)], dtype=np.int64)
    f = np.array([Bc[j][1] for j in range(N)], dtype=np.int64)
    pa = np.array([[plane_values(x, par.moduli) for x in Ar[i][0]] for i in range(M)],
                  dtype=np.int64).reshape(M, K, par.G).transpose(2, 0, 1)   # [G, M, K]
    pb = np.array([[plane_values(x, par.moduli) for x in Bc[j][0]] for j in range(N)],
                  dtype=np.int64).reshape(N, K, par.G).transpose(2, 0, 1)   # [G, N, K]
    prods = np.matmul(pa, pb.transpose(0, 2, 1))                            # [G, M, N]
    assert np.abs(prods).max(initial=0) < 2 ** 31
    nl = (p + 63) // 64
    u = np.zeros((par.L, M, N), dtype=np.int64)
    g_ = 0
    for l, m in enumerate(par.moduli):
        if m <= ONE_LIMB_MAX:
            u[l] = prods[g_] % m
            g_ += 1
        else:
            P0, P2, Ps = prods[g_], prods[g_ + 1], prods[g_ + 2]
            u[l] = (P0 + 128 * (Ps - P0 - P2) + 16384 * P2) % m
            g_ += 3
    out_limbs = np.zeros((nl, M, N), dtype=np.uint64)
    out_exp = np.zeros((M, N), dtype=np.int32)
    out_sign = np.zeros((M, N), dtype=np.int8)
    chat = np.empty((M, N), dtype=object)
    for i in range(M):
        for j in range(N):
            c = crt_signed([int(x) for x in u[:, i, j]], par.tab)
            chat[i, j] = c
            sg, S, ex = round_to_p(c, int(e[i] + f[j]) - 2 * par.t, p)
            limbs, eo, so = encode_rounded(sg, S, ex, p)
            for q in range(nl):
                out_limbs[q, i, j] = limbs[q]
            out_exp[i, j] = eo
            out_sign[i, j] = so
    return {"par": par, "e": e, "f": f, "planes_a": pa, "planes_b": pb,
            "prods": prods, "u": u, "chat": chat,
            "C": {"p": p, "limbs": out_limbs, "exp": out_exp, "sign": out_sign}}


# ---------------------------------------------------------------------------
# (T) the truth: exact product rounded once
# ---------------------------------------------------------------------------

def truth_entry(A: dict, B: dict, i: int, j: int, p: int) -> tuple[list[int], int, int]:
    """Exact sum_k a_ik b_kj (dyadic, Python ints) rounded to p bits RNE."""
    K = A["exp"].shape[1]
    terms = []
    for k in range(K):
        sa, ea, nla = decode(A, i, k)
        sb, eb, nlb = decode(B, k, j)
        if sa and sb:
            terms.append((sa * sb, ea - 64 * nla + eb - 64 * nlb))
    if not terms:
        return encode_rounded(0, 0, 0, p)
    lo = min(s for _, s in terms)
    num = sum(v << (s - lo) for v, s in terms)
    sg, S, e = round_to_p(num, lo, p)
    return encode_rounded(sg, S, e, p)


def truth_full(A: dict, B: dict, p: int) -> dict:
    """Exact product of whole (small) matrices rounded to p bits."""
    M, K = A["exp"].shape
    N = B["exp"].shape[1]
    nl_a, nl_b = A["limbs"].shape[0], B["limbs"].shape[0]
    # exact integer rows/columns relative to the smallest exponent of the line
    Ai = np.empty((M, K), dtype=object)
    rmin = []
    for i in range(M):
        vals = [decode(A, i, k) for k in range(K)]
        exps = [e - 64 * nl for s, e, nl in vals if s]
        lo = min(exps) if exps else 0
        rmin.append(lo)
        for k, (s, e, nl) in enumerate(vals):
            Ai[i, k] = (s << (e - 64 * nl - lo)) if s else 0
    Bi = np.empty((K, N), dtype=object)
    cmin = []
    for j in range(N):
        vals = [decode(B, k, j) for k in range(K)]
        exps = [e - 64 * nl for s, e, nl in vals if s]
        lo = min(exps) if exps else 0
        cmin.append(lo)
        for k, (s, e, nl) in enumerate(vals):
            Bi[k, j] = (s << (e - 64 * nl - lo)) if s else 0
    Ci = Ai.dot(Bi)
    nl = (p + 63) // 64
    out_limbs = np.zeros((nl, M, N), dtype=np.uint64)
    out_exp = np.zeros((M, N), dtype=np.int32)
    out_sign = np.zeros((M, N), dtype=np.int8)
    for i in range(M):
        for j in range(N):
            sg, S, e = round_to_p(int(Ci[i, j]), rmin[i] + cmin[j], p)
            limbs, eo, so = encode_rounded(sg, S, e, p)
            for q in range(nl):
                out_limbs[q, i, j] = limbs[q]
            out_exp[i, j] = eo
            out_sign[i, j] = so
    del nl_a, nl_b
    return {"p": p, "limbs": out_limbs, "exp": out_exp, "sign": out_sign}


# ---------------------------------------------------------------------------
# Error measure: distance in ulps of the target precision
# ---------------------------------------------------------------------------

def to_fraction(limbs, e: int, s: int) -> Fraction:
    nl = len(limbs)
    sig = 0
    for q in range(nl):
        sig |= int(limbs[q]) << (64 * q)
    if sig == 0:
        return Fraction(0)
    v = Fraction(sig) * Fraction(2) ** (e - 64 * nl)
    return -v if s else v


def ulp_distance(x: Fraction, ref: Fraction, p: int) -> Fraction:
    """|x - ref| in units of ulp(ref) = 2^(exp(ref) - p); for ref = 0 the
    distance is 0 when x = 0 and infinite otherwise."""
    if ref == 0:
        return Fraction(0) if x == 0 else Fraction(10 ** 9)
    return abs(x - ref) / Fraction(2) ** (mpfr_exp(ref) - p)


def matrix_entry(mat: dict, i: int, j: int):
    nl = mat["limbs"].shape[0]
    return ([int(mat["limbs"][q, i, j]) for q in range(nl)], int(mat["exp"][i, j]),
            int(mat["sign"][i, j]))


# ---------------------------------------------------------------------------
# binary64 mode (forward and the reading used for the backward)
# ---------------------------------------------------------------------------

def from_double(x: float) -> tuple[int, int, int]:
    """(ssig, exp, nl=1) of a finite binary64 value, exact."""
    if x == 0.0:
        return 0, 0, 1
    fr = Fraction(x)
    e = mpfr_exp(fr)
    sig = abs(fr) * Fraction(2) ** (64 - e)
    assert sig.denominator == 1
    return (-1 if x < 0 else 1) * sig.numerator, e, 1


def fp64_as_mat(X: np.ndarray) -> dict:
    """A binary64 matrix in the limb format (p = 53, one limb)."""
    R, C = X.shape
    limbs = np.zeros((1, R, C), dtype=np.uint64)
    exp = np.zeros((R, C), dtype=np.int32)
    sign = np.zeros((R, C), dtype=np.int8)
    for r in range(R):
        for c in range(C):
            s, e, _ = from_double(float(X[r, c]))
            if s:
                limbs[0, r, c] = abs(s)
                exp[r, c] = e
                sign[r, c] = 1 if s < 0 else 0
    return {"p": 53, "limbs": limbs, "exp": exp, "sign": sign}


def to_double(limbs, e: int, s: int) -> float:
    return float(to_fraction(limbs, e, s))


# ---------------------------------------------------------------------------
# binary64 mode: forward and backward entries (reading for the backward, which
# the paper does not cover: the forward's integerized B_hat / A_hat are reused;
# dC is scaled by 2^f_j per column (dA) or 2^e_i per row (dB), exactly, and
# integerized with its own shared exponents per row (dA) / column (dB))
# ---------------------------------------------------------------------------

def f64_exponents(X: np.ndarray, axis: int) -> np.ndarray:
    """MPFR exponent max over the nonzero entries of each row (axis=1 reduces
    over columns) or column (axis=0); None for an all-zero line."""
    m, e = np.frexp(X)            # X = m 2^e, |m| in [0.5, 1): MPFR exponent e
    e = np.where(X != 0, e.astype(np.int64), np.iinfo(np.int64).min)
    best = e.max(axis=axis)
    return [None if b == np.iinfo(np.int64).min else int(b) for b in best]


def _f64_int(x: float, shift: int, e_line: int, t: int) -> int:
    if x == 0.0:
        return 0
    ssig, e, nl = from_double(float(x))
    return integerize(ssig, e + shift, nl, e_line, t)


def dgemm_params(M: int, N: int, K: int) -> Params:
    return Params(K, 53, inner=max(M, N, K))


def _round_double(chat: int, scale: int) -> float:
    sg, S, e = round_to_p(chat, scale, 53)
    return float((-1) ** sg * Fraction(S) * Fraction(2) ** (e - 53)) if S else 0.0


def dgemm_fwd_entry(X, Y, i, j, par: Params, e=None, f=None) -> float:
    e = f64_exponents(X, 1) if e is None else e
    f = f64_exponents(Y, 0) if f is None else f
    if e[i] is None or f[j] is None:
        return 0.0
    arow = [_f64_int(x, 0, e[i], par.t) for x in X[i, :]]
    bcol = [_f64_int(y, 0, f[j], par.t) for y in Y[:, j]]
    return _round_double(entry(arow, e[i], bcol, f[j], par)["chat"], e[i] + f[j] - 2 * par.t)


def dgemm_dA_entry(Y, dC, i, k, par: Params, f=None) -> float:
    """dA_ik = sum_j dC_ij B_kj through the cached B_hat (see module notes)."""
    f = f64_exponents(Y, 0) if f is None else f
    d1 = [(float(dC[i, j]), f[j]) for j in range(Y.shape[1])]
    exps = [from_double(x)[1] + fj for x, fj in d1 if x != 0.0 and fj is not None]
    if not exps:
        return 0.0
    g_i = max(exps)
    drow = [_f64_int(x, fj, g_i, par.t) if fj is not None else 0 for x, fj in d1]
    brow = [_f64_int(float(Y[k, j]), 0, f[j], par.t) if f[j] is not None else 0
            for j in range(Y.shape[1])]
    return _round_double(entry(drow, g_i, brow, 0, par)["chat"], g_i - 2 * par.t)


def dgemm_dB_entry(X, dC, k, j, par: Params, e=None) -> float:
    """dB_kj = sum_i A_ik dC_ij through the cached A_hat (see module notes)."""
    e = f64_exponents(X, 1) if e is None else e
    d2 = [(float(dC[i, j]), e[i]) for i in range(X.shape[0])]
    exps = [from_double(x)[1] + ei for x, ei in d2 if x != 0.0 and ei is not None]
    if not exps:
        return 0.0
    h_j = max(exps)
    dcol = [_f64_int(x, ei, h_j, par.t) if ei is not None else 0 for x, ei in d2]
    acol = [_f64_int(float(X[i, k]), 0, e[i], par.t) if e[i] is not None else 0
            for i in range(X.shape[0])]
    return _round_double(entry(acol, 0, dcol, h_j, par)["chat"], h_j - 2 * par.t)


def exact_dot_double(xs, ys) -> float:
    """Correctly rounded binary64 value of sum x*y (exact rational sum)."""
    return float(sum(Fraction(float(a)) * Fraction(float(b)) for a, b in zip(xs, ys)))


# ---------------------------------------------------------------------------
# Complex products, 3M form in the residue domain (the paper's Sec. 11 names
# complex 3M/4M products as future work; this is the reading used here).
# C = (Ar + i Ai)(Br + i Bi).  Rows of Ar and Ai share one exponent e_i (the
# largest over both), columns of Br and Bi one f_j, so that all four integer
# matrices carry the same scale and Cr_hat = sum ar br - ai bi and
# Ci_hat = sum ar bi + ai br are exact integers with |C_hat| <= 2K 2^(2t); t
# and the modulus set are chosen for inner length 2K.  Per modulus, three
# plane products T1 = ar br, T2 = ai bi, T3 = (ar + ai)(br + bi) of centered
# residues (the sums' residues are those of the integer sums), then
# u_r = T1 - T2 and u_i = T3 - T1 - T2 mod m, the direct CRT of each, and
# one rounding of each part to p bits.
# ---------------------------------------------------------------------------

def complex_params(K: int, p: int, g: int = GUARD_BITS) -> Params:
    """t and the modulus set of a complex product: inner length 2K."""
    return Params(K, p, g, inner=2 * K)


def joint_exponent(mats, r: int, axis: int) -> int:
    """Largest MPFR exponent over the nonzero entries of row r (axis=0) or
    column r (axis=1) of every matrix in mats; 0 when all of them are zero."""
    best = None
    for mat in mats:
        R, C = mat["exp"].shape
        n = C if axis == 0 else R
        for k in range(n):
            rr, cc = (r, k) if axis == 0 else (k, r)
            ssig, e, _ = decode(mat, rr, cc)
            if ssig != 0 and (best is None or e > best):
                best = e
    return 0 if best is None else best


def joint_lines(mats, r: int, axis: int, t: int):
    """The integerized lines of each matrix with their joint shared exponent."""
    e = joint_exponent(mats, r, axis)
    out = []
    for mat in mats:
        R, C = mat["exp"].shape
        n = C if axis == 0 else R
        line = []
        for k in range(n):
            rr, cc = (r, k) if axis == 0 else (k, r)
            ssig, ex, nl = decode(mat, rr, cc)
            line.append(integerize(ssig, ex, nl, e, t))
        out.append(line)
    return out, e


def complex_entry(ar, ai, e_i, br, bi, f_j, par: Params) -> dict:
    """All stages of one complex output entry (3M in the residue domain)."""
    def planes(xs):
        return [plane_values(x, par.moduli) for x in xs]
    pa_r, pa_i = planes(ar), planes(ai)
    pa_s = planes([x + y for x, y in zip(ar, ai)])
    pb_r, pb_i = planes(br), planes(bi)
    pb_s = planes([x + y for x, y in zip(br, bi)])
    K = len(ar)

    def prods(pa, pb):
        out = [sum(pa[k][g] * pb[k][g] for k in range(K)) for g in range(par.G)]
        assert all(abs(c) < 2 ** 31 for c in out)
        return out
    T1, T2, T3 = prods(pa_r, pb_r), prods(pa_i, pb_i), prods(pa_s, pb_s)
    u1, u2, u3 = (reduce_planes(T, par.moduli) for T in (T1, T2, T3))
    u_r = [(a - b) % m for a, b, m in zip(u1, u2, par.moduli)]
    u_i = [(c - a - b) % m for a, b, c, m in zip(u1, u2, u3, par.moduli)]
    chat_r, chat_i = crt_signed(u_r, par.tab), crt_signed(u_i, par.tab)
    out = {"T1": T1, "T2": T2, "T3": T3, "u_r": u_r, "u_i": u_i, "chat_r": chat_r, "chat_i": chat_i}
    for part, chat in (("r", chat_r), ("i", chat_i)):
        sg, S, e = round_to_p(chat, e_i + f_j - 2 * par.t, par.p)
        out["C" + part] = encode_rounded(sg, S, e, par.p)
    return out


def complex_entries(Ar, Ai, Br, Bi, p: int, pairs, g: int = GUARD_BITS) -> list[dict]:
    """The complex method at the listed (i, j) output entries."""
    K = Ar["exp"].shape[1]
    par = complex_params(K, p, g)
    rows = {i: joint_lines([Ar, Ai], i, 0, par.t) for i in sorted({i for i, _ in pairs})}
    cols = {j: joint_lines([Br, Bi], j, 1, par.t) for j in sorted({j for _, j in pairs})}
    out = []
    for i, j in pairs:
        (ar, ai), e_i = rows[i]
        (br, bi), f_j = cols[j]
        out.append(complex_entry(ar, ai, e_i, br, bi, f_j, par))
    return out


def complex_full(Ar, Ai, Br, Bi, p: int, g: int = GUARD_BITS) -> dict:
    """The complex method for every entry of a small product: Cr and Ci in the
    storage format, with the CRT integers and the reduced values."""
    M, K = Ar["exp"].shape
    N = Br["exp"].shape[1]
    nl = (p + 63) // 64
    ents = complex_entries(Ar, Ai, Br, Bi, p, [(i, j) for i in range(M) for j in range(N)], g)
    res = {"par": complex_params(K, p, g)}
    for part in ("r", "i"):
        limbs = np.zeros((nl, M, N), dtype=np.uint64)
        exp = np.zeros((M, N), dtype=np.int32)
        sign = np.zeros((M, N), dtype=np.int8)
        chat = np.empty((M, N), dtype=object)
        u = np.zeros((len(res["par"].moduli), M, N), dtype=np.int64)
        for n, e in enumerate(ents):
            i, j = divmod(n, N)
            lb, ex, sg = e["C" + part]
            for q in range(nl):
                limbs[q, i, j] = lb[q]
            exp[i, j], sign[i, j] = ex, sg
            chat[i, j] = e["chat_" + part]
            u[:, i, j] = e["u_" + part]
        res["C" + part] = {"p": p, "limbs": limbs, "exp": exp, "sign": sign}
        res["chat_" + part] = chat
        res["u_" + part] = u
    return res


def complex_truth_entry(Ar, Ai, Br, Bi, i: int, j: int, p: int):
    """Exact real and imaginary parts of entry (i, j), each rounded once."""
    K = Ar["exp"].shape[1]
    re = sum(value(Ar, i, k) * value(Br, k, j) - value(Ai, i, k) * value(Bi, k, j) for k in range(K))
    im = sum(value(Ar, i, k) * value(Bi, k, j) + value(Ai, i, k) * value(Br, k, j) for k in range(K))
    out = []
    for x in (re, im):
        if x == 0:
            out.append(encode_rounded(0, 0, 0, p))
            continue
        lo = x.denominator.bit_length() - 1               # dyadic: denominator 2^lo
        num = x.numerator                                  # x = num 2^-lo
        sg, S, e = round_to_p(num, -lo, p)
        out.append(encode_rounded(sg, S, e, p))
    return out
