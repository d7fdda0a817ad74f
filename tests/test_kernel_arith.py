"""Arithmetic facts the CUDA kernels rely on, checked exhaustively on the CPU.

The CUDA-core residue kernel reduces the byte-product sum a (one-limb
modulus m, a <= 4 * 32 words * 255 * 250 < 2^23) in fp32 with
q = round(a * rcp), rcp = 1/m rounded to fp32 as the library's host code
computes it.  For odd m the kernel takes r = a - q m as the centered residue
without a correction step; that holds exactly when q = round(a / m) for every
such a, which this test checks for all odd one-limb moduli of the method
(Sec. 4.3's moduli <= 255) and every reachable a.
"""
import numpy as np

from oracle import ozaki2_oracle as o


def test_fp32_rounded_quotient_is_exact_for_odd_one_limb_moduli():
    mods = [m for m in o.Params(1024, 2048).moduli if m <= 255]
    assert len(mods) == 54 and sum(m % 2 == 0 for m in mods) == 1      # 128 is the even one
    amax = 4 * 32 * 255 * 250
    assert amax < 2 ** 23
    a = np.arange(amax + 1, dtype=np.int64)
    af = a.astype(np.float64)
    for m in mods:
        if m % 2 == 0:
            continue
        rcp = np.float64(np.float32(1.0 / m))      # as the host computes it
        prod = af * rcp                            # exact in binary64 (23 x 24 bits)
        assert not np.any(prod - np.floor(prod) == 0.5), m
        q = np.rint(prod).astype(np.int64)
        q_true = (2 * a + m) // (2 * m)            # round(a / m); no ties for odd m
        assert np.array_equal(q, q_true), m
        r = a - q * m
        assert r.min() >= -(m // 2) and r.max() <= m // 2, m


def test_fp32_rounded_quotient_is_exact_for_two_limb_moduli():
    """Two-limb moduli (odd primes in (255, 16191]): the kernel reduces the
    high-byte sum with the rounded quotient, then y = s lo + 256 r_hi the same
    way; up to 24 words |y| <= 24 * 4 * 255^2 + 256 * 8095 < 2^23 / (1 + 2^-29)
    (beyond, up to 32 words, the low-byte sum is reduced first and |y| < 2^21).
    Exhaustive over |y| <= 4 * 32 * 255^2 (which covers both) for the smallest,
    the largest and a spread of the moduli in between."""
    mods = [m for m in o.Params(1024, 2048).moduli if m > 255]
    assert all(m % 2 == 1 for m in mods)
    pick = sorted(set([mods[0], mods[-1]] + mods[:: max(1, len(mods) // 10)]))
    amax = 4 * 32 * 255 * 255
    assert amax * (1 + 2.0 ** -29) < 2 ** 23
    assert 24 * 4 * 255 * 255 + 256 * 8095 <= amax
    a = np.arange(amax + 1, dtype=np.int64)
    af = a.astype(np.float64)
    for m in pick:
        rcp = np.float64(np.float32(1.0 / m))
        q = np.rint(af * rcp).astype(np.int64)
        assert np.array_equal(q, (2 * a + m) // (2 * m)), m
    # y = r_lo + 256 r_hi over its whole range, for the same moduli
    for m in pick:
        h = (m - 1) // 2
        y = np.arange(-257 * h, 257 * h + 1, dtype=np.int64)
        rcp = np.float64(np.float32(1.0 / m))
        q = np.rint(y.astype(np.float64) * rcp).astype(np.int64)
        assert np.array_equal(q, np.floor_divide(2 * y + m, 2 * m)), m


def test_tensor_core_two_limb_reduction_needs_no_correction():
    """The warp-specialised tensor-core residues reduce a two-limb modulus
    from the byte sums y0 (table halves |T0| <= 64) and y1 (|T1| <= 63) of at
    most 265 bytes: r1 = y1 - RN(y1 rcp) m, x = y0 + 128 r1, r = x - RN(x rcp) m,
    with no correction step.  Exhaustive over every |y1| <= 265 * 255 * 63 and
    every |x| <= 265 * 255 * 64 + 128 * 8095 for a spread of the moduli: the
    rounded quotient is round(y / m) and the remainder the centered residue."""
    mods = [m for m in o.Params(1024, 2048).moduli if m > 255]
    pick = sorted(set([mods[0], mods[-1]] + mods[:: max(1, len(mods) // 8)]))
    y1max = 265 * 255 * 63
    xmax = 265 * 255 * 64 + 128 * 8095
    assert max(y1max, xmax) < 2 ** 23
    for bound in (y1max, xmax):
        y = np.arange(-bound, bound + 1, dtype=np.int64)
        yf = y.astype(np.float64)
        for m in pick:
            rcp = np.float64(np.float32(1) / np.float32(m))     # RN(1/m), as the host computes it
            assert rcp == np.float64(np.float32(1.0 / m))
            q = np.rint(yf * rcp).astype(np.int64)              # y rcp is exact in binary64
            r = y - q * m
            assert r.min() >= -(m - 1) // 2 and r.max() <= (m - 1) // 2, m
            assert np.array_equal(np.mod(r - y, m), np.zeros_like(y)), m


def test_balanced_split_by_shifted_rounding():
    """split128: hi = RN((r - 0.5) / 128), lo = r - 128 hi is the balanced
    base-128 split (lo in (-64, 64]) for every |r| <= 8095."""
    r = np.arange(-8095, 8096, dtype=np.int64)
    h = (r.astype(np.float64) - 0.5) / 128.0
    assert not np.any(h - np.floor(h) == 0.5)
    hi = np.rint(h).astype(np.int64)
    lo = r - 128 * hi
    assert lo.min() == -63 and lo.max() == 64
    assert np.array_equal(lo + 128 * hi, r)


def _byte_perm(x, y, sel):
    """Byte permute: result byte n is byte (sel >> 4 n) & 7 of the pair
    (x low, y high), as the CUDA byte-permute intrinsic defines it."""
    src = [(x >> (8 * i)) & 0xFF for i in range(4)] + [(y >> (8 * i)) & 0xFF for i in range(4)]
    return sum(src[(sel >> (4 * n)) & 7] << (8 * n) for n in range(4))


def _f16_bits(v):
    """f16 bits derived from the value alone (sign, 5-bit exponent with bias
    15, 10 mantissa bits) for an integer |v| < 2^11."""
    if v == 0:
        return 0
    sgn = 0x8000 if v < 0 else 0
    a = abs(v)
    e = a.bit_length() - 1
    return sgn | ((15 + e) << 10) | (((a << 10) >> e) & 0x3FF)


def _f16(bits):
    return np.array([bits], dtype=np.uint16).view(np.float16)[0]


def _h2(word):
    return _f16(word & 0xFFFF), _f16(word >> 16)


def test_f16_bytes_of_the_tensor_core_residue_builders():
    """Both tensor-core residue kernels feed the bytes of |a_hat| to the MMA
    as f16.  The byte permute with 0x64646464 puts byte b under the exponent
    bits of 2^10 (0x64xx is 1024 + b: the mantissa's unit is 1 there); then
    the unsigned form subtracts 1024 (packed) and the signed form takes one
    packed fma with {s, s} and {-1024 s, -1024 s}.  Every intermediate is an
    integer below 2^11, so each step is exact in f16; checked for every byte,
    byte position and sign against f16 bits derived from the value."""
    for v in (1, 127, -64, 255, 1024, 1279, -1279):
        assert float(_f16(_f16_bits(v))) == v                   # the bits rule itself
    m1024 = _f16(0x6400)
    assert float(_f16(0x3C00)) == 1.0 and float(m1024) == 1024.0
    for sel, lo_pos in ((0x5140, 0), (0x7362, 2)):
        for b in range(256):
            for other in (0x00, 0xFF, 0x5A):
                x = (b << (8 * lo_pos)) | (other << (8 * (lo_pos + 1)))
                x |= 0xA5A50000 if lo_pos == 0 else 0x0000A5A5     # the bytes the selector skips
                lo, hi = _h2(_byte_perm(x, 0x64646464, sel))
                assert float(lo) == 1024 + b and float(hi) == 1024 + other
                # unsigned: one packed subtraction of {1024, 1024}
                u = (np.float16(lo - m1024), np.float16(hi - m1024))
                assert [int(t.view(np.uint16)) for t in u] == [_f16_bits(b), _f16_bits(other)]
                # signed: fma(p, s, -1024 s); the product and the sum are exact
                for s2, c2, sg in ((0x3C003C00, 0xE400E400, 1), (0xBC00BC00, 0x64006400, -1)):
                    s_lo, c_lo = _h2(s2)[0], _h2(c2)[0]
                    assert float(s_lo) == sg and float(c_lo) == -1024 * sg
                    r = np.float16(np.float16(lo * s_lo) + c_lo)
                    assert int(r.view(np.uint16)) == _f16_bits(sg * b)   # +0, never -0, for b = 0
