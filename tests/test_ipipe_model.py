"""CPU pin of the integer-pipe FP64 square root, reciprocal and quotient (the algorithm of
paper_2401_04576_gb300/csrc/ipipe.cuh), without a GPU.

A bit-level model of the fixed-point steps (64-bit unsigned / signed high products, Q62
Newton steps, remainders modulo 2^64, one-step corrections) is run with the FP32 seed
approximations perturbed by up to 2^-21 relative (the PTX rcp.approx / rsqrt.approx are
documented near 2^-23), and its results are compared with correctly rounded results from
exact rational arithmetic: rounded down, up and to nearest, over random significands and
exponents, the edge significands, perfect squares and their neighbours, and zero
numerators.  It also checks that the corrections never need more than the steps the
kernel takes, and that the remainders the kernel forms modulo 2^64 are far from
wrapping."""
import math
import random
import struct
from fractions import Fraction

M64 = (1 << 64) - 1


def dbits(x):
    return struct.unpack("<Q", struct.pack("<d", x))[0]


def bdouble(b):
    return struct.unpack("<d", struct.pack("<Q", b & M64))[0]


def f32(x):
    return struct.unpack("<f", struct.pack("<f", x))[0]


def fbits(x):
    return struct.unpack("<I", struct.pack("<f", x))[0]


def s64(a):
    a &= M64
    return a - (1 << 64) if a >> 63 else a


def umulhi(a, b):
    return ((a & M64) * (b & M64)) >> 64


def smulhi(a, b):
    return (s64(a) * s64(b)) >> 64          # floor, as mul.hi.s64


def q62(y):
    b = fbits(y)
    return ((b & 0x7FFFFF) | 0x800000) << (((b >> 23) & 0xFF) - 88)


class Steps:
    """Largest correction counts and remainder magnitudes seen."""
    lo = hi = 0
    rem_bits = 0


def corr(q, rem, m, st):
    n = 0
    while rem < 0:
        q, rem, n = q - 1, rem + m, n + 1
    st.lo = max(st.lo, n)
    n = 0
    while rem >= m:
        q, rem, n = q + 1, rem - m, n + 1
    st.hi = max(st.hi, n)
    return q, rem


def recip_q62(m, rel):
    g = struct.unpack("<f", struct.pack("<I", 0x3F800000 | ((m >> 29) & 0x7FFFFF)))[0]
    R = q62(f32((1.0 / g) * (1 + rel)))
    for _ in range(2):
        e = s64((1 << 61) - umulhi(m << 11, R))
        R = (R + smulhi(R, (e << 3) & M64)) & M64
    return R


def rcp_model(x, rel, st):
    """(rd bits, inexact, rn-up) of 1/x for x > 0 with biased exponent in [1, 2044]."""
    b = dbits(x)
    eb, m = b >> 52, (b & ((1 << 52) - 1)) | (1 << 52)
    q = recip_q62(m, rel) >> 9
    rem = s64(-(q * m))
    st.rem_bits = max(st.rem_bits, abs(rem).bit_length())
    q, rem = corr(q, rem, m, st)
    return ((2045 - eb) << 52) + q - (1 << 52), rem != 0, 2 * rem >= m


def sqrt_model(x, rel, st):
    b = dbits(x)
    ex, frac = b >> 52, b & ((1 << 52) - 1)
    odd = (ex & 1) ^ 1
    M2 = ((1 << 52) | frac) << odd
    f = struct.unpack("<f", struct.pack("<I", ((127 + odd) << 23) | (frac >> 29)))[0]
    Y = q62(f32((1.0 / math.sqrt(f)) * (1 + rel)))
    for _ in range(2):
        yy = umulhi(Y, Y)
        e = s64((1 << 58) - umulhi(M2 << 10, yy))
        Y = (Y + smulhi(Y, (e << 5) & M64)) & M64
    S = umulhi(M2 << 10, Y) >> 8
    r = s64((M2 << 52) - S * S)
    st.rem_bits = max(st.rem_bits, abs(r).bit_length())
    n = 0
    while r < 0:
        S -= 1
        r += 2 * S + 1
        n += 1
    st.lo = max(st.lo, n)
    n = 0
    while r > 2 * S:
        r -= 2 * S + 1
        S += 1
        n += 1
    st.hi = max(st.hi, n)
    ef = 1049 + ((ex - 1075 - odd) >> 1)
    return (ef << 52) + S - (1 << 52), r != 0, r > S


def div_model(a, b, rel, st):
    """(magnitude rd bits, inexact, rn-up, negative) of a / b, both normal, normal result."""
    A, B = dbits(a), dbits(b)
    ea, eb = (A >> 52) & 0x7FF, (B >> 52) & 0x7FF
    ma, mb = (A & ((1 << 52) - 1)) | (1 << 52), (B & ((1 << 52) - 1)) | (1 << 52)
    small = 1 if ma < mb else 0
    q = umulhi(ma << 11, recip_q62(mb, rel)) >> (9 - small)
    rem = s64((ma << (52 + small)) - q * mb)
    st.rem_bits = max(st.rem_bits, abs(rem).bit_length())
    q, rem = corr(q, rem, mb, st)
    be = ea - eb + 1023 - small
    assert 1 <= be <= 2046
    return (be << 52) + q - (1 << 52), rem != 0, 2 * rem > mb, ((A ^ B) >> 63) == 1


def rounded(t, mode):
    """Correctly rounded double of a positive rational t (normal range)."""
    x = float(t)
    c = sorted({x, math.nextafter(x, 0), math.nextafter(x, math.inf)})
    lo = max(v for v in c if Fraction(v) <= t)
    hi = min(v for v in c if Fraction(v) >= t)
    if mode == "rd" or lo == hi:
        return lo if mode != "ru" else hi
    if mode == "ru":
        return hi
    return lo if t - Fraction(lo) < Fraction(hi) - t else hi


def sqrt_rounded(v, mode):
    t = Fraction(v)
    s = math.sqrt(v)
    c = sorted({s, math.nextafter(s, 0), math.nextafter(s, math.inf)})
    lo = max(u for u in c if Fraction(u) ** 2 <= t)
    hi = min(u for u in c if Fraction(u) ** 2 >= t)
    if lo == hi or mode == "rd":
        return lo if mode != "ru" else hi
    if mode == "ru":
        return hi
    mid = (Fraction(lo) + Fraction(hi)) / 2
    return hi if mid * mid < t else lo


def _finish(bits, inexact, up, mode):
    return bdouble(bits + {"rd": 0, "ru": int(inexact), "rn": int(up)}[mode])


RELS = (-2.0 ** -21, 2.0 ** -21, 0.0)


def _normals(rng, n, lo=1, hi=2044):
    xs = [bdouble((rng.randint(lo, hi) << 52) | rng.getrandbits(52)) for _ in range(n)]
    for e in (1, 2, 1022, 1023, 1024, 2043, hi):
        for f in (0, 1, 2, (1 << 52) - 1, (1 << 52) - 2, 1 << 51, (1 << 51) + 1, (1 << 51) - 1):
            xs.append(bdouble((e << 52) | f))
    return xs


def test_reciprocal_model_correctly_rounded():
    rng = random.Random(1)
    st = Steps()
    for i, x in enumerate(_normals(rng, 2500)):
        rel = RELS[i % 3] if i % 5 else rng.uniform(-2.0 ** -21, 2.0 ** -21)
        bits, inexact, up = rcp_model(x, rel, st)
        t = 1 / Fraction(x)
        for mode in ("rd", "ru", "rn"):
            assert _finish(bits, inexact, up, mode) == rounded(t, mode), (x, mode)
    assert st.lo <= 2 and st.hi <= 2          # the kernel takes two steps each way
    assert st.rem_bits < 60                   # far from wrapping modulo 2^64


def test_square_root_model_correctly_rounded():
    rng = random.Random(2)
    st = Steps()
    xs = _normals(rng, 2500, 1, 2046)
    for _ in range(800):                      # perfect squares and their neighbours
        s = rng.randint(1 << 26, (1 << 27) - 1)
        for d in (-1, 0, 1):
            xs.append(float(s * s + d) * 2.0 ** rng.randint(-300, 300))
    for i, x in enumerate(xs):
        rel = RELS[i % 3] if i % 5 else rng.uniform(-2.0 ** -21, 2.0 ** -21)
        bits, inexact, up = sqrt_model(x, rel, st)
        for mode in ("rd", "ru", "rn"):
            assert _finish(bits, inexact, up, mode) == sqrt_rounded(x, mode), (x, mode)
    assert st.lo <= 2 and st.hi <= 2
    assert st.rem_bits < 60


def test_quotient_model_correctly_rounded():
    rng = random.Random(3)
    st = Steps()
    n = 0
    for i in range(3000):
        ea = rng.randint(200, 1800)
        eb = ea + rng.randint(-150, 150)
        fa = rng.getrandbits(52) if i % 7 else rng.choice([0, 1, (1 << 52) - 1])
        fb = rng.getrandbits(52) if i % 5 else rng.choice([0, (1 << 52) - 1, fa])
        a = bdouble((rng.getrandbits(1) << 63) | (ea << 52) | fa)
        b = bdouble((rng.getrandbits(1) << 63) | (eb << 52) | fb)
        rel = RELS[i % 3]
        bits, inexact, up, neg = div_model(a, b, rel, st)
        t = abs(Fraction(a) / Fraction(b))
        # magnitude rounded down / up / nearest; the signed directed results follow from
        # these by the sign (rd of a negative quotient is minus the magnitude rounded up)
        assert bdouble(bits) == rounded(t, "rd")
        assert bdouble(bits + int(inexact)) == rounded(t, "ru")
        assert bdouble(bits + int(up)) == rounded(t, "rn")
        assert neg == ((a < 0) != (b < 0))
        n += 1
    assert n == 3000 and st.lo <= 2 and st.hi <= 2 and st.rem_bits < 60
