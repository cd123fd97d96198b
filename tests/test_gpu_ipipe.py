"""The library's integer-pipe FP64 square root, reciprocal and quotient (rounded down, up
and to nearest) against the CUDA library's __dsqrt_* / __drcp_* / __ddiv_* bit for bit,
on random bit patterns over the whole normal range, on the edge significands (1, 1 + 2^-52, 2 - 2^-52), perfect squares
and their neighbours, the ends of the exponent range, and the arguments outside the fast
path (zero, subnormals, infinities, NaN, negatives); and a sample against exact rational
rounding computed here."""
import math
from fractions import Fraction

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2401_04576_gb300 import apo  # noqa: E402

OPS = ("rcp_rd", "rcp_ru", "rcp_rn", "sqrt_rd", "sqrt_ru", "sqrt_rn")


def _bits_to_f64(b):
    return np.asarray(b, dtype=np.uint64).view(np.float64)


def _inputs():
    rng = np.random.default_rng(11)
    n = 1 << 21
    exp = rng.integers(1, 2047, n, dtype=np.uint64)
    frac = rng.integers(0, 1 << 52, n, dtype=np.uint64)
    parts = [_bits_to_f64((exp << np.uint64(52)) | frac)]
    # edge significands at every exponent
    e = np.arange(0, 2048, dtype=np.uint64)
    for f in (0, 1, 2, (1 << 52) - 1, (1 << 52) - 2, 1 << 51, (1 << 51) - 1, (1 << 51) + 1):
        parts.append(_bits_to_f64((e << np.uint64(52)) | np.uint64(f)))
    # perfect squares of 26/27-bit and 53-bit integers, scaled, and their neighbours
    s = rng.integers(1 << 26, 1 << 27, 1 << 16).astype(np.float64)
    sq = s * s * np.ldexp(1.0, rng.integers(-900, 900, s.size))
    parts += [sq, np.nextafter(sq, 0), np.nextafter(sq, np.inf)]
    # subnormals, zeros, infinities, NaN, negatives (outside the fast path)
    parts.append(_bits_to_f64(rng.integers(1, 1 << 52, 4096, dtype=np.uint64)))
    parts.append(np.array([0.0, -0.0, np.inf, -np.inf, np.nan, -1.0, -2.5, -1e-310,
                           np.finfo(np.float64).max, np.finfo(np.float64).tiny]))
    return np.concatenate(parts)


def test_ipipe_matches_cuda_library():
    x = _inputs()
    xt = torch.as_tensor(x, device="cuda")
    for k, name in enumerate(OPS):
        got = apo.dops(k, xt).cpu().numpy()
        ref = apo.dops(k + 6, xt).cpu().numpy()
        bad = np.flatnonzero(~_same(got, ref))
        assert bad.size == 0, (name, bad.size, [(x[i], got[i], ref[i]) for i in bad[:5]])


def _same(got, ref):
    return (got.view(np.uint64) == ref.view(np.uint64)) | (np.isnan(got) & np.isnan(ref))


def _pairs():
    """(a, b) interleaved: random signs and significands, exponent differences over the
    whole range (quotients that overflow, underflow or go subnormal included), equal
    significands, zero numerators, and special divisors."""
    rng = np.random.default_rng(13)
    n = 1 << 20
    ea = rng.integers(1, 2047, n, dtype=np.uint64)
    eb = np.clip(ea.astype(np.int64) + rng.integers(-1100, 1100, n), 1, 2046).astype(np.uint64)
    fa = rng.integers(0, 1 << 52, n, dtype=np.uint64)
    fb = np.where(rng.random(n) < 0.05, fa, rng.integers(0, 1 << 52, n, dtype=np.uint64))
    sa = rng.integers(0, 2, n, dtype=np.uint64) << np.uint64(63)
    sb = rng.integers(0, 2, n, dtype=np.uint64) << np.uint64(63)
    a = _bits_to_f64(sa | (ea << np.uint64(52)) | fa)
    b = _bits_to_f64(sb | (eb << np.uint64(52)) | fb)
    a[::97] = 0.0
    a[1::97] = -0.0
    special = np.array([0.0, -0.0, np.inf, -np.inf, np.nan, 1e-310, -1e-310,
                        np.finfo(np.float64).max, np.finfo(np.float64).tiny, 1.0, -3.0])
    a2 = np.repeat(special, special.size)
    b2 = np.tile(special, special.size)
    a, b = np.concatenate([a, a2]), np.concatenate([b, b2])
    out = np.empty(2 * a.size)
    out[0::2], out[1::2] = a, b
    return out


def test_ipipe_quotients():
    x = _pairs()
    xt = torch.as_tensor(x, device="cuda")
    for k, name in enumerate(("div_rd", "div_ru", "div_rn")):
        got = apo.dops(12 + k, xt).cpu().numpy()[0::2]
        ref = apo.dops(15 + k, xt).cpu().numpy()[0::2]
        bad = np.flatnonzero(~_same(got, ref))
        assert bad.size == 0, (name, bad.size, [(x[2 * i], x[2 * i + 1], got[i], ref[i]) for i in bad[:5]])


def _exact(name, v):
    """Correctly rounded result of a positive normal v by exact rational arithmetic."""
    if name.startswith("rcp"):
        t = 1 / Fraction(v)
        cmp = lambda c: (Fraction(c) > t) - (Fraction(c) < t)          # noqa: E731
        a = 1.0 / v
    else:
        t = Fraction(v)
        cmp = lambda c: (Fraction(c) ** 2 > t) - (Fraction(c) ** 2 < t)   # noqa: E731
        a = math.sqrt(v)
    cands = sorted({a, math.nextafter(a, 0), math.nextafter(a, math.inf),
                    math.nextafter(math.nextafter(a, 0), 0)})
    lo = max(c for c in cands if cmp(c) <= 0)
    hi = min(c for c in cands if cmp(c) >= 0)
    if name.endswith("rd"):
        return lo
    if name.endswith("ru"):
        return hi
    if lo == hi:
        return lo
    # nearest: compare the distances exactly (no ties for these operations)
    if name.startswith("rcp"):
        return lo if t - Fraction(lo) < Fraction(hi) - t else hi
    mid = (Fraction(lo) + Fraction(hi)) / 2
    return hi if mid * mid < t else lo


def test_ipipe_exact_rounding_sample():
    rng = np.random.default_rng(12)
    exp = rng.integers(1, 2045, 3000, dtype=np.uint64)
    frac = rng.integers(0, 1 << 52, 3000, dtype=np.uint64)
    x = _bits_to_f64((exp << np.uint64(52)) | frac)
    xt = torch.as_tensor(x, device="cuda")
    for k, name in enumerate(OPS):
        got = apo.dops(k, xt).cpu().numpy()
        for i in range(0, x.size, 7):
            assert got[i] == _exact(name, float(x[i])), (name, x[i], got[i])
    # quotients within 2^+-41 of 1 (normal), negative divisors
    x = x[(exp > 100) & (exp < 1900)]
    b = -(x * rng.uniform(0.5, 2.0, x.size)) * np.ldexp(1.0, rng.integers(-40, 40, x.size))
    pairs = np.empty(2 * x.size)
    pairs[0::2], pairs[1::2] = x, b
    pt = torch.as_tensor(pairs, device="cuda")
    for k, mode in enumerate(("rd", "ru", "rn")):
        got = apo.dops(12 + k, pt).cpu().numpy()[0::2]
        for i in range(0, x.size, 7):
            t = Fraction(float(x[i])) / Fraction(float(b[i]))
            q = float(x[i]) / float(b[i])
            cands = (q, math.nextafter(q, -math.inf), math.nextafter(q, math.inf))
            want = {"rd": max(c for c in cands if Fraction(c) <= t),
                    "ru": min(c for c in cands if Fraction(c) >= t), "rn": q}[mode]
            assert got[i] == want, (mode, x[i], b[i], got[i], want)
