"""Host checks of the arithmetic behind the pivot reciprocal square root
(kkt_numerics.cuh), with no GPU: Halley's step for f(r) = r^-2 - d',
evaluated as r + e (r/2 + (3r/8) e) with e = 1 - (d' r) r, starting from an
estimate of 24 significant bits within 2^-21 of 1/sqrt(d'), lands within
one unit in the last place of 1/sqrt(d') when every FP64 operation rounds
once (FMAs exact before rounding, emulated with fractions); and the
integer construction of r/2 and 3r/8 on the bits of r is exact over the
whole range of estimates. The device test (test_gpu_numerics.py) checks the
function itself on the GPU against the same bound over every exponent."""
import random
import struct
from decimal import Decimal, getcontext
from fractions import Fraction

getcontext().prec = 60


def _bits(x: float) -> int:
    return struct.unpack("<q", struct.pack("<d", x))[0]


def _dbl(b: int) -> float:
    return struct.unpack("<d", struct.pack("<q", b))[0]


def _f32(x: float) -> float:
    return struct.unpack("<f", struct.pack("<f", x))[0]


def _fma(a, b, c):
    return float(Fraction(a) * Fraction(b) + Fraction(c))


def _mul(a, b):
    return float(Fraction(a) * Fraction(b))


def _half_and_three_eighths(r: float):
    rb = _bits(r)
    re = (rb >> 52) & 0x7FF
    half = _dbl(rb - (1 << 52))
    sig3 = 3 * ((rb & ((1 << 52) - 1)) | (1 << 52))
    if sig3 >= (1 << 54):
        c = _dbl(((re - 1) << 52) | ((sig3 >> 2) - (1 << 52)))
    else:
        c = _dbl(((re - 2) << 52) | ((sig3 >> 1) - (1 << 52)))
    return half, c


def _ulp(x: float) -> Decimal:
    return Decimal(_dbl(_bits(x) + 1) - x)


def test_half_and_three_eighths_exact():
    """r/2 and 3r/8 from the bits: exact for estimates in (1/2, 1] with 24
    significant bits, including both sides of the renormalisation at a
    significand of 4/3."""
    rng = random.Random(7)
    samples = [_f32(0.5 + 2.0 ** -24), 1.0, _f32(2.0 / 3.0), _f32(2.0 / 3.0 + 2.0 ** -23),
               _f32(0.75), _f32(0.9999999)]
    samples += [struct.unpack("<f", struct.pack("<I", rng.randint(0x3F000001, 0x3F800000)))[0] for _ in range(3000)]
    for r in samples:
        half, c = _half_and_three_eighths(r)
        assert Fraction(half) == Fraction(r) / 2
        assert Fraction(c) == Fraction(3, 8) * Fraction(r)


def test_halley_step_within_one_ulp():
    rng = random.Random(11)
    worst = 0.0
    for t in range(4000):
        dp = 1.0 + 3.0 * rng.random() if t % 4 else rng.choice([1.0, 2.0, 3.999999999, 1.0000001])
        exact = Decimal(1) / Decimal(dp).sqrt()
        # an estimate of 24 significant bits within 2^-21 of 1/sqrt(d')
        r = _f32(float(exact) * (1.0 + (2.0 * rng.random() - 1.0) * 2.0 ** -21))
        half, c = _half_and_three_eighths(r)
        e = _fma(-_mul(dp, r), r, 1.0)
        r1 = _fma(_fma(c, e, half), e, r)
        worst = max(worst, float(abs(Decimal(r1) - exact) / _ulp(float(exact))))
    assert worst <= 1.0, f"{worst:.3f} ulp"
