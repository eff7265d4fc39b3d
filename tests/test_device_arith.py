"""CPU checks of arithmetic identities the CUDA kernels rely on for bit-exact
agreement with the oracle (no GPU needed; exact rational arithmetic stands in
for the FP64 units).

Division by a constant c in {3, 12, 20} (the predictor's dt/3 and the
corrector's a2/12, a3/20, a2/3): the kernels form q0 = RN(a y) with
y = RN(1/c), the exact residual r = a - c q0 (one FMA) and q = RN(q0 + r y)
(one FMA), which is RN(a / c) by Markstein's theorem (IBM J. Res. Dev. 34,
1990: q0 within one ulp of a/c, y within half an ulp of 1/c).  Here the three
steps are replayed exactly and compared with the correctly rounded quotient
on random operands over a wide exponent range and on operands whose quotient
lies next to a rounding midpoint.

Subtraction as the addition of the negated operand (the packed two-lane adds
of the DS force kernels): RN(a + (-b)) = RN(a - b) bit for bit in float32,
signed zeros, subnormals, infinities and NaN included.
"""
import math
import random
from fractions import Fraction as F

import pytest

CONSTS = (3, 12, 20)


def _markstein(a, c):
    y = 1.0 / c                       # RN(1/c), as the compiler folds it
    q0 = float(F(a) * F(y))           # RN(a * y)
    r = F(a) - F(q0) * c              # a - c q0, which the FMA forms exactly
    assert float(r) == r, "residual not representable"
    return float(F(q0) + r * F(y))    # RN(q0 + r y), the second FMA


def _operands(rng, count):
    for _ in range(count):
        m = rng.getrandbits(52) | (1 << 52)
        e = rng.randint(-200, 200)
        yield math.ldexp(m, e - 52) * rng.choice((1.0, -1.0))


@pytest.mark.parametrize("c", CONSTS)
def test_division_by_constant_is_correctly_rounded(c):
    rng = random.Random(c)
    for a in _operands(rng, 20000):
        assert _markstein(a, c) == float(F(a) / c), (a, c)


@pytest.mark.parametrize("c", CONSTS)
def test_division_by_constant_near_midpoints(c):
    # quotients within a few ulps of a midpoint between two doubles
    rng = random.Random(100 + c)
    for _ in range(4000):
        k = rng.getrandbits(52) | (1 << 52)
        mid = F(2 * k + 1, 2) * F(2) ** rng.randint(-60, 60)
        a0 = float(mid * c)
        for d in range(-3, 4):
            a = a0
            for _ in range(abs(d)):
                a = math.nextafter(a, math.inf if d > 0 else -math.inf)
            assert _markstein(a, c) == float(F(a) / c), (a, c)


def test_fast_path_limits_cover_the_faithful_quotient():
    # the kernels take the three-step path only for 2^-900 < |a| < 2^1000;
    # there neither a y nor the residual leaves the normal range
    for c in CONSTS:
        for a in (math.ldexp(1.0, -899), math.ldexp(1.999, 999), -math.ldexp(1.5, -899)):
            assert _markstein(a, c) == float(F(a) / c)


def test_adding_the_negation_rounds_as_the_subtraction():
    # The DS force kernels take the x and y components of x_j - x_i (hi and
    # lo parts) and of v_j - v_i as packed two-lane adds of the negated i
    # values: RN(a + (-b)) must be RN(a - b) bit for bit, signed zeros
    # included, for the forces to equal the scalar form's.  Negation is exact
    # in IEEE arithmetic, so the two are one operation; checked here in float32
    # on random magnitudes over the whole range, on equal and nearly equal
    # operands, and on the special values.
    np = pytest.importorskip("numpy")
    rng = np.random.default_rng(17)
    k = 200000
    mant = rng.uniform(-2.0, 2.0, size=(2, k))
    expo = rng.integers(-140, 128, size=(2, k))
    with np.errstate(over="ignore"):
        ab = np.ldexp(mant, expo).astype(np.float32)   # subnormal to overflowing
    a, b = ab[0], ab[1]
    b2 = np.nextafter(a, np.float32(np.inf))            # one ulp apart
    special = np.array([0.0, -0.0, 1.0, -1.0, np.inf, -np.inf, np.nan, 1e-45, -1e-45,
                        np.finfo(np.float32).max, -np.finfo(np.float32).max,
                        np.finfo(np.float32).tiny], dtype=np.float32)
    sa, sb = np.meshgrid(special, special)
    with np.errstate(over="ignore", invalid="ignore"):
        for x, y in ((a, b), (a, a), (a, b2), (b2, a), (sa.ravel(), sb.ravel())):
            x = np.asarray(x, dtype=np.float32)
            y = np.asarray(y, dtype=np.float32)
            sub = x - y
            add = x + (-y)
            assert sub.dtype == np.float32 and add.dtype == np.float32
            same = (sub.view(np.uint32) == add.view(np.uint32)) | (np.isnan(sub) & np.isnan(add))
            assert same.all(), (x[~same][:5], y[~same][:5])
