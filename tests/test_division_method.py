"""The correction step the detection uses for the contact normals (Markstein's
theorem: with y = RN(1/b), q = RN(a y), r = a - b q exact by one fused
multiply-add, RN(q + r y) = RN(a / b)), checked on the CPU in exact rational
arithmetic against IEEE division, on random quotients over many binades and
on the divisors that stress it (significands of all ones, powers of two,
neighbours of both).  The GPU's own outputs are compared with IEEE division
in tests/test_gpu_edge_cases.py."""
from fractions import Fraction

import numpy as np


def rn(x: Fraction) -> float:
    """Round a rational to the nearest double (ties to even)."""
    f = float(x)   # Python rounds a Fraction correctly to nearest, ties to even
    return f


def fma(a: float, b: float, c: float) -> float:
    return rn(Fraction(a) * Fraction(b) + Fraction(c))


def div_by(a: float, b: float) -> float:
    y = rn(Fraction(1) / Fraction(b))
    q = rn(Fraction(a) * Fraction(y))
    r = fma(-q, b, a)
    return fma(r, y, q)


def test_rn_is_correct_rounding():
    # a few hand cases of round-to-nearest-even at the double boundary
    one = Fraction(1)
    ulp = Fraction(1, 2 ** 52)
    assert rn(one + ulp / 2) == 1.0                      # tie to even (down)
    assert rn(one + 3 * ulp / 2) == 1.0 + 2 * float(ulp)   # tie to even (up)
    assert rn(one + ulp / 2 + Fraction(1, 2 ** 80)) == 1.0 + float(ulp)


def test_correction_step_gives_ieee_quotients():
    rng = np.random.default_rng(3)
    a = rng.normal(size=4000) * np.exp2(rng.integers(-60, 60, 4000))
    b = np.abs(rng.normal(size=4000)) * np.exp2(rng.integers(-60, 60, 4000)) + 1e-300
    ones = np.nextafter(2.0, 0.0)
    hard = []
    for e in range(-8, 9):
        for bb in (np.ldexp(ones, e), np.ldexp(1.0, e), np.nextafter(np.ldexp(1.0, e), 0.0),
                   np.nextafter(np.ldexp(1.0, e), 4.0), np.ldexp(1.5, e)):
            for aa in (1.0, -3.0, 0.1, np.nextafter(1.0, 2.0), np.ldexp(ones, 3), 0.7071067811865476):
                hard.append((aa, bb))
    cases = list(zip(a.tolist(), b.tolist())) + hard
    bad = [(x, y) for x, y in cases if div_by(x, y) != x / y]
    assert not bad, bad[:5]


def test_normals_as_the_detection_forms_them():
    """d = sqrt((x^2 + y^2) + z^2) correctly rounded, then the three components
    by the correction step: equal to the IEEE quotients."""
    rng = np.random.default_rng(9)
    dv = rng.uniform(-1.5, 1.5, (2000, 3))
    for x, y, z in dv.tolist():
        d = float(np.sqrt((x * x + y * y) + z * z))
        for comp in (x, y, z):
            assert div_by(comp, d) == comp / d
