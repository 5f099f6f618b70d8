"""Pins for the oracle's number format (oracle/mpfloat.py).

Each primitive must return the exact result truncated toward zero to n limbs.
That is checked here as a property against Fraction arithmetic on the
operands: r is normalised, has the sign of the exact value v, and
|r| <= |v| < |r| + ulp(r).  Operands cover random values, large exponent gaps
(far-below operands), total and near-total cancellation, all-ones limbs and
zeros.
"""
import random
from fractions import Fraction

import pytest

from oracle import mpfloat as F
from tests import inputs


def check_trunc(r, v, n):
    assert F.is_normal(r, n)
    if v == 0:
        assert r == F.ZERO
        return
    rv = F.to_fraction(r)
    assert (rv > 0) == (v > 0)
    assert abs(rv) <= abs(v) < abs(rv) + F.ulp(r)


@pytest.mark.parametrize("n", [1, 2, 4, 7])
def test_rnd_and_from_fraction(n):
    rng = random.Random(n)
    for _ in range(400):
        v = rng.getrandbits(rng.randint(1, 40 * n)) * rng.choice([1, -1])
        e = rng.randint(-20, 20)
        r = F.rnd(v, e, n)
        check_trunc(r, Fraction(v) * Fraction(2) ** (32 * e), n)
        q = Fraction(v, rng.randint(1, 1 << 70) | 1)
        check_trunc(F.from_fraction(q, n), q, n)


@pytest.mark.parametrize("n", [1, 2, 4, 8])
def test_fused_property(n):
    rng = random.Random(100 + n)
    for a, x, y in inputs.fused_operands(rng, n, 600):
        v = F.to_fraction(a) - F.to_fraction(x) * F.to_fraction(y)
        check_trunc(F.fused(a, x, y, n), v, n)


@pytest.mark.parametrize("n", [1, 2, 4, 8])
def test_div_mul_add_property(n):
    rng = random.Random(200 + n)
    for a, x, y in inputs.fused_operands(rng, n, 400):
        if y[0] != 0:
            check_trunc(F.div(a, y, n), F.to_fraction(a) / F.to_fraction(y), n)
        check_trunc(F.mul(x, y, n), F.to_fraction(x) * F.to_fraction(y), n)
        check_trunc(F.add(a, x, n), F.to_fraction(a) + F.to_fraction(x), n)


def test_exact_cases():
    n = 3
    one = F.from_int(1, n)
    two = F.from_int(2, n)
    three = F.from_int(3, n)
    assert F.fused(three, one, two, n) == one            # 3 - 1*2
    assert F.fused(two, one, two, n) == F.ZERO           # total cancellation
    assert F.to_fraction(F.div(one, three, n)) < Fraction(1, 3)
    # 1 - tiny truncates to the largest n-limb value below 1
    tiny = (1 << 95, -10)  # far below one's last limb
    r = F.fused(one, tiny, one, n)
    assert r == ((1 << 96) - 1, -3)
    # limb round trip
    for x in [F.ZERO, one, F.neg(three), F.div(one, three, n)]:
        assert F.from_limbs(*F.limbs_of(x, n)) == x
