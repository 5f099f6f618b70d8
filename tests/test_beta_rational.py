"""The differentiable front end takes beta as a float or tensor and works on
the exact rational a/b (b <= 1000) that the float stands for; anything
further than 2^-50 (relative) from such a rational is refused.  Host logic
only (no GPU)."""
import math
from fractions import Fraction

import pytest

torch = pytest.importorskip("torch")


def test_exact_beta_recovers_the_rational():
    from paper_1810_01478_gb300 import _exact_beta
    assert _exact_beta(0.5) == Fraction(1, 2)
    assert _exact_beta(0.45) == Fraction(9, 20)
    assert _exact_beta(torch.tensor(0.55, dtype=torch.float64)) == Fraction(11, 20)
    assert _exact_beta(1.0 / 3.0) == Fraction(1, 3)
    assert _exact_beta(Fraction(7, 999)) == Fraction(7, 999)


def test_exact_beta_refuses_irrational_and_large_denominators():
    from paper_1810_01478_gb300 import _exact_beta
    for v in (1.0 / math.pi, math.sqrt(2.0) / 3.0, 1.0 / 1009.0):
        with pytest.raises(ValueError):
            _exact_beta(v)
