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


def test_front_end_asks_for_constants_at_rational_beta():
    """beta = 9/20 without the Gamma and psi constants is refused before any
    device work."""
    import paper_1810_01478_gb300 as hk
    for c in (None, {"gamma": ([], [])}):
        with pytest.raises(ValueError):
            hk.lambda1(torch.tensor(0.45, dtype=torch.float64, requires_grad=True), 48, 8, 4096, constants=c)
