"""hk_alu_peak: the integer multiply pipe's measured rates, which the bench's
rooflines divide by.  An SM issues at most 4 x 32 thread instructions per
clock, so a rate above 128 operations per SM clock would mean the benchmark
did not do its work; the lazy Shoup modular multiplication takes three
multiplies, so it cannot run faster than the plain multiply-add."""
import pytest

pytestmark = pytest.mark.gpu


def test_alu_peak_rates_are_physical():
    import paper_1810_01478_gb300 as hk
    imad = hk.hk_alu_peak(0, 0)
    mod = hk.hk_alu_peak(0, 1)
    assert 8.0 <= imad <= 128.0
    assert 2.0 <= mod <= imad
    with pytest.raises(hk.HKError):
        hk.hk_alu_peak(0, 2)
