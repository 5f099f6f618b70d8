"""The precision check of the factorisation: hk_precision_loss (formed on the
device right after hk_ldlt) against the oracle's loss estimate
max(0, max_i ceil(log2(mu_{2i} / d_i))) on the same factor
(oracle.precision), and hk_lambda1's HK_ERR_PRECISION when the working
precision is below 2 loss + 229 bits (beta = 1/2, N = 384 at 1024 bits,
where the estimate is over 500 bits; N = 256 at the same width passes)."""
from fractions import Fraction

import pytest

mpm = pytest.importorskip("mpmath")

from oracle import ldlt as LD
from oracle import moments as OM
from oracle import precision as PR
from tests.test_gpu_moments_gamma import as_limbs, constants

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("beta,N,bits", [((1, 2), 48, 4096), ((1, 1), 40, 2048), ((1, 2), 128, 1024),
                                         ((9, 20), 64, 2048)])
def test_loss_estimate_vs_oracle(beta, N, bits):
    import paper_1810_01478_gb300 as hk
    n = bits // 32
    bq = Fraction(*beta)
    with hk.Hankel(0) as h:
        if bq.numerator == 1:
            mu = OM.moments(bq, N, n)
            h.moments(beta[0], beta[1], N, bits)
        else:
            consts = constants(bq)
            mu = OM.moments_from_constants(bq, N, n, consts)
            h.moments_gamma(beta[0], beta[1], N, bits, *as_limbs(consts))
        h.ldlt()
        loss, mb = h.precision_loss()
    D, _ = LD.ldlt(mu, N, n)
    want = PR.loss_estimate(mu, D)
    assert loss == want
    assert mb == PR.min_bits(loss)


@pytest.mark.parametrize("N,fires", [(384, True), (256, False)])
def test_lambda_guard(N, fires):
    import paper_1810_01478_gb300 as hk
    bits = 1024
    with hk.Hankel(0) as h:
        h.moments(1, 2, N, bits)
        h.ldlt()
        loss, mb = h.precision_loss()
        assert (bits < mb) == fires
        h.inv_block(16)
        if fires:
            with pytest.raises(hk.HKError) as ei:
                h.lambda1(1)
            assert ei.value.status == hk.HK_ERR_PRECISION
        else:
            h.lambda1(1)
