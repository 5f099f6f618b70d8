"""The weight's regimes away from beta = 1/2 against the oracle: beta = 1/3
(lambda_1 bounded below) and beta = 1 (exponential decay) at N = 128 and
256, k = 64, 2048 bits (the settings of bench.py --workload regimes at these
N, where the precision check accepts 2048 bits): the whole factor and X bit
for bit, and lambda_1..3 to 1e-40 (tests/golden/r_<a>_<b>_<N>.json)."""
import json
import os

import pytest

mpm = pytest.importorskip("mpmath")

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.mark.parametrize("name", ["r_1_3_128", "r_1_3_256", "r_1_1_128", "r_1_1_256"])
def test_regime_against_oracle(name):
    import paper_1810_01478_gb300 as hk
    from oracle import mpfloat as F
    from tests.digest import factor_digest, x_digest
    path = os.path.join(HERE, "golden", name + ".json")
    if not os.path.exists(path):
        pytest.skip(f"golden {name} not generated")
    gd = json.load(open(path))
    (bn, bd), N, k, bits = gd["beta"], gd["N"], gd["k"], gd["bits"]
    hk.load()
    with hk.Hankel(0) as h:
        h.moments(bn, bd, N, bits)
        h.ldlt()
        loss, need = h.precision_loss()
        assert need <= bits
        h.inv_block(k)
        assert factor_digest(h, hk, N) == gd["factor_sha256"]
        assert x_digest(h, hk, N, k) == gd["x_sha256"]
        s, e, m, _, _ = h.lambda1(3)
    with mpm.workprec(2 * bits):
        for j in range(3):
            want = mpm.mpf(gd["lambdas"][j])
            got = F.to_mpf(F.from_limbs(int(s[j]), int(e[j]), m[j]), mpm)
            assert abs(got - want) / want < mpm.mpf(10) ** -40, (name, j)
