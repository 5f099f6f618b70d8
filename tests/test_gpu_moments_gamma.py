"""a1 for a rational beta: hk_moments_gamma forms mu_j from the constants
Gamma(r/a) on the device, bit for bit as the oracle's exact rational times
constant, truncated once (oracle.moments.moments_from_constants, with the
oracle's own constants from tests/golden/c3_gamma_constants.json at 12416
bits).  beta in {9/20, 11/20}, N in {128, 384} at 32 N bits; and the
factor, X and lambda at N = 128 compared with the path on imported moments."""
import json
import os
from fractions import Fraction

import numpy as np
import pytest

mpm = pytest.importorskip("mpmath")

from oracle import moments as OM
from tests.layout import to_arrays

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


def constants(beta):
    d = json.load(open(os.path.join(HERE, "golden", "c3_gamma_constants.json")))
    raw = d["constants"][f"{beta.numerator}/{beta.denominator}"]
    return [None] + [Fraction(int(p, 16), int(q, 16)) for p, q in raw[1:]]


def as_limbs(consts):
    """Fractions p / 2^s as (limb exponent, mantissa limbs), exactly."""
    rows, exps = [], []
    for v in consts[1:]:
        p, q = v.numerator, v.denominator
        s = q.bit_length() - 1
        assert q == 1 << s
        e = -((s + 31) // 32)
        m = p << (32 * -e - s)
        rows.append(m)
        exps.append(e)
    nc = max((m.bit_length() + 31) // 32 for m in rows)
    limbs = np.zeros((len(rows), nc), np.uint32)
    for i, m in enumerate(rows):
        ml = (m.bit_length() + 31) // 32
        for k in range(ml):
            limbs[i, k] = (m >> (32 * k)) & 0xFFFFFFFF
        # normalise to nc limbs: shift the mantissa up, the exponent down
        sh = nc - ml
        if sh:
            limbs[i] = np.roll(limbs[i], sh)
            limbs[i, :sh] = 0
            exps[i] -= sh
    return np.array(exps, np.int32), limbs


@pytest.mark.parametrize("beta", [Fraction(9, 20), Fraction(11, 20)])
@pytest.mark.parametrize("N", [128, 384])
def test_moments_gamma_bit_exact(beta, N):
    import paper_1810_01478_gb300 as hk
    hk.load()
    bits = 32 * N
    n = bits // 32
    consts = constants(beta)
    ce, cl = as_limbs(consts)
    want = to_arrays(OM.moments_from_constants(beta, N, n, consts), n)
    with hk.Hankel(0) as h:
        h.moments_gamma(beta.numerator, beta.denominator, N, bits, ce, cl)
        got = h.export(hk.HK_MU, 0, 2 * N - 1)
    for a, b in zip(got, want):
        assert np.array_equal(np.asarray(a).reshape(-1), np.asarray(b).reshape(-1))


def test_moments_gamma_path_matches_imported():
    import paper_1810_01478_gb300 as hk
    from tests.digest import factor_digest, x_digest
    hk.load()
    beta, N, bits = Fraction(9, 20), 128, 4096
    consts = constants(beta)
    ce, cl = as_limbs(consts)
    outs = []
    for mode in ("gamma", "import"):
        with hk.Hankel(0) as h:
            if mode == "gamma":
                h.moments_gamma(9, 20, N, bits, ce, cl)
            else:
                h.set_moments(N, bits, *to_arrays(OM.moments_from_constants(beta, N, bits // 32, consts), bits // 32),
                              9, 20)
            h.ldlt()
            h.inv_block(16)
            lam = h.lambda1(1)
            outs.append((factor_digest(h, hk, N), x_digest(h, hk, N, 16), np.asarray(lam[2]).tobytes()))
    assert outs[0] == outs[1]
