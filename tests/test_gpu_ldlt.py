"""GPU parity of moments and Algorithm 1 (LDL^T) against the oracle, bit for bit."""
from fractions import Fraction

import pytest

from oracle import mpfloat as F
from oracle import moments as OM
from oracle import ldlt as OL
from tests import inputs
from tests.layout import from_arrays, to_arrays

pytestmark = pytest.mark.gpu


def run_factor(hk, N, bits, beta=(1, 2), mu=None):
    h = hk.Hankel(0)
    if mu is None:
        h.moments(beta[0], beta[1], N, bits)
    else:
        s, e, m = to_arrays(mu, bits // 32)
        h.set_moments(N, bits, s, e, m)
    h.ldlt()
    return h


def check_factor(h, hk, D, L, N):
    tri = N * (N + 1) // 2
    s, e, m = h.export(hk.HK_FACTOR, 0, tri)
    got = from_arrays(s, e, m)
    pos = 0
    bad = []
    for c in range(N):
        for r in range(c, N):
            want = D[c] if r == c else L[r][c]
            if got[pos] != want:
                bad.append((r, c))
            pos += 1
    assert not bad, f"{len(bad)} entries differ, first {bad[:5]}"


@pytest.mark.parametrize("beta,N,bits", [((1, 2), 95, 4096), ((1, 1), 60, 2048), ((1, 3), 40, 1024)])
def test_moments_bit_exact(beta, N, bits):
    import paper_1810_01478_gb300 as hk
    n = bits // 32
    with hk.Hankel(0) as h:
        h.moments(beta[0], beta[1], N, bits)
        got = from_arrays(*h.export(hk.HK_MU, 0, 2 * N - 1))
    assert got == OM.moments(Fraction(*beta), N, n)


@pytest.mark.parametrize("product_algorithm", [1, 2], indirect=True)
@pytest.mark.parametrize("N,bits", [(48, 4096), (1, 4096), (2, 1024), (33, 1024), (20, 24576), (40, 8192),
                                    (30, 12288), (25, 3072)])
def test_ldlt_beta_half_bit_exact(N, bits, product_algorithm):
    import paper_1810_01478_gb300 as hk
    n = bits // 32
    mu = OM.moments(Fraction(1, 2), N, n)
    D, L = OL.ldlt(mu, N, n)
    h = run_factor(hk, N, bits)
    try:
        check_factor(h, hk, D, L, N)
    finally:
        h.close()


def test_ldlt_beta_one_closed_form_and_oracle():
    import paper_1810_01478_gb300 as hk
    N, bits = 40, 2048
    n = bits // 32
    mu = OM.moments(Fraction(1), N, n)
    D, L = OL.ldlt(mu, N, n)
    with run_factor(hk, N, bits, beta=(1, 1)) as h:
        check_factor(h, hk, D, L, N)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_ldlt_measure_fuzz_bit_exact(seed):
    import paper_1810_01478_gb300 as hk
    N, bits = 24, 3072
    n = bits // 32
    mu = [F.from_int(v, n) for v in inputs.measure_moments(seed, N)]
    D, L = OL.ldlt(mu, N, n)
    with run_factor(hk, N, bits, mu=mu) as h:
        check_factor(h, hk, D, L, N)


def test_not_positive_definite_is_reported():
    import paper_1810_01478_gb300 as hk
    N, bits = 3, 1024
    mu = [F.from_int(v, 32) for v in [2, 3, 5, 9, 17]]  # a 2-atom measure: singular H_3
    h = run_factor(hk, N, bits, mu=mu)
    try:
        with pytest.raises(hk.HKError) as ei:
            h.export(hk.HK_D, 0, N)
        assert ei.value.status == hk.HK_ERR_NOT_PD
    finally:
        h.close()


def test_schoolbook_and_ntt_factors_identical():
    """The two exact-product algorithms give the same factor bit for bit
    (N = 160 at 12288 bits; digests of the whole packed factor)."""
    import paper_1810_01478_gb300 as hk
    from tests.digest import factor_digest
    hk.load()
    digests = []
    try:
        for alg in (hk.HK_PRODUCT_SCHOOLBOOK, hk.HK_PRODUCT_NTT):
            hk.hk_set_product_algorithm(alg)
            with hk.Hankel(0) as h:
                h.moments(1, 2, 160, 12288)
                h.ldlt()
                digests.append(factor_digest(h, hk, 160))
    finally:
        hk.hk_set_product_algorithm(hk.HK_PRODUCT_AUTO)
    assert digests[0] == digests[1]


def test_schoolbook_and_ntt_paths_identical():
    """Algorithm 4, the block, the eigen-solver (its matrix squarings run as
    NTT chains at NTT widths) and the gradient give the same limbs with either
    exact-product algorithm (N = 72, k = 16, 8192 bits)."""
    import numpy as np
    import paper_1810_01478_gb300 as hk
    from tests.digest import x_digest
    hk.load()
    outs = []
    try:
        for alg in (hk.HK_PRODUCT_SCHOOLBOOK, hk.HK_PRODUCT_NTT):
            hk.hk_set_product_algorithm(alg)
            with hk.Hankel(0) as h:
                h.moments(1, 2, 72, 8192)
                h.ldlt()
                h.inv_block(16)
                lam = h.lambda1(3)
                g = h.lambda1_grad()
                outs.append((x_digest(h, hk, 72, 16), [np.asarray(a).tobytes() for a in lam[:3]],
                             [np.asarray(a).tobytes() for a in g[:3]]))
    finally:
        hk.hk_set_product_algorithm(hk.HK_PRODUCT_AUTO)
    assert outs[0] == outs[1]
