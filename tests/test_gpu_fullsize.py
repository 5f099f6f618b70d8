"""Parity at the benchmark's full size: beta = 1/2, N = 1024, k = 32.

At 24576 bits (the bench workload, same calls as bench.py) the full factor is
beyond the oracle's reach, so it is checked on samples the oracle can compute
one by one: factor entries L[r][c] (and pivots) by Algorithm 1 on the index
set {0..c} U {r} (oracle.ldlt.sample_entry, which reproduces the full
factor's entry exactly), the first 40 rows of X (which depend only on the
leading 40 x 40 block), lambda_1..3 against the oracle's N = 1024 runs
(tests/golden/c5_1024_*.json, accurate far beyond 1e-40 at 4096 bits), and
the gradient against the oracle's analytic gradient at N = 1024 (and by
precision doubling).  At 4096 bits (schoolbook products) and 8192 bits (NTT
products) the whole N = 1024 factor and X are compared bit for bit through
their SHA-256 digests; at the widest widths the whole factor and X are
compared at N = 256 and N = 320 (24576 bits) and N = 160 (16384 bits).
"""
import json
import os
from fractions import Fraction

import pytest

mpm = pytest.importorskip("mpmath")

from oracle import mpfloat as F
from oracle import moments as OM
from oracle import ldlt as OL
from oracle import invblock as IB
from tests.layout import from_arrays

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))
N, K = 1024, 32
TOL = mpm.mpf(10) ** -40


def golden(name):
    path = os.path.join(HERE, "golden", name + ".json")
    if not os.path.exists(path):
        pytest.skip(f"golden {name} not generated")
    return json.load(open(path))


def run(hk, bits):
    h = hk.Hankel(0)
    h.moments(1, 2, N, bits)
    h.ldlt()
    h.inv_block(K)
    lam = h.lambda1(3)
    g = h.lambda1_grad()
    return h, lam, g


def value(s, e, m):
    return F.to_mpf(F.from_limbs(int(s), int(e), m), mpm)


def test_bench_workload_sampled_parity():
    import paper_1810_01478_gb300 as hk
    from oracle.mpfloat import LIMB  # noqa: F401
    bits = 24576
    n = bits // 32
    hk.load()
    h, lam, g = run(hk, bits)
    try:
        mu = OM.moments(Fraction(1, 2), N, n)
        # factor samples
        samples = [(c, c) for c in (0, 7, 31)] + [(r, c) for c in (0, 3, 15, 31) for r in (c + 1, 257, 700, N - 1)]
        for r, c in samples:
            s, e, m = h.export(hk.HK_FACTOR, c * N - c * (c - 1) // 2 + (r - c), 1)
            assert F.from_limbs(int(s[0]), int(e[0]), m[0]) == OL.sample_entry(mu, r, c, n), (r, c)
        # the first 40 rows of X depend only on the leading 40 x 40 block
        D40, L40 = OL.ldlt_subset(mu, list(range(40)), n)
        X40 = IB.partial_inverse(L40, 40, K, n)
        got = from_arrays(*h.export(hk.HK_X, 0, 40 * K))
        assert all(got[r * K + c] == X40[r][c] for r in range(40) for c in range(K))
        # lambda against the oracle's N = 1024 runs
        for name in ("c5_1024_4096", "c5_1024_8192"):
            path = os.path.join(HERE, "golden", name + ".json")
            if not os.path.exists(path):
                continue
            gd = json.load(open(path))
            with mpm.workprec(2 * bits):
                for j in range(3):
                    want = mpm.mpf(gd["lambdas"][j])
                    assert abs(value(lam[0][j], lam[1][j], lam[2][j]) - want) / want < TOL, (name, j)
        # the gradient against the oracle's (analytic, at 4096 bits: its error is far below 1e-40)
        gd = golden("c5_1024_4096")
        with mpm.workprec(2 * bits):
            want = mpm.mpf(gd["grad"])
            got = value(g[0][0], g[1][0], g[2][0])
            assert abs(got - want) / abs(want) < TOL
        # the gradient at half the precision agrees (precision doubling)
        h2, lam2, g2 = run(hk, bits // 2)
        h2.close()
        with mpm.workprec(2 * bits):
            a, b = value(g[0][0], g[1][0], g[2][0]), value(g2[0][0], g2[1][0], g2[2][0])
            assert abs(a - b) / abs(a) < TOL
            for j in range(3):
                x, y = value(lam[0][j], lam[1][j], lam[2][j]), value(lam2[0][j], lam2[1][j], lam2[2][j])
                assert abs(x - y) / x < TOL
    finally:
        h.close()


@pytest.mark.parametrize("bits", [4096, 8192])
def test_full_factor_bit_exact(bits):
    """The whole N = 1024 factor and X bit for bit: at 4096 bits with
    schoolbook products, at 8192 bits with NTT products."""
    import paper_1810_01478_gb300 as hk
    from tests.digest import factor_digest, x_digest
    gd = golden("c5_1024_%d" % bits)
    hk.load()
    h, lam, _ = run(hk, bits)
    try:
        assert factor_digest(h, hk, N) == gd["factor_sha256"]
        assert x_digest(h, hk, N, K) == gd["x_sha256"]
        with mpm.workprec(2 * bits):
            for j in range(3):
                want = mpm.mpf(gd["lambdas"][j])
                assert abs(value(lam[0][j], lam[1][j], lam[2][j]) - want) / want < TOL
    finally:
        h.close()


@pytest.mark.parametrize("n_", [512, 768])
def test_sweep_sizes(n_):
    """The paper-scale sweep sizes N = 512, 768 (k = 32): the whole factor and
    X bit for bit at 4096 bits, and lambda_1..3 at 24576 bits against the
    oracle's 4096-bit values (accurate far beyond 1e-40 at these N)."""
    import paper_1810_01478_gb300 as hk
    from tests.digest import factor_digest, x_digest
    gd = golden("c5_%d_4096" % n_)
    hk.load()
    for bits in (4096, 24576):
        with hk.Hankel(0) as h:
            h.moments(1, 2, n_, bits)
            h.ldlt()
            h.inv_block(K)
            s, e, m, _, _ = h.lambda1(3)
            if bits == 4096:
                assert factor_digest(h, hk, n_) == gd["factor_sha256"]
                assert x_digest(h, hk, n_, K) == gd["x_sha256"]
            with mpm.workprec(2 * bits):
                for j in range(3):
                    want = mpm.mpf(gd["lambdas"][j])
                    assert abs(value(s[j], e[j], m[j]) - want) / want < TOL, (n_, bits, j)


def test_planned_block_at_the_widest_width():
    """N = 320 at 24576 bits with hk_plan_block(k): the 64 steps with at least
    256 trailing rows run Algorithm 4 inside their tensor-core launches; the
    factor, X and lambda_1..3 equal the oracle's (tests/golden/w_320_24576)."""
    import paper_1810_01478_gb300 as hk
    from tests.digest import factor_digest, x_digest
    gd = golden("w_320_24576")
    N_, k_, bits = gd["N"], gd["k"], gd["bits"]
    hk.load()
    with hk.Hankel(0) as h:
        h.moments(1, 2, N_, bits)
        h.ldlt(k=k_)
        h.inv_block(k_)
        assert factor_digest(h, hk, N_) == gd["factor_sha256"]
        assert x_digest(h, hk, N_, k_) == gd["x_sha256"]
        s, e, m, _, _ = h.lambda1(3)
        with mpm.workprec(2 * bits):
            for j in range(3):
                want = mpm.mpf(gd["lambdas"][j])
                assert abs(value(s[j], e[j], m[j]) - want) / want < TOL, j


@pytest.mark.parametrize("name", ["w_256_24576", "w_160_16384", "w_320_24576"])
def test_widest_widths_whole_factor(name):
    """The whole factor and X bit for bit at 24576 bits (M = 24 limbs per
    lane: every step shape of the widest product width, from the first
    steps to the late ones) and at 16384 bits (M = 16), with lambda_1..3 and,
    where the oracle computed it, the gradient to 1e-40."""
    import paper_1810_01478_gb300 as hk
    from tests.digest import factor_digest, x_digest
    gd = golden(name)
    N_, k_, bits = gd["N"], gd["k"], gd["bits"]
    hk.load()
    with hk.Hankel(0) as h:
        h.moments(1, 2, N_, bits)
        h.ldlt()
        h.inv_block(k_)
        assert factor_digest(h, hk, N_) == gd["factor_sha256"]
        assert x_digest(h, hk, N_, k_) == gd["x_sha256"]
        s, e, m, _, _ = h.lambda1(3)
        g = h.lambda1_grad() if "grad" in gd else None
        with mpm.workprec(2 * bits):
            for j in range(3):
                want = mpm.mpf(gd["lambdas"][j])
                assert abs(value(s[j], e[j], m[j]) - want) / want < TOL, (name, j)
            if g is not None:
                want = mpm.mpf(gd["grad"])
                assert abs(value(g[0][0], g[1][0], g[2][0]) - want) / abs(want) < TOL
