"""Parity of the tensor-core products (HK_PRODUCT_TENSOR) with the oracle and
with the other exact-product algorithms, bit for bit.

The tensor-core path forms each product as a bf16 GEMM of balanced 7-bit
digits with fp32 accumulators; it is exact only if every digit-product sum
stays an integer below 2^24 and every limb is assembled without loss, so the
checks here are the same bit-for-bit checks as for the schoolbook and NTT
products: the elementwise fused update against the oracle (random,
structured, deep-cancellation and far-apart operands, plus operands whose
digits all have the largest magnitude, 64, which push the sums to within 1 %
of the bound), and whole factors against the NTT path and the oracle's
digests.
"""
import random

import pytest

from oracle import mpfloat as F
from tests import inputs
from tests.layout import DevNums

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("M", [8, 12, 16, 24])
def test_tensor_fused_batch_bit_exact(M):
    import torch
    import paper_1810_01478_gb300 as hk
    hk.load()
    n = 32 * M
    rng = random.Random(3000 + M)
    ops = inputs.fused_operands(rng, n, 300 if M < 24 else 200)
    ext = inputs.digit_extreme_mant(n)
    ops += [((rng.getrandbits(32 * n) | 1 << (32 * n - 1), 3), (ext, 1), (ext, 2)),
            ((0, 0), (-ext, -4), (ext, 7)),
            (((1 << (32 * n)) - 1, 2 * n), (ext, n), ((1 << (32 * n)) - 1, 0))]
    a, x, y = (list(t) for t in zip(*ops))
    A, X, Y = DevNums(a, n=n), DevNums(x, n=n), DevNums(y, n=n)
    OUT = DevNums(count=len(ops), n=n)
    try:
        hk.hk_set_product_algorithm(hk.HK_PRODUCT_TENSOR)
        hk.hk_fused_batch(32 * n, len(ops), A.ptrs, X.ptrs, Y.ptrs, OUT.ptrs,
                          torch.cuda.current_stream().cuda_stream)
    finally:
        hk.hk_set_product_algorithm(hk.HK_PRODUCT_AUTO)
    torch.cuda.synchronize()
    got = OUT.to_host()
    for i, t in enumerate(ops):
        assert got[i] == F.fused(*t, n), (M, i)


@pytest.mark.parametrize("N,bits", [(300, 8192), (320, 12288), (300, 16384), (290, 24576)])
def test_tensor_factor_matches_ntt(N, bits):
    """The whole factor with tensor-core trailing updates (every step whose
    trailing triangle has at least 256 rows) against the NTT path."""
    import paper_1810_01478_gb300 as hk
    from tests.digest import factor_digest
    hk.load()
    digests = []
    try:
        for alg in (hk.HK_PRODUCT_NTT, hk.HK_PRODUCT_TENSOR):
            hk.hk_set_product_algorithm(alg)
            with hk.Hankel(0) as h:
                h.moments(1, 2, N, bits)
                h.ldlt()
                digests.append(factor_digest(h, hk, N))
    finally:
        hk.hk_set_product_algorithm(hk.HK_PRODUCT_AUTO)
    assert digests[0] == digests[1]


@pytest.mark.parametrize("b,N,bits,rerun", [(1, 300, 8192, "most"), (2, 320, 12288, "few")])
def test_short_products_and_their_reruns(b, N, bits, rerun):
    """The trailing update forms only the product positions that can reach
    the truncated result and re-runs, with whole products, the 128-row items
    where that cannot be decided.  beta = 1 at 8192 bits keeps every entry
    an exact integer (mu_j = j!, D_i = (i!)^2), so the guard limbs of the
    differences are zero and nearly every item is re-run; at beta = 1/2 the
    entries stop being integers after the first step (L[r][1] is already a
    proper fraction) and only that step's items are re-run.  Both factors
    must equal the NTT path's bit for bit."""
    import paper_1810_01478_gb300 as hk
    from tests.digest import factor_digest
    hk.load()
    digests, prof = [], None
    try:
        for alg in (hk.HK_PRODUCT_NTT, hk.HK_PRODUCT_TENSOR):
            hk.hk_set_product_algorithm(alg)
            with hk.Hankel(0) as h:
                h.moments(1, b, N, bits)
                hk.hk_set_profiling(h.ctx, True)
                h.ldlt()
                prof = hk.hk_get_profile(h.ctx)
                digests.append(factor_digest(h, hk, N))
    finally:
        hk.hk_set_product_algorithm(hk.HK_PRODUCT_AUTO)
    assert digests[0] == digests[1]
    items = sum(hk_items(N, i) for i in range(N - 1) if N - 1 - i >= hk.HK_TC_MIN_ROWS)
    assert prof["tc_launches"] > 0
    if rerun == "most":
        assert prof["tc_redo_items"] > 0.5 * items, (prof["tc_redo_items"], items)
    else:
        assert prof["tc_redo_items"] < 0.05 * items, (prof["tc_redo_items"], items)


def hk_items(N, i):
    """128-row items of step i of the tensor-core trailing update."""
    m, s, kt = N - 1 - i, 0, 0
    while m - 1 > 128 * kt:
        s += m - 128 * kt
        kt += 1
    return s


@pytest.mark.parametrize("plan", [None, 32, 16])
def test_tensor_full_factor_golden(plan):
    """beta = 1/2, N = 1024, 8192 bits: the whole factor and X against the
    oracle's digests (tests/golden/c5_1024_8192.json), tensor-core updates in
    the 767 steps with at least 256 trailing rows.  plan = 32: Algorithm 4
    runs inside those launches (hk_plan_block) and hk_inv_block(32) finishes
    it; a second hk_inv_block(32) starts again from the identity.  plan = 16:
    the planned k differs from the one asked for, and hk_inv_block runs every
    step itself."""
    import json
    import os
    import paper_1810_01478_gb300 as hk
    from tests.digest import factor_digest, x_digest
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "c5_1024_8192.json")
    gd = json.load(open(path))
    hk.load()
    try:
        hk.hk_set_product_algorithm(hk.HK_PRODUCT_TENSOR)
        with hk.Hankel(0) as h:
            h.moments(1, 2, 1024, 8192)
            h.ldlt(k=plan)
            h.inv_block(32)
            assert factor_digest(h, hk, 1024) == gd["factor_sha256"]
            assert x_digest(h, hk, 1024, 32) == gd["x_sha256"]
            if plan == 32:
                h.inv_block(32)
                assert x_digest(h, hk, 1024, 32) == gd["x_sha256"]
    finally:
        hk.hk_set_product_algorithm(hk.HK_PRODUCT_AUTO)
