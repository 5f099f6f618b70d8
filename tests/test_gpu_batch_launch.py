"""hk_ldlt_batch: Algorithm 1 (Sec. 4.3) for several instances of one width
in one persistent launch.

* Every factor is bit-identical to the oracle's (stored whole-factor digests
  at N = 512 and 768, 4096 bits, and N = 256, 8192 bits) or, for instances
  without a stored digest, to hk_ldlt's on the same moments, across uneven
  N (1, 2, 33, 130 ...) and several beta.
* Instances planned with a block size k (hk_plan_block) also run Algorithm 4
  inside the launch: X = L^-1[:, :k] is bit-identical to the oracle's
  (stored X digests, k = 32 at N = 512 and k = 16 at N = 256, 8192 bits) or
  to the single path's (hk_ldlt, then hk_inv_block(k)).
* A non-positive pivot (moments all 1: H is the rank-one all-ones matrix,
  so d_1 = 0) ends that instance only, with HK_ERR_NOT_PD; the others in the
  same launch are unaffected.
* An idle-wait limit of zero makes the launch give up at once (nothing is
  claimable while each instance's first reciprocal runs) and every instance
  reports HK_ERR_TIMEOUT; the device then runs a fresh batch correctly.
"""
import json
import os

import pytest

from tests.digest import factor_digest, x_digest

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


def golden(name):
    path = os.path.join(HERE, "golden", name + ".json")
    if not os.path.exists(path):
        pytest.skip(name + " not generated")
    return json.load(open(path))


def single_digest(hk, beta, N, bits):
    with hk.Hankel(0) as r:
        r.moments(beta[0], beta[1], N, bits)
        r.ldlt()
        return factor_digest(r, hk, N)


def single_x_digest(hk, beta, N, bits, k):
    with hk.Hankel(0) as r:
        r.moments(beta[0], beta[1], N, bits)
        r.ldlt()
        r.inv_block(k)
        return x_digest(r, hk, N, k)


def run_batch(hk, specs, limit=-1.0):
    """specs: (beta, N, bits, golden name or None[, planned k])"""
    hs = []
    for spec in specs:
        beta, N, bits = spec[:3]
        h = hk.Hankel(0)
        h.moments(beta[0], beta[1], N, bits)
        if len(spec) > 4 and spec[4]:
            hk.hk_plan_block(h.ctx, spec[4])
        hs.append(h)
    hk.hk_ldlt_batch([h.ctx for h in hs], limit)
    return hs


@pytest.mark.parametrize("width", [1024, 3072, 4096, 8192])
def test_batch_launch_factors_are_bit_exact(width):
    import paper_1810_01478_gb300 as hk
    hk.load()
    if width in (1024, 3072):  # odd limbs per lane: scalar loads
        specs = [((1, 2), 48, width, None, 8), ((1, 3), 17, width, None, 0), ((1, 1), 1, width, None, 0),
                 ((1, 4), 40, width, None, 40)]
    elif width == 4096:
        specs = [((1, 2), 512, 4096, "c5_512_4096", 32), ((1, 3), 64, 4096, None, 8), ((1, 1), 1, 4096, None, 1),
                 ((1, 2), 768, 4096, "c5_768_4096", 0), ((1, 2), 33, 4096, None, 33), ((1, 4), 130, 4096, None, 0),
                 ((1, 2), 2, 4096, None, 2)]
    else:
        specs = [((1, 2), 256, 8192, "c2", 16), ((1, 1), 100, 8192, None, 5), ((1, 3), 31, 8192, None, 0)]
    hs = run_batch(hk, specs)
    try:
        for (beta, N, bits, g, k), h in zip(specs, hs):
            got = factor_digest(h, hk, N)
            want = golden(g)["factor_sha256"] if g else single_digest(hk, beta, N, bits)
            assert got == want, (beta, N, bits)
            if k:
                h.inv_block(k)
                gx = golden(g) if g else None
                want_x = gx["x_sha256"] if gx and gx["k"] == k else single_x_digest(hk, beta, N, bits, k)
                assert x_digest(h, hk, N, k) == want_x, (beta, N, bits, k)
    finally:
        for h in hs:
            h.close()


def test_batch_launch_non_pd_instance_ends_alone():
    import paper_1810_01478_gb300 as hk
    from oracle import mpfloat as F
    from tests.layout import to_arrays
    hk.load()
    N, bits = 40, 4096
    ones = to_arrays([F.from_int(1, bits // 32)] * (2 * N - 1), bits // 32)
    good = [((1, 2), 48), ((1, 3), 40)]
    hs = []
    for beta, n_ in good:
        h = hk.Hankel(0)
        h.moments(beta[0], beta[1], n_, bits)
        hs.append(h)
    bad = hk.Hankel(0)
    bad.set_moments(N, bits, *ones)
    try:
        hk.hk_ldlt_batch([hs[0].ctx, bad.ctx, hs[1].ctx])
        with pytest.raises(hk.HKError) as ei:
            bad.export(hk.HK_D, 0, N)
        assert ei.value.status == hk.HK_ERR_NOT_PD
        for (beta, n_), h in zip(good, hs):
            assert factor_digest(h, hk, n_) == single_digest(hk, beta, n_, bits)
    finally:
        bad.close()
        for h in hs:
            h.close()


def test_batch_launch_wait_limit_reports_timeout_and_device_recovers():
    import paper_1810_01478_gb300 as hk
    hk.load()
    specs = [((1, 2), 64, 4096, None), ((1, 3), 80, 4096, None, 16), ((1, 1), 72, 4096, None)]
    hs = run_batch(hk, specs, limit=0.0)
    try:
        for (beta, N, bits, *_), h in zip(specs, hs):
            with pytest.raises(hk.HKError) as ei:
                h.export(hk.HK_D, 0, N)
            assert ei.value.status == hk.HK_ERR_TIMEOUT
    finally:
        for h in hs:
            h.close()
    hs = run_batch(hk, specs)
    try:
        for (beta, N, bits, *_), h in zip(specs, hs):
            assert factor_digest(h, hk, N) == single_digest(hk, beta, N, bits)
    finally:
        for h in hs:
            h.close()


def test_batch_launch_rejects_mixed_widths_and_duplicates():
    import paper_1810_01478_gb300 as hk
    hk.load()
    with hk.Hankel(0) as a, hk.Hankel(0) as b:
        a.moments(1, 2, 16, 4096)
        b.moments(1, 2, 16, 2048)
        with pytest.raises(hk.HKError) as ei:
            hk.hk_ldlt_batch([a.ctx, b.ctx])
        assert ei.value.status == hk.HK_ERR_ARG
    with hk.Hankel(0) as a:
        a.moments(1, 2, 16, 4096)
        with pytest.raises(hk.HKError) as ei:
            hk.hk_ldlt_batch([a.ctx, a.ctx])
        assert ei.value.status == hk.HK_ERR_ARG
    with hk.Hankel(0) as a, hk.Hankel(0) as b:
        a.moments(1, 2, 16, 12288)
        b.moments(1, 3, 16, 12288)
        with pytest.raises(hk.HKError) as ei:
            hk.hk_ldlt_batch([a.ctx, b.ctx])
        assert ei.value.status == hk.HK_ERR_UNSUPPORTED


def test_tuner_picks_a_shape_and_batches_stay_exact():
    import paper_1810_01478_gb300 as hk
    hk.load()
    b, g, t = hk.hk_tune_batch(0, 2048, 48, 6)
    assert b in (1, 2, 3, 4, 6, 8, 12, 16) and g in (1, 4, 8, 16) and t > 0
    # a later batch whose largest N is in the same bucket takes the tuned shape
    specs = [((1, 2), 40, 2048, None), ((1, 3), 48, 2048, None), ((1, 1), 7, 2048, None)]
    hs = run_batch(hk, specs)
    try:
        for (beta, N, bits, _), h in zip(specs, hs):
            assert factor_digest(h, hk, N) == single_digest(hk, beta, N, bits)
    finally:
        for h in hs:
            h.close()
