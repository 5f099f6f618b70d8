"""The batched form (hk_batch_run): 16 instances of uneven size solved
concurrently, beta in {9/20, 1/2, 11/20, 1} x N in {128, 192, 256, 384},
k = 16, 32 N bits each.  Every instance must give exactly the lambda of the
plain single-instance path (same kernels, bit for bit) and match the oracle
to 1e-40.  Moments: on the device; for 9/20 and 11/20 from the constants
Gamma(r/a) (hk_moments_gamma), the oracle's own stored constants, and the
single-instance path imports the oracle's moments formed from them (so the
two routes to the moments are compared too).
"""
import json
import os
from fractions import Fraction

import pytest

mpm = pytest.importorskip("mpmath")

from oracle import mpfloat as F
from tests.layout import to_arrays
from tests.test_gpu_moments_gamma import as_limbs

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))
BETAS = [(9, 20), (1, 2), (11, 20), (1, 1)]
NS = [128, 192, 256, 384]


def constants(beta):
    path = os.path.join(HERE, "golden", "c3_gamma_constants.json")
    if not os.path.exists(path):
        pytest.skip("c3 constants not generated")
    d = json.load(open(path))["constants"][f"{beta.numerator}/{beta.denominator}"]
    return [None] + [Fraction(int(p, 16), int(q, 16)) for p, q in d[1:]]


def problems(ns=NS, betas=BETAS):
    from oracle import moments as OM
    out = []
    for a, b in betas:
        for N in ns:
            bits = 32 * N
            p = dict(beta=(a, b), N=N, k=16, bits=bits, n_eig=1)
            if a != 1:
                beta = Fraction(a, b)
                p["gamma"] = as_limbs(constants(beta))
                p["mu_oracle"] = to_arrays(OM.moments_from_constants(beta, N, bits // 32, constants(beta)),
                                           bits // 32)
            out.append(p)
    return out


def single(hk, p):
    with hk.Hankel(0) as h:
        if "mu_oracle" in p:
            h.set_moments(p["N"], p["bits"], *p["mu_oracle"], p["beta"][0], p["beta"][1])
        else:
            h.moments(p["beta"][0], p["beta"][1], p["N"], p["bits"])
        h.ldlt()
        h.inv_block(p["k"])
        return h.lambda1(1)


def test_batched_config3_matches_single_path_and_oracle():
    import paper_1810_01478_gb300 as hk
    hk.load()
    probs = problems()
    st, res = hk.hk_batch_run(0, probs, max_concurrent=16)
    assert st == hk.HK_OK, [(r["status"], r["message"]) for r in res if r["status"]]
    for p, r in zip(probs, res):
        s, e, m, f64, _ = single(hk, p)
        bs, be, bm = r["lambda"]
        assert int(bs[0]) == int(s[0]) and int(be[0]) == int(e[0]) and (bm[0] == m[0]).all(), p["beta"]
        gpath = os.path.join(HERE, "golden", "c3_%d_%d_%d.json" % (p["beta"][0], p["beta"][1], p["N"]))
        if os.path.exists(gpath):
            with mpm.workprec(2 * p["bits"]):
                want = mpm.mpf(json.load(open(gpath))["lambdas"][0])
                got = F.to_mpf(F.from_limbs(int(bs[0]), int(be[0]), bm[0]), mpm)
                assert abs(got - want) / want < mpm.mpf(10) ** -40, (p["beta"], p["N"])


def test_batch_rejects_bad_instances():
    import paper_1810_01478_gb300 as hk
    hk.load()
    st, _ = hk.hk_batch_run(0, [dict(beta=(1, 2), N=10, k=20, bits=4096)])
    assert st == hk.HK_ERR_ARG
