"""a8 at a rational beta = a/b (a > 1): d lambda_1 / d beta from the device's
digamma values psi((s+1) b / a), built from the constants psi(r/a),
r = 1..a-1, by the recurrence psi(x + 1) = psi(x) + 1/x (Sec. 4.2's
moments differentiated in beta).  Compared with the oracle's analytic
gradient (oracle.grad.analytic_grad: mpmath's digamma at every x, mpmath's
Gamma for mu) on the factor of the same moments, to 1e-40, at a schoolbook
width (2048 bits) and at an NTT width (8192 bits), and at beta = 11/20
(ten constants) with N = 64, k = 16, 4096 bits; the psi constants are
handed over wider and narrower than the working width.  The oracle's psi
at rational points is Gauss's digamma theorem after the same recurrence
(pinned against mpmath.digamma on the CPU), and its mu are the oracle's
Gamma(r/a) constants (12416 bits) times the exact rational factor."""
import math
from fractions import Fraction

import numpy as np
import pytest

mpm = pytest.importorskip("mpmath")

from oracle import grad as GR
from oracle import moments as OM
from oracle import mpfloat as F
from oracle import pipeline as PL
from tests.layout import to_arrays
from tests.test_gpu_moments_gamma import as_limbs, constants

pytestmark = pytest.mark.gpu
TOL = mpm.mpf(10) ** -40


def psi_constants(a, nc):
    """psi(r/a), r = 1..a-1, truncated to nc limbs (the oracle's format)."""
    out = []
    with mpm.workprec(32 * nc + 256):
        for r in range(1, a):
            v = GR.psi_gauss(r, a, mpm)
            man, exp = v.man_exp                  # |v| = man 2^exp
            q = Fraction(int(man)) * (Fraction(2) ** int(exp)) * (-1 if v < 0 else 1)
            out.append(F.from_fraction(q, nc))
    return to_arrays(out, nc)


@pytest.mark.parametrize("beta,N,k,bits,dn", [(Fraction(9, 20), 40, 8, 2048, 4), (Fraction(9, 20), 40, 8, 8192, -2),
                                               (Fraction(11, 20), 64, 16, 4096, 0)])
def test_grad_rational_beta_vs_oracle(beta, N, k, bits, dn):
    import paper_1810_01478_gb300 as hk
    n = bits // 32
    a, b = beta.numerator, beta.denominator
    consts = constants(beta)
    ce, cl = as_limbs(consts)
    mu = OM.moments_from_constants(beta, N, n, consts)
    ref = PL.run(beta, N, k, n, n_eig=1, mu=mu)

    def mu_exact(s):
        q, r = divmod(b * (s + 1), a)
        g = Fraction(math.factorial(q - 1)) if r == 0 else consts[r]
        for i in range(q if r else 0):
            g *= Fraction(r + i * a, a)
        g *= Fraction(b, a)
        return mpm.mpf(g.numerator) / g.denominator

    want, lam_want, _ = GR.analytic_grad(beta, mu_exact, ref["L"], ref["D"], ref["X"], k, n)
    ps, pe, pm = psi_constants(a, n + dn)
    with hk.Hankel(0) as h:
        h.moments_gamma(a, b, N, bits, ce, cl)
        h.ldlt()
        h.inv_block(k)
        h.lambda1(1)
        h.set_psi_constants(ps, pe, pm)
        gs, ge, gm, gf = h.lambda1_grad()
    with mpm.workprec(2 * bits + 64):
        got = F.to_mpf(F.from_limbs(int(gs[0]), int(ge[0]), gm[0]), mpm)
        assert abs(got - want) / abs(want) < TOL
        assert abs(gf[0] - float(want)) <= 1e-15 * abs(float(want))


@pytest.mark.parametrize("count", [None, 3])
def test_grad_rational_beta_needs_psi_constants(count):
    """Without the a - 1 constants (none, or too few) the gradient at
    beta = 9/20 is HK_ERR_UNSUPPORTED (an error of the context, which stays
    sticky)."""
    import paper_1810_01478_gb300 as hk
    beta, N, bits = Fraction(9, 20), 8, 1024
    ce, cl = as_limbs(constants(beta))
    with hk.Hankel(0) as h:
        h.moments_gamma(9, 20, N, bits, ce, cl)
        h.ldlt()
        h.inv_block(4)
        h.lambda1(1)
        if count:
            ps, pe, pm = psi_constants(9, bits // 32)
            h.set_psi_constants(ps[:count], pe[:count], pm[:count])
        with pytest.raises(hk.HKError) as ei:
            h.lambda1_grad()
        assert ei.value.status == hk.HK_ERR_UNSUPPORTED
