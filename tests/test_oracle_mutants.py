"""The pins catch plausible mistakes: each test plants one mistake in the
oracle (on the CPU, through monkeypatch, for the duration of the test) and
checks that a pin of tests/test_oracle_pins.py or test_oracle_format.py then
fails.  A pin that still passed would not be pinning that part of the oracle.

Mistakes planted: the sign of the fused update, a double rounding in it, a
quotient through a rounded reciprocal, round-to-nearest instead of
truncation, an off-by-one moment index, a pivot that misses its updates,
Algorithm 4 without the negated column or without its last term, the block
without 1/D, the smallest eigenvalue instead of the largest, a sign error in
Gauss's digamma theorem, a gradient with the wrong sign of psi, a floor
where the loss estimate takes a ceiling, a harmonic number one index too
far, a missing 1/a in the Gamma-constant route to the moments, the loss
estimate against mu_i instead of mu_2i, truncation errors of the wrong sign,
and an entry sample that takes the wrong row."""
from fractions import Fraction
from math import factorial

import pytest

mpm = pytest.importorskip("mpmath")

from oracle import eigen as EG
from oracle import grad as GR
from oracle import invblock as IB
from oracle import ldlt as LD
from oracle import moments as M
from oracle import mpfloat as F
from oracle import precision as PR
from tests import test_oracle_format as TF
from tests import test_oracle_pins as TP


def caught(pin, *args):
    """True when one of the pin's assertions fails (any other error, such as
    a mutant with the wrong signature, propagates and fails the test)."""
    try:
        pin(*args)
    except AssertionError:
        return True
    return False


def test_pins_pass_unmutated():
    for pin, args in ((TF.test_fused_property, (4,)), (TP.test_ldlt_beta1_closed_forms, ()),
                      (TP.test_partial_inverse_beta1_closed_form, ()),
                      (TP.test_block_is_top_left_of_exact_inverse, ()),
                      (TP.test_loss_estimate_closed_form_beta1, ())):
        assert not caught(pin, *args), pin.__name__


def test_fused_sign(monkeypatch):
    orig = F.fused
    monkeypatch.setattr(F, "fused", lambda a, x, y, n: orig(a, F.neg(x), y, n))  # a + x y
    assert caught(TF.test_fused_property, 4)
    assert caught(TP.test_ldlt_beta1_closed_forms)


def test_fused_double_rounding(monkeypatch):
    monkeypatch.setattr(F, "fused", lambda a, x, y, n: F.add(a, F.neg(F.mul(x, y, n)), n))
    assert caught(TF.test_fused_property, 4)


def test_division_through_rounded_reciprocal(monkeypatch):
    orig = F.div
    monkeypatch.setattr(F, "div", lambda a, d, n: F.mul(a, orig(F.from_int(1, n), d, n), n))
    assert caught(TF.test_div_mul_add_property, 4)


def test_round_to_nearest(monkeypatch):
    orig = F.rnd

    def rnd_nearest(v, e, n):
        a = abs(v)
        limbs = (a.bit_length() + 31) // 32
        if limbs > n:
            sh = 32 * (limbs - n)
            a += 1 << (sh - 1)
        return orig(a if v >= 0 else -a, e, n)
    monkeypatch.setattr(F, "rnd", rnd_nearest)
    assert caught(TF.test_rnd_and_from_fraction, 2)


def test_moment_index_off_by_one(monkeypatch):
    monkeypatch.setattr(M, "moment_exact", lambda j, m: m * factorial(m * (j + 2) - 1))
    assert caught(TP.test_moments_closed_forms_and_gamma)


def test_pivot_without_updates(monkeypatch):
    orig = LD.ldlt_subset

    def stale_pivots(mu, idx, n):
        D, L = orig(mu, idx, n)
        return [mu[2 * i] for i in idx], L                       # d_i = H[i][i] as given
    monkeypatch.setattr(LD, "ldlt_subset", stale_pivots)
    assert caught(TP.test_ldlt_beta1_closed_forms)


def _alg4(L, N, k, n, negate=True, last_term=True):
    k = min(k, N)
    X = [[F.ZERO] * k for _ in range(N)]
    for c in range(k):
        X[c][c] = IB.one(n)
    for i in range(N):
        for j in range(i + 1, N):
            f = L[j][i]
            if i < k:
                X[j][i] = F.neg(f) if negate else f
            for c in range(min(k, i) - (0 if last_term else 1)):
                X[j][c] = F.fused(X[j][c], f, X[i][c], n)
    return X


def test_alg4_without_negation(monkeypatch):
    monkeypatch.setattr(IB, "partial_inverse", lambda L, N, k, n: _alg4(L, N, k, n, negate=False))
    assert caught(TP.test_partial_inverse_beta1_closed_form)


def test_alg4_dropped_term(monkeypatch):
    monkeypatch.setattr(IB, "partial_inverse", lambda L, N, k, n: _alg4(L, N, k, n, last_term=False))
    assert caught(TP.test_partial_inverse_beta1_closed_form)


def test_block_without_pivots(monkeypatch):
    orig = IB.inverse_block
    monkeypatch.setattr(IB, "inverse_block",
                        lambda X, D, k, n, mp=None: orig(X, [F.from_int(1, n)] * len(D), k, n, mp))
    assert caught(TP.test_block_is_top_left_of_exact_inverse)


def test_smallest_block_eigenvalue(monkeypatch):
    orig = EG.block_eigs

    def ascending(S, mp):
        ev, vec = orig(S, mp)
        return ev[::-1], vec[::-1]
    monkeypatch.setattr(EG, "block_eigs", ascending)
    assert caught(TP.test_full_block_gives_true_smallest_eigenvalue)


def test_gauss_digamma_cot_sign(monkeypatch):
    def wrong(r, m, mp):
        v = -mp.euler - mp.log(2 * m) + mp.pi / 2 * mp.cot(mp.pi * r / m)   # + instead of -
        for j in range(1, (m - 1) // 2 + 1):
            v += 2 * mp.cos(2 * mp.pi * j * r / m) * mp.log(mp.sin(mp.pi * j / m))
        return v
    monkeypatch.setattr(GR, "psi_gauss", wrong)
    assert caught(TP.test_psi_integer_identity_matches_digamma)


def test_gradient_psi_sign(monkeypatch):
    orig = GR.psi
    monkeypatch.setattr(GR, "psi", lambda x, mp: -orig(x, mp))
    assert caught(TP.test_gradient_analytic_vs_finite_difference)


def test_loss_estimate_floor(monkeypatch):
    def floor_log2(q):
        t = q.numerator.bit_length() - q.denominator.bit_length()
        while Fraction(2) ** t > q:
            t -= 1
        while Fraction(2) ** (t + 1) <= q:
            t += 1
        return t
    monkeypatch.setattr(PR, "ceil_log2", floor_log2)
    assert caught(TP.test_loss_estimate_closed_form_beta1)


def test_harmonic_index_off_by_one(monkeypatch):
    orig = GR.psi

    def psi_h(x, mp):
        v = orig(x, mp)
        if isinstance(x, int) or (isinstance(x, Fraction) and x.denominator == 1):
            v += mp.mpf(1) / int(x)                          # H_x instead of H_{x-1}
        return v
    monkeypatch.setattr(GR, "psi", psi_h)
    assert caught(TP.test_psi_integer_identity_matches_digamma)


def test_gamma_route_missing_factor(monkeypatch):
    def moments_wrong(beta, N, n, consts):
        beta = Fraction(beta)
        a, b = beta.numerator, beta.denominator
        mus = []
        for j in range(2 * N - 1):
            q, r = divmod(b * (j + 1), a)
            if r == 0:
                v = Fraction(b, a) * factorial(q - 1)
            else:
                num = b
                for i in range(q):
                    num *= r + i * a
                v = Fraction(num, a ** q) * consts[r]          # a^q for a^(q+1)
            mus.append(F.from_fraction(v, n))
        return mus
    monkeypatch.setattr(M, "moments_from_constants", moments_wrong)
    assert caught(TP.test_rational_beta_moments_from_constants)


def test_loss_estimate_wrong_moment(monkeypatch):
    def loss_wrong(mu, D):
        best = 0
        for i, d in enumerate(D):
            best = max(best, PR.ceil_log2(F.to_fraction(mu[i]) / F.to_fraction(d)))   # mu_i for mu_2i
        return best
    monkeypatch.setattr(PR, "loss_estimate", loss_wrong)
    assert caught(TP.test_loss_estimate_closed_form_beta1)


def test_truncation_error_sign(monkeypatch):
    orig = EG.lambdas

    def flipped(S, n_eig=3, prec=None):
        lam, err, ev, vec = orig(S, n_eig, prec)
        return lam, [None if e is None else -e for e in err], ev, vec   # lambda(k-1) - lambda(k)
    monkeypatch.setattr(EG, "lambdas", flipped)
    assert caught(TP.test_interlacing_and_precision_doubling)


def test_subset_sampling_forgets_the_row(monkeypatch):
    orig = LD.sample_entry

    def sample_wrong(mu, r, c, n):
        if r == c:
            return orig(mu, r, c, n)
        D, L = LD.ldlt_subset(mu, list(range(c + 2)), n)              # row c + 1 for row r
        return L[c + 1][c]
    monkeypatch.setattr(LD, "sample_entry", sample_wrong)
    assert caught(TP.test_subset_sampling_reproduces_full_factor)
