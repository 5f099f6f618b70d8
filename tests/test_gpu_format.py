"""GPU parity of the number-format primitives against the oracle, bit for bit.

hk_fused_batch computes trunc(a - x*y) and hk_div_batch trunc(a/d) on the
device; the oracle's mpfloat.fused / mpfloat.div are the reference.  Operands
come from tests/inputs.fused_operands: random and structured mantissas,
near-total cancellation, exponent gaps beyond the combine frame (sticky
cases) and zeros, at widths of 1, 4 and 24 limbs per lane, with both exact
product algorithms (schoolbook limb products and the three-prime NTT).
"""
import random

import pytest

from oracle import mpfloat as F
from tests import inputs
from tests.layout import DevNums

pytestmark = pytest.mark.gpu


def first_mismatch(got, want, ops):
    for i, (g, w) in enumerate(zip(got, want)):
        if g != w:
            return i, ops[i], g, w
    return None


SCHOOLBOOK, NTT = 1, 2


@pytest.mark.parametrize("product_algorithm", [SCHOOLBOOK, NTT], indirect=True)
@pytest.mark.parametrize("M", [1, 2, 3, 4, 5, 7, 12, 16, 24])
def test_fused_batch_bit_exact(M, product_algorithm):
    import torch
    import paper_1810_01478_gb300 as hk
    n = 32 * M
    rng = random.Random(1000 + M)
    ops = inputs.fused_operands(rng, n, 700 if M < 24 else 300)
    a, x, y = (list(t) for t in zip(*ops))
    A, X, Y = DevNums(a, n=n), DevNums(x, n=n), DevNums(y, n=n)
    OUT = DevNums(count=len(ops), n=n)
    hk.hk_fused_batch(32 * n, len(ops), A.ptrs, X.ptrs, Y.ptrs, OUT.ptrs, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    got = OUT.to_host()
    want = [F.fused(*t, n) for t in ops]
    assert first_mismatch(got, want, ops) is None


@pytest.mark.parametrize("M", [1, 4, 24])
def test_div_batch_bit_exact(M):
    import torch
    import paper_1810_01478_gb300 as hk
    n = 32 * M
    rng = random.Random(2000 + M)
    cnt = 300 if M < 24 else 100
    a = [inputs.rand_num(rng, n, kinds=inputs.KINDS) for _ in range(cnt)]
    d = [inputs.rand_num(rng, n, kinds=inputs.KINDS) for _ in range(cnt)]
    a[0] = (0, 0)
    d[1] = (1 << (32 * n - 32), 3)            # power of two: the clamped reciprocal
    d[2] = ((1 << (32 * n)) - 1, -2)          # all ones
    a[3] = d[3]                               # exact quotient 1
    A, D = DevNums(a, n=n), DevNums(d, n=n)
    OUT = DevNums(count=cnt, n=n)
    hk.hk_div_batch(32 * n, cnt, A.ptrs, D.ptrs, OUT.ptrs, torch.cuda.current_stream().cuda_stream)
    got = OUT.to_host()
    want = [F.div(a[i], d[i], n) for i in range(cnt)]
    assert first_mismatch(got, want, list(zip(a, d))) is None
