"""hk_ldlt_noalloc (the allocation-free factorisation) gives the same factor
as hk_ldlt, bit for bit, on calls in a row.

The entry point exists for callers that cannot let a library allocate device
memory; its scratch is one fixed array that every call reuses, so each later
call (a different size and width) also checks that nothing stale from the
one before leaks into the result.  The third call is at 8192 bits, where
hk_ldlt (AUTO) takes NTT products and NTT quotients while hk_ldlt_noalloc
keeps its schoolbook kernels: there the two share no product code.  This
file is collected last on purpose.
"""
import pytest

from tests.layout import DevNums, from_arrays

pytestmark = pytest.mark.gpu


def reference_factor(hk, N, bits):
    with hk.Hankel(0) as h:
        h.moments(1, 2, N, bits)
        mu = from_arrays(*h.export(hk.HK_MU, 0, 2 * N - 1))
        h.ldlt()
        fac = from_arrays(*h.export(hk.HK_FACTOR, 0, N * (N + 1) // 2))
    return mu, fac


def test_ldlt_noalloc_matches_ldlt_on_calls_in_a_row():
    import torch
    import paper_1810_01478_gb300 as hk
    hk.load()
    hk.hk_set_product_algorithm(hk.HK_PRODUCT_AUTO)
    stream = torch.cuda.current_stream().cuda_stream
    for N, bits in [(48, 4096), (33, 2048), (40, 8192)]:
        n = bits // 32
        mu, want = reference_factor(hk, N, bits)
        MU = DevNums(mu, n=n)
        OUT = DevNums(count=N * (N + 1) // 2, n=n)
        hk.hk_ldlt_noalloc(bits, N, MU.ptrs, OUT.ptrs, stream)
        got = OUT.to_host()
        bad = [i for i, (g, w) in enumerate(zip(got, want)) if g != w]
        assert not bad, f"N={N} bits={bits}: {len(bad)} factor entries differ, first {bad[:5]}"


def test_ldlt_noalloc_rejects_sizes_beyond_its_scratch():
    import paper_1810_01478_gb300 as hk
    L = hk.load()
    # N (n + 2) + n + 35 words must fit in HK_NOALLOC_SCRATCH_WORDS (2^20): N = 2000 at 24576 bits does not
    st = L.hk_ldlt_noalloc(24576, 2000, *([None] * 6), None)
    assert st == hk.HK_ERR_ARG
