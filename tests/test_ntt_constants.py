"""Host-side checks of the constants behind the NTT products (no GPU).

The exact products of the wide formats are cyclic convolutions modulo three
primes recombined by the Chinese remainder theorem.  They are exact only if
every prime is prime, has roots of unity of every length the library uses
(2^a and 3 2^a up to 3 2^11), keeps the lazy-reduction ranges inside 32 bits
(p < 2^30), satisfies Garner's ordering (p1 > p2 > p3, p1 < 2 p3), and the
product p1 p2 p3 exceeds every convolution coefficient (n 2^64 at n = 1024
limbs).  The constants are read from the library source as text.
"""
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "paper_1810_01478_gb300", "csrc", "hk_abi.cu")


def _array(name):
    text = open(SRC).read()
    m = re.search(name + r"\[NTT_Q\]\s*=\s*\{([^}]*)\}", text)
    assert m, name
    return [int(v.strip().rstrip("u")) for v in m.group(1).split(",")]


def _is_prime(p):
    if p < 2:
        return False
    d, s = p - 1, 0
    while d % 2 == 0:
        d //= 2
        s += 1
    for a in (2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37):
        x = pow(a, d, p)
        if x in (1, p - 1):
            continue
        for _ in range(s - 1):
            x = x * x % p
            if x == p - 1:
                break
        else:
            return False
    return True


def _factors(m):
    out, f = set(), 2
    while f * f <= m:
        while m % f == 0:
            out.add(f)
            m //= f
        f += 1
    if m > 1:
        out.add(m)
    return out


def test_primes_roots_and_ranges():
    ps, gs = _array("kPrimes"), _array("kGen")
    assert len(ps) == 3 and len(gs) == 3
    for p, g in zip(ps, gs):
        assert _is_prime(p) and p < 2 ** 30
        assert (p - 1) % (3 * 2 ** 11) == 0
        # g generates the whole multiplicative group
        assert all(pow(g, (p - 1) // f, p) != 1 for f in _factors(p - 1))
    p1, p2, p3 = ps
    assert p1 > p2 > p3 and p1 < 2 * p3
    assert p1 * p2 * p3 > 1024 * 2 ** 64


def test_binding_threshold_matches_header():
    import paper_1810_01478_gb300 as hk
    text = open(os.path.join(ROOT, "include", "hk.h")).read()
    m = re.search(r"#define HK_NTT_AUTO_MIN_M (\d+)", text)
    assert m and int(m.group(1)) == hk.HK_NTT_AUTO_MIN_M


def test_tensor_core_constants_match_the_header():
    """The Python binding's copies of the tensor-core thresholds are the header's."""
    import re
    import paper_1810_01478_gb300 as hk
    text = open(os.path.join(ROOT, "include", "hk.h")).read()
    for name in ("HK_TC_MIN_M", "HK_TC_AUTO_MIN_M", "HK_TC_MIN_ROWS", "HK_PRODUCT_TENSOR"):
        m = re.search(r"#define %s (\d+)" % name, text)
        assert m and int(m.group(1)) == getattr(hk, name), name


def test_bench_short_product_cut_matches_the_kernel():
    """bench.tc_cut restates TcShape::QCUT (csrc/tc.cuh) for the roofline's
    algorithmic work: the same guard and the same formula at every width."""
    import re
    import sys
    sys.path.insert(0, ROOT)
    import bench
    text = open(os.path.join(ROOT, "paper_1810_01478_gb300", "csrc", "tc.cuh")).read()
    guard = int(re.search(r"static constexpr int GUARD = (\d+);", text).group(1))
    assert re.search(r"static constexpr int QCUT = 32 \* \(\(n - GUARD - 2\) / 7\);", text)
    for M in (8, 12, 16, 24):
        n = 32 * M
        assert bench.tc_cut(n) == 32 * ((n - guard - 2) // 7)
