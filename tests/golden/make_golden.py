"""Writes the oracle's expected values for workloads too slow to run inside a test.

Calls only ``oracle/``.  Each target runs the oracle pipeline (moments ->
Algorithm 1 -> Algorithm 4 -> block -> eigenvalues, and the gradient where
asked) and stores, in tests/golden/<name>.json:
  lambdas / trunc_errors  as decimal strings (80 significant digits)
  grad, grad_fd           analytic d lambda_1/d beta and the central
                          difference at beta +- 1e-30 (where asked)
  factor_sha256           SHA-256 of the packed factor in the library's export
                          order: for c in 0..N-1, r in c..N-1 the entry
                          (D_c on the diagonal, L[r][c] below) as int32 sign,
                          int32 exp, n uint32 limbs, all little endian
  x_sha256                the same for X (row major N x k)
Usage:  python tests/golden/make_golden.py <target> [<target> ...]
Targets: c1, c2, c5_512_4096, c5_768_4096, c5_1024_4096, c5_1024_8192,
         w_256_24576, w_160_16384, w_320_24576 (whole factors at 24576 and
         16384 bits), r_<a>_<b>_<N> (beta = a/b at N = 128, 256: the regimes),
         c3const (Gamma(r/a) constants for beta = 9/20, 11/20),
         c3_<a>_<b>_<N> (one batched-config instance; beta = a/b, k = 16,
         bits = 32 N, non-dyadic moments from the stored constants)
"""
import hashlib
import json
import os
import struct
import sys
import time
from fractions import Fraction

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import mpfloat as F       # noqa: E402
from oracle import pipeline as PL     # noqa: E402
from oracle import grad as GR         # noqa: E402

TARGETS = {
    "c1": dict(beta=(1, 2), N=48, k=8, bits=4096, grad=True, fd=False),
    "c2": dict(beta=(1, 2), N=256, k=16, bits=8192, grad=True, fd=True),
    "c5_512_4096": dict(beta=(1, 2), N=512, k=32, bits=4096, grad=False, fd=False),
    "c5_768_4096": dict(beta=(1, 2), N=768, k=32, bits=4096, grad=False, fd=False),
    "c5_1024_4096": dict(beta=(1, 2), N=1024, k=32, bits=4096, grad=True, fd=False),
    "c5_1024_8192": dict(beta=(1, 2), N=1024, k=32, bits=8192, grad=False, fd=False),
    # whole factors at the widest product widths the library runs (M = 24, 16)
    "w_256_24576": dict(beta=(1, 2), N=256, k=32, bits=24576, grad=True, fd=False),
    "w_160_16384": dict(beta=(1, 2), N=160, k=32, bits=16384, grad=True, fd=False),
    # N > 256: the first steps of Algorithm 1 have at least 256 trailing rows
    "w_320_24576": dict(beta=(1, 2), N=320, k=32, bits=24576, grad=False, fd=False),
    # the regimes of the weight away from beta = 1/2 (k = 64, as bench.py --workload regimes)
    "r_1_3_128": dict(beta=(1, 3), N=128, k=64, bits=2048, grad=False, fd=False),
    "r_1_3_256": dict(beta=(1, 3), N=256, k=64, bits=2048, grad=False, fd=False),
    "r_1_1_128": dict(beta=(1, 1), N=128, k=64, bits=2048, grad=False, fd=False),
    "r_1_1_256": dict(beta=(1, 1), N=256, k=64, bits=2048, grad=False, fd=False),
}


def num_bytes(x, n):
    s, e, limbs = F.limbs_of(x, n)
    return struct.pack("<ii", s, e) + struct.pack("<%dI" % n, *limbs)


def factor_digest(D, L, N, n):
    h = hashlib.sha256()
    for c in range(N):
        for r in range(c, N):
            h.update(num_bytes(D[c] if r == c else L[r][c], n))
    return h.hexdigest()


def x_digest(X, N, k, n):
    h = hashlib.sha256()
    for r in range(N):
        for c in range(k):
            h.update(num_bytes(X[r][c], n))
    return h.hexdigest()


C3_BETAS = [(9, 20), (1, 2), (11, 20), (1, 1)]
C3_NS = [128, 192, 256, 384]
C3_CONST_BITS = 32 * 384 + 128


def c3_bits(N):
    """Working precision of a batched instance: 32 N bits (4096 .. 12288)."""
    return 32 * N


def write_c3_constants():
    from oracle import moments as OM
    out = {}
    for a, b in C3_BETAS:
        if a == 1:
            continue
        consts = OM.gamma_constants(Fraction(a, b), C3_CONST_BITS)
        out[f"{a}/{b}"] = [None] + [[hex(c.numerator), hex(c.denominator)] for c in consts[1:]]
    with open(os.path.join(HERE, "c3_gamma_constants.json"), "w") as f:
        json.dump(dict(bits=C3_CONST_BITS, source="oracle.moments.gamma_constants (mpmath Gamma(r/a))",
                       constants=out), f)


def load_c3_constants(beta):
    d = json.load(open(os.path.join(HERE, "c3_gamma_constants.json")))
    lst = d["constants"][f"{beta.numerator}/{beta.denominator}"]
    return [None] + [Fraction(int(p, 16), int(q, 16)) for p, q in lst[1:]]


def c3_moments(beta, N, n):
    from oracle import moments as OM
    if beta.numerator == 1:
        return OM.moments(beta, N, n)
    return OM.moments_from_constants(beta, N, n, load_c3_constants(beta))


def run_c3(a, b, N):
    import mpmath as mpm
    beta = Fraction(a, b)
    bits = c3_bits(N)
    n = bits // 32
    k = 16
    t0 = time.time()
    mu = c3_moments(beta, N, n)
    r = PL.run(beta, N, k, n, mu=mu)
    out = dict(name=f"c3_{a}_{b}_{N}", beta=[a, b], N=N, k=k, bits=bits,
               source="tests/golden/make_golden.py (oracle only)")
    with mpm.workprec(r["prec"]):
        out["lambdas"] = [mpm.nstr(v, 80) for v in r["lambdas"]]
        out["trunc_errors"] = [mpm.nstr(v, 30) for v in r["trunc_errors"]]
        out["evals"] = [mpm.nstr(v, 30) for v in r["evals"][:4]]
    out["factor_sha256"] = factor_digest(r["D"], r["L"], N, n)
    out["oracle_seconds"] = round(time.time() - t0, 1)
    with open(os.path.join(HERE, out["name"] + ".json"), "w") as f:
        json.dump(out, f, indent=1)
    print(out["name"], "done in", out["oracle_seconds"], "s", flush=True)


def run(name):
    import mpmath as mpm
    if name == "c3const":
        return write_c3_constants()
    if name.startswith("c3_"):
        a, b, N = (int(v) for v in name.split("_")[1:])
        return run_c3(a, b, N)
    cfg = TARGETS[name]
    N, k, bits = cfg["N"], cfg["k"], cfg["bits"]
    n = bits // 32
    beta = Fraction(*cfg["beta"])
    t0 = time.time()
    r = PL.run(beta, N, k, n)
    out = dict(name=name, beta=list(cfg["beta"]), N=N, k=k, bits=bits,
               source="tests/golden/make_golden.py (oracle only)")
    with mpm.workprec(r["prec"]):
        out["lambdas"] = [mpm.nstr(v, 80) for v in r["lambdas"]]
        out["trunc_errors"] = [mpm.nstr(v, 30) for v in r["trunc_errors"]]
    out["factor_sha256"] = factor_digest(r["D"], r["L"], N, n)
    out["x_sha256"] = x_digest(r["X"], N, r["k"], n)
    if cfg["grad"]:
        m = beta.denominator // beta.numerator
        with mpm.workprec(2 * bits + 64):
            g, _, _ = GR.analytic_grad(beta, lambda s: m * mpm.factorial(m * (s + 1) - 1), r["L"], r["D"], r["X"],
                                       r["k"], n)
            out["grad"] = mpm.nstr(g, 80)
    if cfg["fd"]:
        with mpm.workprec(2 * bits + 64):
            out["grad_fd"] = mpm.nstr(GR.fd_grad(beta, N, k, n, h_exp=-30), 80)
    out["oracle_seconds"] = round(time.time() - t0, 1)
    with open(os.path.join(HERE, name + ".json"), "w") as f:
        json.dump(out, f, indent=1)
    print(name, "done in", out["oracle_seconds"], "s", flush=True)


if __name__ == "__main__":
    for t in sys.argv[1:]:
        run(t)
