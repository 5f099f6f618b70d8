"""The C++/OpenMP oracle (oracle/cpp/hk_oracle.cpp) agrees with the Python
oracle bit for bit: its two primitives (the fused update trunc(a - x y) and
the quotient trunc(a / d)) on random, structured, cancelling, far-apart and
zero operands, and whole factors of Algorithm 1 run with the paper's parallel
loop (Sec. 4.3.3) on any number of threads.  It is the all-cores CPU
baseline of bench.py, so it is pinned to the pinned Python oracle here."""
import hashlib
import os
import random
import subprocess
import sys
from fractions import Fraction

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from oracle import build_cpp          # noqa: E402
from oracle import mpfloat as F       # noqa: E402
from oracle import moments as OM      # noqa: E402
from oracle import ldlt as OL         # noqa: E402
from tests import inputs              # noqa: E402


@pytest.fixture(scope="module")
def exe():
    return build_cpp.build()


def enc(x, n):
    s, e, limbs = F.limbs_of(x, n)
    return "%x %x " % (s, e & 0xFFFFFFFF) + " ".join("%x" % v for v in limbs)


def dec(line):
    v = [int(t, 16) for t in line.split()]
    e = v[1] - (1 << 32) if v[1] >= 1 << 31 else v[1]
    return F.from_limbs(v[0], e, v[2:])


def run_prims(exe, n, lines):
    r = subprocess.run([exe, "prims", str(n)], input="\n".join(lines) + "\n", capture_output=True, text=True,
                       check=True)
    return [dec(x) for x in r.stdout.strip().splitlines()]


@pytest.mark.parametrize("n", [32, 96])
def test_primitives_match_python_oracle(exe, n):
    rng = random.Random(77 + n)
    ops = inputs.fused_operands(rng, n, 240)
    got = run_prims(exe, n, ["F " + " ".join(enc(t, n) for t in op) for op in ops])
    assert got == [F.fused(*op, n) for op in ops]
    quo = []
    for _ in range(120):
        a = inputs.rand_num(rng, n, kinds=inputs.KINDS)
        d = inputs.rand_num(rng, n, kinds=inputs.KINDS)
        quo.append((a, d))
    quo += [((0, 0), (3 << (32 * n - 2), 1)), (((1 << (32 * n)) - 1, 0), (1 << (32 * n - 1), 4)),
            ((5 << (32 * n - 4), -2), (5 << (32 * n - 4), -2)), ((1 << (32 * n - 1), 0), ((1 << (32 * n)) - 1, 0))]
    got = run_prims(exe, n, ["Q " + enc(a, n) + " " + enc(d, n) for a, d in quo])
    assert got == [F.div(a, d, n) for a, d in quo]


def factor_file_digest(path):
    return hashlib.sha256(open(path, "rb").read()).hexdigest()


def test_factor_matches_golden_config_1(exe, tmp_path):
    """beta = 1/2, N = 48, 4096 bits: the whole factor against the Python
    oracle's digest stored in tests/golden/c1.json."""
    import json
    gd = json.load(open(os.path.join(ROOT, "tests", "golden", "c1.json")))
    out = tmp_path / "f.bin"
    subprocess.run([exe, "factor", "2", "48", "4096", str(out)], check=True)
    assert factor_file_digest(out) == gd["factor_sha256"]


def test_factor_matches_python_oracle_any_threads(exe, tmp_path):
    """beta = 1/3, N = 24, 8192 bits, against the Python oracle's factor, with
    1 and 4 OpenMP threads (the dynamic schedule must not change a bit)."""
    n = 256
    mu = OM.moments(Fraction(1, 3), 24, n)
    D, L = OL.ldlt(mu, 24, n)
    h = hashlib.sha256()
    import struct
    for c in range(24):
        for r in range(c, 24):
            s, e, limbs = F.limbs_of(D[c] if r == c else L[r][c], n)
            h.update(struct.pack("<ii", s, e) + struct.pack("<%dI" % n, *limbs))
    want = h.hexdigest()
    for threads in ("1", "4"):
        out = tmp_path / ("f%s.bin" % threads)
        env = dict(os.environ, OMP_NUM_THREADS=threads)
        subprocess.run([exe, "factor", "3", "24", "8192", str(out)], check=True, env=env)
        assert factor_file_digest(out) == want, threads


def test_time_mode_reports_its_sample(exe):
    import json
    r = subprocess.run([exe, "time", "2", "64", "4096", "8"], capture_output=True, text=True, check=True)
    d = json.loads(r.stdout)
    assert d["quotients"] == 63 and d["updates"] == sum(63 - c for c in range(8))
    assert d["threads"] >= 1 and d["update_seconds"] >= 0 and d["scale_seconds"] >= 0
