"""Host logic of bench.py, on the CPU.  The multi-GPU path is replicas only:
every rank solves its own instance, the job time is the slowest rank's, and
the value counts the solves of all ranks.  Checked here with two gloo ranks
(no GPU): the cross-rank maximum, the throughput formula, and that only rank
0 of the reference arm prints.  Also the arithmetic of the roofline object
and of the regimes workload's slopes."""
import json
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, port, out):
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=2)
    try:
        dev_ms, wall_ms = bench.reduce_max([100.0 + 50.0 * rank, 300.0 - 10.0 * rank], "cpu")
        dist.barrier()
        out[rank] = (dev_ms, wall_ms, bench.solves_per_hour(2, dist.get_world_size(), dev_ms))
    finally:
        dist.destroy_process_group()


def test_two_rank_max_and_throughput():
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(port, out), nprocs=2, join=True)
        res = dict(out)
    for rank in (0, 1):
        dev_ms, wall_ms, v = res[rank]
        assert dev_ms == 150.0 and wall_ms == 300.0
        assert v == pytest.approx(3600.0 * 2 * 2 / 0.150)


def test_single_rank_reduce_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_max([1.5, 2.5], "cpu") == [1.5, 2.5]
    assert bench.solves_per_hour(2, 1, 1000.0) == pytest.approx(7200.0)


def test_reference_arm_prints_on_rank_zero_only():
    env = dict(os.environ, WORLD_SIZE="2", RANK="1", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], capture_output=True, text=True, env=env, cwd=ROOT, timeout=600)
    assert r.returncode == 0 and r.stdout.strip() == ""


def test_local_slopes_of_the_regimes_workload():
    """bench.local_slopes: a power law N^-a has log-log slope -a, and
    exp(-c sqrt N) has slope -c against sqrt N, between every pair."""
    import math
    import bench
    pts = [(n, n ** -0.6366) for n in (128, 256, 512, 1024)]
    assert all(abs(s + 0.6366) < 1e-12 for s in bench.local_slopes(pts, math.log))
    pts = [(n, math.exp(-3.5 * math.sqrt(n))) for n in (100, 400, 900)]
    assert all(abs(s + 3.5) < 1e-9 for s in bench.local_slopes(pts, math.sqrt))


def test_trailing_roofline_arithmetic():
    """bench.trailing_roofline: achieved = work per launch / average launch
    time against 152 SMs x 64 IMAD/clk / 4 slots per modular multiplication x
    the clock; measured rates are kept only when physical."""
    import bench
    n, per_launch, launches, ms = 768, 1000, 2, 10.0
    prof = dict(trailing_launches=launches, trailing_ms=ms, trailing_limb_macs=launches * per_launch * n * n)
    r = bench.trailing_roofline(prof, n, True, 152, 2070.0, (63.8, 16.0), 6807.3, 0.52)
    mm = bench.ntt_modmuls_per_update(n)
    assert mm == 31488
    want = mm * per_launch / (ms / launches / 1e3) / 1e12
    assert abs(r["achieved"] - want) < 1e-12 * want
    assert abs(r["peak"] - 152 * 16 * 2070e6 / 1e12) < 1e-9
    assert abs(r["frac"] - want / r["peak"]) < 1e-12
    assert abs(r["traffic"] - 6807.3 * per_launch) < 1e-6
    assert r["measured_rates"]["modmul_per_clk_sm"] == 16.0 and r["issue_active_frac"] == 0.52
    sb = r["schoolbook_equiv"]
    assert abs(sb["peak"] - 152 * 32 * 2070e6 / 1e12) < 1e-9
    assert abs(sb["achieved"] - per_launch * n * n / (ms / launches / 1e3) / 1e12) < 1e-9
    # a rate above the issue limit is not a rate; no traffic capture gives null
    r = bench.trailing_roofline(prof, n, True, 152, 2070.0, (252.8, 16.0), None, None)
    assert r["measured_rates"] is None and r["traffic"] is None
    r = bench.trailing_roofline(prof, 128, False, 152, 2070.0, None, None, None)
    assert r["unit"] == "Tlimb-MAC/s" and r["measured_rates"] is None


def test_tensor_roofline_arithmetic():
    """bench.tensor_roofline: algorithmic flops of the short products (2 per
    digit product at positions >= the cut) per fused update of the
    tensor-core launches (every step with at least min_rows trailing rows,
    less its look-ahead entry), times the factorisations profiled, over their
    device time, against the sustained bf16 peak; the executed rate counts
    the MMA instructions (128 x 256 x 16 each)."""
    import bench
    N, n, min_rows = 300, 768, 256
    upd = sum((N - 1 - i) * (N - i) // 2 - 1 for i in range(N - 1) if N - 1 - i >= min_rows)
    assert bench.tc_updates(N, min_rows) == upd
    D = bench.tc_digits(n)
    assert D == 3512 and bench.tc_cut(n) == 3424
    # the digit products of a D x D convolution at positions >= q, counted directly
    for d, q in ((5, 0), (5, 3), (7, 6), (9, 16)):
        assert bench.tc_pairs(d, q) == sum(1 for a in range(d) for b in range(d) if a + b >= q)
    pairs = bench.tc_pairs(D, 3424)
    assert pairs == D * (D + 1) // 2 + sum(s + 1 for s in range(3424, D - 1))
    prof = dict(tc_launches=10, tc_ms=2000.0, tc_mmas=1.0e6)
    r = bench.tensor_roofline(prof, N, n, min_rows, 100.0, 2)
    want = 2.0 * pairs * upd * 2 / 2.0 / 1e12
    assert abs(r["achieved"] - want) < 1e-9 * want
    assert abs(r["frac"] - want / r["peak"]) < 1e-12
    assert abs(r["executed_tflops"] - 1.0e6 * 2 * 128 * 256 * 16 / 2.0 / 1e12) < 1e-9
    assert r["bound"] == "tensor" and abs(r["traffic"] - 100.0 * upd * 2 / 10) < 1e-6
    # a planned block adds Algorithm 4's updates of the same steps
    a4 = sum(min(32, i) * (N - 1 - i) for i in range(N - 1) if N - 1 - i >= min_rows)
    assert bench.alg4_updates(N, 32, min_rows) == a4 > 0
    r4 = bench.tensor_roofline(prof, N, n, min_rows, None, 2, k=32)
    assert abs(r4["achieved"] - 2.0 * pairs * (upd + a4) * 2 / 2.0 / 1e12) < 1e-9 * r4["achieved"]


def test_exact_lambda_comparison_helpers():
    """bench.num_fraction reads the library's number layout exactly, and
    bench.rel_diff_log10 gives log10 of the relative difference."""
    import bench
    from fractions import Fraction
    assert bench.num_fraction(1, -1, [0, 3]) == Fraction(-3)
    assert bench.num_fraction(0, 2, [5]) == Fraction(5 * 2 ** 64)
    x, y = Fraction(1) + Fraction(1, 10 ** 45), Fraction(1)
    assert -45.01 < bench.rel_diff_log10(x, y) < -44.99
    assert bench.rel_diff_log10(y, y) == float("-inf")


def test_sec61_fit_reproduces_the_printed_coefficients():
    """bench.sec61_fit on Table 2's printed lambda_1 column (Sec. 5.1) gives
    the coefficients Sec. 6.1 prints, 0.04630 and 0.63646 (the slope within
    the printed 95 % interval [0.63510, 0.63781], which holds 2/pi)."""
    import json
    import math
    import bench
    t = json.load(open(os.path.join(ROOT, "tests", "golden", "table2_beta_half.json")))
    pts = [(r["N"], float(r["lambda"][0])) for r in t["rows"]]
    a, b = bench.sec61_fit(pts)
    assert round(a, 5) == float(t["fit"]["intercept"]) and round(b, 5) == float(t["fit"]["slope"])
    assert 0.63510 <= b <= 0.63781 and 0.63510 <= 2 / math.pi <= 0.63781


def test_regime_fits_recover_their_models():
    """bench.limit_fit recovers lambda_inf and p of lambda_inf + C N^-p from
    three doubling points; bench.sqrt_decay_fit recovers log A and log B of
    A N^(1/4) B^sqrt(N)."""
    import math
    import bench
    pts = [(n, 3.3 + 2.0 * n ** -0.55) for n in (256, 512, 1024)]
    li, p = bench.limit_fit(pts)
    assert abs(li - 3.3) < 1e-9 and abs(p - 0.55) < 1e-9
    pts = [(n, math.exp(-1.5) * n ** 0.25 * math.exp(-4.0 * math.sqrt(n))) for n in (128, 256, 512, 1024)]
    la, lb, gam = bench.sqrt_decay_fit(pts)
    assert abs(la + 1.5) < 1e-9 and abs(lb + 4.0) < 1e-9 and 0.4 < gam < 0.6
