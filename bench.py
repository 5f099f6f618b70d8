#!/usr/bin/env python
"""lambda_1 solves/hour at beta = 1/2, N = 1024 (arXiv 1810.01478's problem) on GB300.

One step = the whole path for one instance: moments mu_j = 2(2j+1)! ->
LDL^T (Algorithm 1) -> first k columns of L^{-1} (Algorithm 4) -> k x k block
of H^{-1} -> lambda_1..3 with truncation estimates -> d lambda_1/d beta, all in
libhk's CUDA kernels.  Workload: beta = 1/2, N = 1024, k = 32 at 24576 bits
(768 limbs), the largest precision of the paper-scale sweep configuration.

Output: one JSON line (rank 0).  value = solves/hour over all ranks (each rank
solves its own instance: replicas, weak scaling), device time from CUDA events
on the stream the library runs on.  roofline: the trailing-update kernel
(Algorithm 1's inner loops): executed modular multiplications of its NTT
products against the INT32 multiply-add (IMAD) pipe, with the
schoolbook-equivalent limb-product rate beside it.
cpu_baseline: the C++/OpenMP oracle on every host core, timed on a bounded
sample of the same workload (step 0 of Algorithm 1 at full size) and
extrapolated by operation count.
--impl reference: the same oracle as the reference arm (rank 0), same
metric and config, a smaller sample per step.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = dict(beta=(1, 2), N=1024, k=32, bits=24576, n_eig=3)
METRIC = "lambda_1 solves/hour (beta=1/2, N=1024, k=32)"
UNIT = "solves/hour"
# The INT32 multiply pipe of one sm_100-class SM issues 64 IMAD per clock; a
# 32x32->64 limb product takes two (mad.lo + mad.hi, with carry).  The lazy
# Shoup modular multiplication of the transforms, x w - hi(x w') p, issues
# three multiplies but takes four IMAD slots (the 32-bit high-half multiply
# issues at half rate): 16 per SM clock.  hk_alu_peak measures both rates on
# the device (63.8 and 16.0 per SM clock on GB300); the bench line carries
# the measured rates beside these derived peaks.
IMAD_PER_CLK_PER_SM = 64
IMAD_PER_LIMB_MAC = 2
IMAD_SLOTS_PER_MODMUL = 4


def ntt_shape(n):
    """(rows, K) of the library's transform for n limbs: the least L = rows K
    >= 2n with K a power of two and rows in {1, 3} (ties to rows = 1)."""
    def log2c(x):
        l = 0
        while (1 << l) < x:
            l += 1
        return l
    k3 = 1 << log2c((2 * n + 2) // 3)
    k1 = 1 << log2c(2 * n)
    return (3, k3) if 3 * k3 < k1 else (1, k1)


def ntt_modmuls_per_update(n):
    """Modular multiplications of one NTT product (three primes): pointwise
    products, column three-point transforms, row butterflies, and Garner's
    three per position; the forward transforms are shared by a whole step."""
    rows, K = ntt_shape(n)
    L = rows * K
    per_prime = L + (K if rows == 3 else 0) + rows * (K // 2) * (K.bit_length() - 1)
    return 3 * per_prime + 3 * L


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--bits", type=int, default=WORKLOAD["bits"])
    ap.add_argument("--N", type=int, default=WORKLOAD["N"])
    ap.add_argument("--k", type=int, default=WORKLOAD["k"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-side", action="store_true",
                    help="skip the rule-width solve and the batched summary after the timed region")
    ap.add_argument("--profile-case", action="store_true",
                    help="only run moments + LDL^T once at --N/--bits (a small case for ncu captures)")
    ap.add_argument("--rows", default="",
                    help="table2 / regimes: comma-separated N values to run (default: all nine rows of "
                         "Table 2 / 128,256,512,1024)")
    ap.add_argument("--workload", default="single", choices=["single", "batch", "table2", "regimes"],
                    help="batch: 16 uneven instances (beta = 1/m, m in 1..4, N in {128..384}, k = 16, "
                         "32 N bits) through hk_batch_run, beside the same instances one by one")
    return ap.parse_args()


def workload_name(a):
    return (f"beta=1/2 Hankel moment matrix, N={a.N}, k={a.k}, {a.bits}-bit ({a.bits // 32}-limb) LDL^T -> "
            f"L^-1[:, :k] -> block of H^-1 -> lambda_1..3 -> dlambda_1/dbeta")


def ops_count(N, k):
    """Algorithmic operation counts of one solve (fused updates, quotients)."""
    trailing = (N ** 3 - N) // 6
    quot = N * (N - 1) // 2 + N * k
    alg4 = sum((N - 1 - i) * min(k, i) for i in range(N))
    block = N * k * (k + 1) // 2
    return trailing, quot, alg4, block


# ---------------------------------------------------------------------------
# CPU oracle sample (the reported baseline; never tuned)
# ---------------------------------------------------------------------------
def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo), or ''."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu model")):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return ""


def cpp_oracle_time(bits, N, cols):
    """One run of the C++/OpenMP oracle's time mode: step 0 of Algorithm 1
    on H_N (beta = 1/2) at `bits`, updates of its first `cols` columns."""
    from oracle import build_cpp
    exe = build_cpp.build()
    r = subprocess.run([exe, "time", "2", str(N), str(bits), str(cols)], capture_output=True, text=True,
                       check=True)
    return json.loads(r.stdout)


def oracle_sample(bits, N, k, budget_s=15.0):
    """The C++/OpenMP oracle (the paper's A12 loop on every host core) timed
    on a bounded sample of the same workload: step 0 of Algorithm 1 on the
    full H_N at the same precision, its N-1 quotients and the updates of its
    first `cols` columns, `cols` chosen from a short calibration run so the
    sample takes about budget_s.  Extrapolated by operation count to one
    solve: the measured cost of a fused update times the fused updates of
    Algorithm 1, Algorithm 4 and the block, plus the measured cost of a
    quotient times the quotients (the eigenvalues and gradient, a few percent
    of the work, are left out)."""
    cal = cpp_oracle_time(bits, N, 8)
    per_update = cal["update_seconds"] / max(cal["updates"], 1)
    m = N - 1
    cols, acc = 0, 0
    while cols < m and acc * per_update < budget_s:
        acc += m - cols
        cols += 1
    d = cpp_oracle_time(bits, N, cols)
    t_u = d["update_seconds"] / d["updates"]
    t_q = d["scale_seconds"] / d["quotients"]
    tr, qu, a4, bl = ops_count(N, k)
    solve_s = t_u * (tr + a4 + bl) + t_q * qu
    return dict(value=3600.0 / solve_s, unit=UNIT, cores=d["threads"], kind="oracle",
                sample=f"C++/OpenMP oracle (oracle/cpp/hk_oracle.cpp, the paper's flattened dynamic-schedule "
                       f"loop, Sec. 4.3.3) on {d['threads']} host threads: step 0 of Algorithm 1 on the full "
                       f"H_{N} at {bits} bits, its {d['quotients']} quotients in {d['scale_seconds']:.2f} s and "
                       f"{d['updates']} fused updates (columns 1..{cols}) in {d['update_seconds']:.2f} s, "
                       f"extrapolated by operation count to one N={N}, k={k} solve ({solve_s:.4g} s: "
                       f"{tr + a4 + bl:.4g} fused updates, {qu} quotients; eigenvalues and gradient left out)",
                extrapolation=(tr + a4 + bl + qu) / (d["updates"] + d["quotients"]),
                nproc=os.cpu_count(), cpu_model=cpu_model(), seconds=round(d["scale_seconds"] + d["update_seconds"], 2))


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class Clocks:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.tmp = tempfile.NamedTemporaryFile(prefix="clocks", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(index), f"--query-gpu={self.FIELDS}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.tmp, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.tmp.close()
        rows = [r.split(",") for r in open(self.tmp.name).read().strip().splitlines() if r.strip()]
        os.unlink(self.tmp.name)
        sm, smax, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[0]))
                smax = max(smax, float(r[1]))
            except (ValueError, IndexError):
                continue
            for nm, v in zip(names, r[4:8]):
                if v.strip().lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return dict(sm_mhz=statistics.median(sm), sm_max_mhz=smax, reasons=sorted(reasons), samples=len(sm))


# ---------------------------------------------------------------------------
def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def reduce_max(values, device):
    """Element-wise maximum over all ranks (the slowest rank's times); the
    values themselves with one rank."""
    import torch
    import torch.distributed as dist
    t = torch.tensor(values, dtype=torch.float64, device=device)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.tolist()


def solves_per_hour(steps, world_size, ms):
    """Whole-job throughput: every rank solves `steps` instances (replicas)
    within the slowest rank's `ms`."""
    return 3600.0 * steps * world_size / (ms / 1e3)


def run_reference(a):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    vals = []
    sample = None
    budget = max(1.0, min(8.0, 150.0 / max(1, a.warmup + a.steps)))  # the whole run within a few minutes
    for i in range(a.warmup + a.steps):
        s = oracle_sample(a.bits, a.N, a.k, budget_s=budget)
        if i >= a.warmup:
            vals.append(s["value"])
            sample = s
    v = statistics.median(vals)
    cpu = dict(value=v, unit=UNIT, cores=sample["cores"], kind="oracle", sample=sample["sample"],
               nproc=sample["nproc"], cpu_model=sample["cpu_model"], extrapolation=sample["extrapolation"])
    print(json.dumps(dict(impl="reference", metric=METRIC, value=v, unit=UNIT, n_gpus=a.gpus, steps=a.steps,
                          warmup=a.warmup, higher_is_better=True, scaling="weak", vs_baseline=None, dtype="u32",
                          data="synthetic", config=dict(workload=workload_name(a), N=a.N, k=a.k, bits=a.bits),
                          cpu_baseline=cpu, e2e=dict(value=v, unit=UNIT, h2d_bytes_per_step=0, d2h_bytes_per_step=0))),
          flush=True)


def trailing_roofline(prof, n, ntt, sms, sm_max, rates, traffic_per_update, issue):
    """The roofline object of the trailing-update kernel from the library's
    per-launch profile (trailing_ms, trailing_launches, trailing_limb_macs):
    achieved = work per launch / average launch time, against the derived
    integer-pipe peak at the maximum SM clock; rates = the measured
    (IMAD, modmul) per SM clock of hk_alu_peak, or None."""
    launches = max(prof["trailing_launches"], 1)
    avg_launch_ms = prof["trailing_ms"] / launches
    macs_per_launch = prof["trailing_limb_macs"] / launches
    updates_per_launch = macs_per_launch / (n * n)
    traffic = traffic_per_update * updates_per_launch if traffic_per_update is not None else None
    ok = rates is not None and 0 < rates[1] <= rates[0] <= 128
    measured = dict(imad_per_clk_sm=rates[0], modmul_per_clk_sm=rates[1],
                    how="hk_alu_peak: 8 independent chains per thread, one 1024-thread block per SM, clock64 "
                        "span, median over SMs") if ok else None
    achieved_sb = macs_per_launch / (avg_launch_ms / 1e3) / 1e12
    peak_sb = sms * IMAD_PER_CLK_PER_SM / IMAD_PER_LIMB_MAC * sm_max * 1e6 / 1e12  # T limb-MAC/s
    schoolbook = dict(achieved=achieved_sb, peak=peak_sb, unit="Tlimb-MAC/s", frac=achieved_sb / peak_sb,
                      note=f"n^2 = {n * n} limb products per update (the schoolbook-equivalent convention); "
                           f"{sms} SMs x {IMAD_PER_CLK_PER_SM} IMAD/clk / {IMAD_PER_LIMB_MAC} IMAD per limb "
                           f"product x {sm_max:.0f} MHz (derived; measured rate in measured_rates)")
    if not ntt:
        return dict(bound="alu", achieved=achieved_sb, peak=peak_sb, unit="Tlimb-MAC/s", frac=achieved_sb / peak_sb,
                    traffic=traffic, kernel="k_trailing (Algorithm 1 trailing update, schoolbook products)",
                    peak_note=schoolbook["note"], measured_rates=measured)
    mm = ntt_modmuls_per_update(n)
    peak = sms * IMAD_PER_CLK_PER_SM / IMAD_SLOTS_PER_MODMUL * sm_max * 1e6 / 1e12  # T modmul/s
    achieved = mm * updates_per_launch / (avg_launch_ms / 1e3) / 1e12
    return dict(bound="alu", achieved=achieved, peak=peak, unit="Tmodmul/s", frac=achieved / peak,
                traffic=traffic, kernel="k_trailing_ntt (Algorithm 1 trailing update, NTT products)",
                work_per_update=f"{mm} modular multiplications (3 primes, length {ntt_shape(n)[0]} x "
                                f"{ntt_shape(n)[1]})",
                peak_note=f"{sms} SMs x {IMAD_PER_CLK_PER_SM} IMAD/clk / {IMAD_SLOTS_PER_MODMUL} IMAD slots per "
                          f"lazy Shoup modular multiplication x {sm_max:.0f} MHz (derived; measured rate in "
                          f"measured_rates)",
                measured_rates=measured,
                issue_active_frac=issue,
                issue_note="fraction of cycles the kernel issues an instruction (ncu capture of the same "
                           "kernel source, profiles/trailing_traffic.json): the bound it actually meets",
                schoolbook_equiv=schoolbook)


def measured_peaks():
    """MEASURED_PEAKS.json (written beside this file by the GPU pool's driver), or None."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        return json.load(open(path))
    except (OSError, ValueError):
        return None


def tc_digits(n):
    """Balanced 7-bit digits per n-limb number in the tensor-core products."""
    return (32 * n) // 7 + 2


def tc_cut(n):
    """First product position the tensor-core launches form (a multiple of 32
    about 16 limbs below the middle of the 2n-limb product)."""
    return 32 * ((n - 16 - 2) // 7)


def tc_pairs(D, q):
    """Digit products k1 + k2 >= q of a D-digit by D-digit convolution: the
    multiply-adds of a short product that starts at position q."""
    return sum(min(s, 2 * D - 2 - s) + 1 for s in range(q, 2 * D - 1))


def tc_updates(N, min_rows):
    """Fused updates of the tensor-core launches of one LDL^T: every step whose
    trailing triangle has at least min_rows rows, less its look-ahead entry."""
    tot = 0
    for i in range(N - 1):
        rows = N - 1 - i
        if rows >= min_rows:
            tot += rows * (rows + 1) // 2 - 1
    return tot


def alg4_updates(N, k, min_rows):
    """Algorithm 4's fused updates that run inside the tensor-core launches
    when the block is planned (hk_plan_block): min(k, i) columns of the N - 1
    - i rows below step i, for every step with at least min_rows rows."""
    return sum(min(k, i) * (N - 1 - i) for i in range(N - 1) if N - 1 - i >= min_rows)


def tensor_roofline(prof, N, n, min_rows, traffic_per_update, solves, k=0):
    """The roofline object of the tensor-core trailing update: algorithmic
    bf16 flops per second of its launches' device time, against the measured
    cuBLAS bf16 throughput sustained over a long run (the launches run inside
    a multi-second step).  The algorithmic work of a fused update is its short
    product: 2 flops for every digit product k1 + k2 >= q (D balanced 7-bit
    digits per number, q = tc_cut(n)); the re-runs with whole products of the
    rows a short product cannot decide count as executed work only."""
    launches = max(prof["tc_launches"], 1)
    sec = prof["tc_ms"] / 1e3
    D, q = tc_digits(n), tc_cut(n)
    pairs = tc_pairs(D, q)
    # the profile covers `solves` factorisations, each with its planned Algorithm 4 steps
    upd = (tc_updates(N, min_rows) + alg4_updates(N, k, min_rows)) * solves
    alg = 2.0 * pairs * upd
    executed = prof["tc_mmas"] * 2.0 * 128 * 256 * 16
    pk = measured_peaks()
    if pk and pk.get("bf16_tflops_sustained"):
        peak, src = float(pk["bf16_tflops_sustained"]), "of measured (bf16_tflops_sustained, MEASURED_PEAKS.json)"
    else:
        peak, src = 1700.0, "of fallback (1.7 PFLOP/s bf16 sustained)"
    achieved = alg / sec / 1e12
    return dict(bound="tensor", achieved=achieved, peak=peak, unit="TFLOP/s", frac=achieved / peak,
                traffic=traffic_per_update * upd / launches if traffic_per_update is not None else None,
                kernel="k_tc_fused (Algorithm 1 trailing update, bf16 tcgen05 digit-convolution GEMMs)",
                peak_note=src,
                work_per_update=f"{2 * pairs} flops: 2 per digit product at positions >= {q} "
                                f"(D = {D} balanced 7-bit digits per number; the whole product is {2 * D * D})",
                rerun_items=int(prof.get("tc_redo_items", 0)),
                updates=upd, launches=int(prof["tc_launches"]),
                executed_tflops=executed / sec / 1e12, executed_frac=executed / sec / 1e12 / peak,
                executed_note="tcgen05.mma instructions issued (128 x 256 x 16 each, including the padding of "
                              "partial 128-row tiles and of the digit bands' edges) per second",
                schoolbook_equiv_tlimb_macs=upd * n * n / sec / 1e12)


def num_fraction(s, e, m):
    """The exact value of one number of the library's layout."""
    from fractions import Fraction
    v = 0
    for i, w in enumerate(m):
        v |= int(w) << (32 * i)
    return Fraction(-v if int(s) else v) * Fraction(2) ** (32 * int(e))


def rel_diff_log10(x, y):
    """log10 |x - y| / |y| of two exact Fractions (-inf when equal)."""
    import math
    d = abs(x - y)
    if d == 0:
        return float("-inf")
    q = d / abs(y)
    return (math.log10(q.numerator) if q.numerator else 0.0) - math.log10(q.denominator)


def at_rule_bits(hk, stream, device, a, loss, need, lam_ref, sms, sm_max, rates, steps=4, warmup=2):
    """The same solve at the width the precision check selects (the least
    compiled width >= min_bits of hk_precision_loss, which the factor's own
    loss estimate sets), timed with CUDA events; its lambda_1..3 against the
    configured-width solve, which has more than twice the bits and so serves
    as the precision-doubling check; and its trailing-update roofline."""
    import torch
    widths = sorted(hk.hk_supported_bits())
    bits = next(w for w in widths if w >= need)
    n = bits // 32
    h = hk.Hankel(device, stream.cuda_stream)
    try:
        def solve():
            h.moments(1, 2, a.N, bits)
            h.ldlt(k=a.k)
            h.inv_block(a.k)
            lam = h.lambda1(3)
            h.lambda1_grad()
            return lam
        for _ in range(warmup):
            solve()
        torch.cuda.synchronize()
        hk.hk_set_profiling(h.ctx, True)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for _ in range(steps):
            lam = solve()
        ev1.record(stream)
        torch.cuda.synchronize()
        ms = ev0.elapsed_time(ev1)
        prof = hk.hk_get_profile(h.ctx)
    finally:
        h.close()
    diffs = [rel_diff_log10(num_fraction(lam[0][j], lam[1][j], lam[2][j]),
                            num_fraction(lam_ref[0][j], lam_ref[1][j], lam_ref[2][j])) for j in range(3)]
    ntt = (bits // 1024) >= hk.HK_NTT_AUTO_MIN_M
    roof = trailing_roofline(prof, n, ntt, sms, sm_max, rates, None, None)
    return dict(bits=bits, loss_bits=int(loss), min_bits=int(need), value=solves_per_hour(steps, 1, ms),
                unit=UNIT, ms_per_solve=ms / steps,
                lambda_log10_rel_diff_vs_configured_bits=diffs, agree_to_1e40=all(x < -40 for x in diffs),
                roofline=roof, phases_ms=dict(ldlt=prof["ldlt_ms"] / steps, trailing=prof["trailing_ms"] / steps),
                note=f"width = least compiled width >= 2 loss + 229 bits (hk_precision_loss); lambda_1..3 compared "
                     f"with the {a.bits}-bit solve (precision doubling)")


def batch_summary(hk, torch, steps=2):
    """The batched configuration's 16 instances through hk_batch_run (the
    instances of each width up to 8192 bits in one persistent launch,
    hk_ldlt_batch; the 12288-bit ones on their own streams) against the same
    instances one after another on one stream; and a sweep of 32 instances
    at one width whose factorisations run in one persistent launch, beside
    concurrent streams and one stream."""
    probs = [dict(beta=(1, m), N=N, k=16, bits=32 * N, n_eig=1) for m in (1, 2, 3, 4) for N in (128, 192, 256, 384)]
    t = batch_times(hk, torch, probs, steps, 1)
    return dict(instances=len(probs),
                form="hk_batch_run: one persistent launch per width up to 8192 bits (hk_ldlt_batch), "
                     "the wider instances on concurrent streams",
                workload="beta=1/m, m in {1,2,3,4} x N in {128,192,256,384}, k=16, 32N bits, moments -> LDL^T -> "
                         "block -> lambda_1",
                seconds_batched=t["batched"], seconds_sequential=t["sequential"],
                speedup=t["sequential"] / t["batched"], instances_per_hour=3600.0 * len(probs) / t["batched"],
                sweep=ldlt_sweep_times(hk, torch))


def ldlt_sweep_times(hk, torch, bits=4096, ns=(96, 128, 160, 192, 224, 256, 288, 320), reps=3):
    """Seconds for the factorisations of 32 instances (beta = 1/m, m = 1..4,
    x ns) at one width: one persistent launch (hk_ldlt_batch), one stream
    and host thread per instance (hk_ldlt on each), and one stream; the best
    of `reps` runs each, from the moments to the last pivot on the host."""
    import threading
    sp = [((1, m), N) for m in (1, 2, 3, 4) for N in ns]

    def persistent():
        hs = [hk.Hankel(0) for _ in sp]
        t0 = time.perf_counter()
        for (b, N), h in zip(sp, hs):
            h.moments(b[0], b[1], N, bits)
        hk.hk_ldlt_batch([h.ctx for h in hs])
        for (b, N), h in zip(sp, hs):
            h.export(hk.HK_D, N - 1, 1)
        dt = time.perf_counter() - t0
        for h in hs:
            h.close()
        return dt

    def streams():
        ss = [torch.cuda.Stream() for _ in sp]
        hs = [hk.Hankel(0, s.cuda_stream) for s in ss]

        def one(q):
            (b, N), h = sp[q], hs[q]
            h.moments(b[0], b[1], N, bits)
            h.ldlt()
            h.export(hk.HK_D, N - 1, 1)
        t0 = time.perf_counter()
        th = [threading.Thread(target=one, args=(q,)) for q in range(len(sp))]
        for x in th:
            x.start()
        for x in th:
            x.join()
        dt = time.perf_counter() - t0
        for h in hs:
            h.close()
        return dt

    def one_stream():
        t0 = time.perf_counter()
        for b, N in sp:
            with hk.Hankel(0) as h:
                h.moments(b[0], b[1], N, bits)
                h.ldlt()
                h.export(hk.HK_D, N - 1, 1)
        return time.perf_counter() - t0

    out = dict(workload=f"LDL^T of 32 instances: beta=1/m, m in 1..4 x N in {list(ns)}, {bits} bits")
    for name, fn in (("persistent_launch", persistent), ("concurrent_streams", streams), ("one_stream", one_stream)):
        fn()
        out["seconds_" + name] = min(fn() for _ in range(reps))
    out["speedup_vs_streams"] = out["seconds_concurrent_streams"] / out["seconds_persistent_launch"]
    out["speedup_vs_one_stream"] = out["seconds_one_stream"] / out["seconds_persistent_launch"]
    return out


def batch_times(hk, torch, probs, steps, warmup):
    """Wall seconds per pass of hk_batch_run over probs and of the same
    instances solved one after another on one stream."""
    def batched():
        st, res = hk.hk_batch_run(0, probs, max_concurrent=len(probs))
        assert st == hk.HK_OK, [r["message"] for r in res if r["status"]]
        return res

    def sequential():
        out = []
        for p in probs:
            with hk.Hankel(0) as h:
                h.moments(*p["beta"], p["N"], p["bits"])
                h.ldlt(k=p["k"])
                h.inv_block(p["k"])
                out.append(h.lambda1(1))
        return out

    for _ in range(max(1, warmup)):
        batched()
    torch.cuda.synchronize()
    times = {}
    for name, fn in (("batched", batched), ("sequential", sequential)):
        t0 = time.perf_counter()
        for _ in range(steps):
            fn()
        torch.cuda.synchronize()
        times[name] = (time.perf_counter() - t0) / steps
    return times


def run_ours(a):
    import torch
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    import __graft_entry__ as g
    g.build()
    import paper_1810_01478_gb300 as hk
    stream = torch.cuda.current_stream()
    h = hk.Hankel(local, stream.cuda_stream)
    beta = WORKLOAD["beta"]
    n = a.bits // 32
    ne = WORKLOAD["n_eig"]

    def step():
        h.moments(beta[0], beta[1], a.N, a.bits)
        h.ldlt(k=a.k)
        h.inv_block(a.k)
        lam = h.lambda1(ne)
        gr = h.lambda1_grad()
        return lam, gr

    for _ in range(a.warmup):
        lam, gr = step()
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks = Clocks(local)
    hk.hk_set_profiling(h.ctx, True)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0 = time.perf_counter()
    ev0.record(stream)
    for _ in range(a.steps):
        lam, gr = step()
    ev1.record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    if ws > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    prof = hk.hk_get_profile(h.ctx)
    dev_ms = ev0.elapsed_time(ev1)
    dev_ms, wall_ms = reduce_max([dev_ms, wall * 1e3], "cuda")
    value = solves_per_hour(a.steps, ws, dev_ms)
    e2e = solves_per_hour(a.steps, ws, wall_ms)
    props = torch.cuda.get_device_properties(local)
    sms = props.multi_processor_count
    sm_max = (clk or {}).get("sm_max_mhz") or 2070.0
    # the integer pipe's measured rates (operations per SM clock), after the timed region
    try:
        rates = (hk.hk_alu_peak(local, 0), hk.hk_alu_peak(local, 1))
    except (RuntimeError, AttributeError):
        rates = None
    ntt = (a.bits // 1024) >= hk.HK_NTT_AUTO_MIN_M
    traffic_per_update = issue = None
    tp = os.path.join(ROOT, "profiles", "trailing_traffic.json")
    if os.path.exists(tp):
        try:
            t = json.load(open(tp))
            if t.get("bits") == a.bits and t.get("kernel_source_sha") == kernel_sha():
                traffic_per_update = t["bytes_per_update"]
                issue = t.get("issue_active_frac")
        except (ValueError, KeyError):
            traffic_per_update = issue = None
    ntt_roof = trailing_roofline(prof, n, ntt, sms, sm_max, rates, traffic_per_update, issue)
    if prof.get("tc_launches", 0) > 0:
        tc_traffic = None
        tp2 = os.path.join(ROOT, "profiles", "tc_traffic.json")
        if os.path.exists(tp2):
            try:
                t = json.load(open(tp2))
                if t.get("bits") == a.bits and t.get("kernel_source_sha") == kernel_sha(("tc.cuh", "mp_warp.cuh")):
                    tc_traffic = t["bytes_per_update"]
            except (ValueError, KeyError):
                tc_traffic = None
        roofline = tensor_roofline(prof, a.N, n, hk.HK_TC_MIN_ROWS, tc_traffic, a.steps, k=a.k)
        roofline["ntt_steps"] = dict(note="the trailing launches of the last steps (fewer than "
                                          f"{hk.HK_TC_MIN_ROWS} rows) and the look-ahead entries keep NTT "
                                          "products; these figures cover every trailing launch",
                                     ms=prof["trailing_ms"] - prof["tc_ms"], measured_rates=ntt_roof.get("measured_rates"))
    else:
        roofline = ntt_roof
    d2h = ne * (8 + 4 * n) + min(ne, a.k - 1) * (8 + 4 * n) + (8 + 4 * n)
    lam_f64 = lam[3].tolist()
    out = dict(metric=METRIC, value=value, unit=UNIT, n_gpus=ws, steps=a.steps, warmup=a.warmup,
               ms_per_step=dev_ms / a.steps, higher_is_better=True, scaling="weak", vs_baseline=None,
               dtype="u32", data="synthetic",
               config=dict(workload=workload_name(a), N=a.N, k=a.k, bits=a.bits, beta="1/2",
                           parallelism=f"replicas x{ws}" if ws > 1 else "single GPU",
                           l2="inputs larger than L2: the packed factor alone is "
                              f"{a.N * (a.N + 1) // 2 * (4 * n + 8) / 1e9:.2f} GB"),
               e2e=dict(value=e2e, unit=UNIT, h2d_bytes_per_step=0, d2h_bytes_per_step=d2h),
               gpu_launches=int(prof["launches"]),
               roofline=roofline,
               phases_ms=dict(moments=prof["moments_ms"] / a.steps, ldlt=prof["ldlt_ms"] / a.steps,
                              trailing=prof["trailing_ms"] / a.steps, scale=prof["scale_ms"] / a.steps,
                              invblock=prof["invblock_ms"] / a.steps,
                              eig=prof["eig_ms"] / a.steps, grad=prof["grad_ms"] / a.steps,
                              trailing_tensor=prof["tc_ms"] / a.steps),
               result=dict(lambda_f64=lam_f64, trunc_err_f64=lam[4].tolist(), dlambda_dbeta_f64=gr[3].tolist()[0]),
               clocks=clk)
    if rank == 0 and ws == 1 and not a.no_side:
        loss, need = h.precision_loss()
        out["at_rule_bits"] = at_rule_bits(hk, stream, local, a, loss, need, lam, sms, sm_max, rates)
        out["batch"] = batch_summary(hk, torch)
    if rank == 0 and ws == 1 and not a.no_cpu_baseline:
        out["cpu_baseline"] = oracle_sample(a.bits, a.N, a.k)
    h.close()
    if rank == 0:
        print(json.dumps(out), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


def kernel_sha(files=("mp_warp.cuh", "ntt.cuh", "k_ldlt.cuh")):
    import hashlib
    hsh = hashlib.sha256()
    d = os.path.join(ROOT, "paper_1810_01478_gb300", "csrc")
    for f in files:
        hsh.update(open(os.path.join(d, f), "rb").read())
    return hsh.hexdigest()[:16]


def profile_case(a):
    import __graft_entry__ as g
    g.build()
    import paper_1810_01478_gb300 as hk
    with hk.Hankel(0) as h:
        h.moments(1, 2, a.N, a.bits)
        h.ldlt()
        h.export(hk.HK_D, a.N - 1, 1)
    print("profile case done", a.N, a.bits)


def run_batch(a):
    """The batched form alone: 16 instances of uneven size through
    hk_batch_run (one persistent launch per width up to 8192 bits, the rest
    on concurrent streams), timed beside the same instances solved one after
    another on one stream, plus the 32-instance factorisation sweep.  beta = 1/m (moments exact on the device) with m in {1, 2, 3, 4},
    N in {128, 192, 256, 384}, k = 16, 32 N bits: the shapes of the
    paper-scale batched configuration."""
    import torch
    import __graft_entry__ as g
    g.build()
    import paper_1810_01478_gb300 as hk
    out = batch_summary(hk, torch, steps=a.steps)
    print(json.dumps(dict(metric="instances/hour (16 uneven lambda_1 solves, hk_batch_run)",
                          value=out["instances_per_hour"], unit="instances/hour", n_gpus=1, steps=a.steps,
                          warmup=a.warmup, higher_is_better=True, data="synthetic", **out)), flush=True)


def run_table2(a):
    """The paper's Table 2 (Sec. 5.1) on one GPU: beta = 1/2, N = 500 ... 4500,
    k = 8, at twice the table's fixed-point bits K (the paper's fixed point
    keeps 2K bits during the LDL^T, Sec. 4.1), rounded up to a compiled width.
    Prints one JSON line per row (the three eigenvalues and truncation
    estimates against the printed ones, and the wall time of the solve) and
    then the Sec. 6.1 fit y = a + b x, x = log(4 pi N e),
    y = log(8 pi sqrt(log N) / lambda_1), N^2-weighted, on these lambda_1."""
    import math
    import torch
    import __graft_entry__ as g
    g.build()
    import paper_1810_01478_gb300 as hk
    table = json.load(open(os.path.join(ROOT, "tests", "golden", "table2_beta_half.json")))
    widths = sorted(hk.hk_supported_bits())
    want = [int(x) for x in a.rows.split(",") if x] if a.rows else None
    pts = []
    for row in table["rows"]:
        N = row["N"]
        if want and N not in want:
            continue
        bits = next(w for w in widths if w >= 2 * row["bits"])
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        with hk.Hankel(0) as h:
            h.moments(1, 2, N, bits)
            h.ldlt()
            h.inv_block(8)
            _, _, _, lam, terr = h.lambda1(3)
        dt = time.perf_counter() - t0
        printed = [float(v) for v in row["lambda"]]
        pts.append((N, float(lam[0])))
        print(json.dumps(dict(workload="table2", N=N, bits=bits, k=8, seconds=dt,
                              lambda_f64=[float(v) for v in lam], lambda_printed=row["lambda"],
                              rel_diff=[abs(float(lam[j]) - printed[j]) / printed[j] for j in range(3)],
                              trunc_err_f64=[float(v) for v in terr], trunc_err_printed=row["trunc_err"])),
              flush=True)
    if len(pts) >= 2:
        a0, b = sec61_fit(pts)
        print(json.dumps(dict(workload="table2_fit", rows=[N for N, _ in pts], intercept=a0, slope=b,
                              paper=table["fit"])), flush=True)


def sec61_fit(pts):
    """Sec. 6.1's fit on (N, lambda_1) points: the N^2-weighted least-squares
    line y = a + b x with x = log(4 pi N e) and y = log(8 pi sqrt(log N) /
    lambda_1); returns (a, b).  The paper reads b against 2/pi."""
    import math
    xs = [math.log(4 * math.pi * N * math.e) for N, _ in pts]
    ys = [math.log(8 * math.pi * math.sqrt(math.log(N)) / l1) for N, l1 in pts]
    ws = [N * N for N, _ in pts]
    sw = sum(ws)
    mx = sum(w * x for w, x in zip(ws, xs)) / sw
    my = sum(w * y for w, y in zip(ws, ys)) / sw
    b = sum(w * (x - mx) * (y - my) for w, x, y in zip(ws, xs, ys)) / sum(w * (x - mx) ** 2 for w, x in zip(ws, xs))
    return my - b * mx, b


def local_slopes(pts, xf):
    """Slopes of log lambda between successive (N, lambda) points against xf(N)."""
    import math
    return [(math.log(l1) - math.log(l0)) / (xf(n1) - xf(n0)) for (n0, l0), (n1, l1) in zip(pts, pts[1:])]


def gamma_constants_limbs(a, b):
    """The constants Gamma(r/a), r = 1..a-1, for hk_moments_gamma, from
    tests/golden/c3_gamma_constants.json (12416 correct bits, written there
    by the repository's golden-value script): (limb exponents, limbs)."""
    import numpy as np
    from fractions import Fraction
    d = json.load(open(os.path.join(ROOT, "tests", "golden", "c3_gamma_constants.json")))
    raw = d["constants"][f"{a}/{b}"]
    vals = [Fraction(int(p, 16), int(q, 16)) for p, q in raw[1:]]
    rows, exps = [], []
    for v in vals:
        s = v.denominator.bit_length() - 1
        e = -((s + 31) // 32)
        rows.append(v.numerator << (32 * -e - s))
        exps.append(e)
    nc = max((m.bit_length() + 31) // 32 for m in rows)
    limbs = np.zeros((len(rows), nc), np.uint32)
    for i, m in enumerate(rows):
        sh = nc - (m.bit_length() + 31) // 32
        m <<= 32 * sh
        exps[i] -= sh
        for k in range(nc):
            limbs[i, k] = (m >> (32 * k)) & 0xFFFFFFFF
    return np.array(exps, np.int32), limbs


def limit_fit(pts):
    """beta < 1/2: lambda_1(N) -> lambda_inf > 0.  On three points at doubling
    N, lambda(N) = lambda_inf + C N^-p is determined exactly (Aitken's delta^2
    on the geometric sequence of differences): returns (lambda_inf, p)."""
    import math
    (n0, l0), (n1, l1), (n2, l2) = pts[-3:]
    assert n1 == 2 * n0 and n2 == 2 * n1
    d0, d1 = l1 - l0, l2 - l1
    r = d1 / d0
    return l2 + d1 * r / (1 - r), -math.log2(r)


def sqrt_decay_fit(pts):
    """beta > 1/2: Szego's form for the Laguerre weight (beta = 1, Sec. 1),
    lambda_1 ~ A N^(1/4) B^sqrt(N): least squares of log lambda_1 - log(N)/4
    on sqrt(N); returns (log A, log B).  Also the effective exponent gamma
    of -log lambda_1 ~ c N^gamma from the last two points."""
    import math
    xs = [math.sqrt(N) for N, _ in pts]
    ys = [math.log(l) - 0.25 * math.log(N) for N, l in pts]
    mx, my = sum(xs) / len(xs), sum(ys) / len(ys)
    b = sum((x - mx) * (y - my) for x, y in zip(xs, ys)) / sum((x - mx) ** 2 for x in xs)
    (n0, l0), (n1, l1) = pts[-2:]
    gamma = (math.log(-math.log(l1)) - math.log(-math.log(l0))) / (math.log(n1) - math.log(n0))
    return my - b * mx, b, gamma


def run_regimes(a):
    """The three regimes of the weight exp(-x^beta) (abstract, Sec. 1 and 6)
    at beta = 1/3, 9/20 (< 1/2: indeterminate moment problem, lambda_1
    bounded below), 1/2 (algebraic decay), 11/20 and 1 (> 1/2: exponential
    decay), N = 128 ... 1024, k = 64 (at beta = 1 and N = 1024 a k = 32 block
    still has a 30 % truncation estimate).  beta = 1/m uses the device's
    exact moments, beta = 9/20, 11/20 the constants Gamma(r/20) (12416 bits).
    Each solve runs at the least compiled width the precision check accepts
    (hk_precision_loss, tried from 2 N + 229 bits up).  One JSON line per
    solve, then one per beta with its fit: the limit lambda_inf (beta < 1/2),
    Sec. 6.1's exponent (beta = 1/2), Szego's sqrt(N) decay rate (beta > 1/2)."""
    import math
    import torch
    import __graft_entry__ as g
    g.build()
    import paper_1810_01478_gb300 as hk
    widths = sorted(hk.hk_supported_bits())
    Ns = [int(x) for x in a.rows.split(",") if x] if a.rows else [128, 256, 512, 1024]
    for bn, bd in ((1, 3), (9, 20), (1, 2), (11, 20), (1, 1)):
        consts = gamma_constants_limbs(bn, bd) if bn > 1 else None
        pts = []
        for N in Ns:
            k = min(64, N)
            bits = next((w for w in widths if w >= 2 * N + 229), widths[-1])
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            while True:
                h = hk.Hankel(0)
                try:
                    if consts is None:
                        h.moments(bn, bd, N, bits)
                    else:
                        h.moments_gamma(bn, bd, N, bits, *consts)
                    h.ldlt()
                    loss, need = h.precision_loss()
                    if need > bits and bits < widths[-1]:
                        bits = next((w for w in widths if w >= need), widths[-1])
                        continue
                    h.inv_block(k)
                    _, _, _, lam, terr = h.lambda1(3)
                    break
                finally:
                    h.close()
            dt = time.perf_counter() - t0
            pts.append((N, float(lam[0])))
            print(json.dumps(dict(workload="regimes", beta=f"{bn}/{bd}", N=N, k=k, bits=bits, loss_bits=loss,
                                  seconds=dt, lambda_f64=[float(v) for v in lam],
                                  trunc_err_f64=[float(v) for v in terr])), flush=True)
        fit = dict(workload="regimes_fit", beta=f"{bn}/{bd}", N=Ns,
                   dlog_lambda_dlog_N=local_slopes(pts, math.log),
                   dlog_lambda_dsqrt_N=local_slopes(pts, math.sqrt))
        if 2 * bn < bd and len(pts) >= 3:
            li, pw = limit_fit(pts)
            fit.update(lambda_inf=li, approach_exponent=pw,
                       model="lambda_1 = lambda_inf + C N^-p through the last three points (doubling N)")
        elif 2 * bn == bd and len(pts) >= 2:
            a0, b0 = sec61_fit(pts)
            fit.update(sec61_intercept=a0, sec61_slope=b0, two_over_pi=2 / math.pi,
                       model="Sec. 6.1: N^2-weighted y = a + b x, x = log(4 pi N e), y = log(8 pi sqrt(log N)/lambda_1)")
        elif len(pts) >= 2:
            la, lb, gam = sqrt_decay_fit(pts)
            fit.update(log_A=la, log_B=lb, B=math.exp(lb), effective_exponent=gam,
                       model="Szego (beta = 1): lambda_1 ~ A N^(1/4) B^sqrt(N); -log lambda_1 ~ c N^gamma")
        print(json.dumps(fit), flush=True)


if __name__ == "__main__":
    args = parse()
    if args.workload == "table2":
        run_table2(args)
    elif args.workload == "regimes":
        run_regimes(args)
    elif args.workload == "batch":
        run_batch(args)
    elif args.profile_case:
        profile_case(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)
