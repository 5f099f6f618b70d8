"""Host check of the batched launch's scheduling arithmetic: compiles
tests/batch_sched_check.cpp against csrc/batch_sched.h and common.cuh with
the host compiler and runs it (phase item counts against Algorithm 1 and 4's
loops, chunk ranges, item decoding, the trailing triangle's enumeration)."""
import os
import shutil
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_batch_schedule_arithmetic():
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        pytest.skip("no host C++ compiler")
    cuda_inc = None
    for d in (os.environ.get("CUDA_HOME", ""), "/usr/local/cuda"):
        if d and os.path.exists(os.path.join(d, "include", "cuda_runtime.h")):
            cuda_inc = os.path.join(d, "include")
            break
    if not cuda_inc:
        pytest.skip("CUDA headers not found")
    with tempfile.TemporaryDirectory() as tmp:
        exe = os.path.join(tmp, "batch_sched_check")
        r = subprocess.run([cxx, "-std=c++17", "-O2", "-I", os.path.join(ROOT, "paper_1810_01478_gb300", "csrc"),
                            "-I", cuda_inc, os.path.join(ROOT, "tests", "batch_sched_check.cpp"), "-o", exe],
                           capture_output=True, text=True)
        assert r.returncode == 0, r.stderr
        r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
        assert r.returncode == 0 and r.stdout.strip() == "ok", r.stdout + r.stderr
