"""The ctypes mirror of hk_instance (include/hk.h) has the C layout: field
offsets and the struct size compared with a C program compiled against the
header (gcc, no GPU)."""
import ctypes
import os
import shutil
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
FIELDS = ["beta_num", "beta_den", "N", "k", "bits", "n_eig", "mu_sign", "mu_exp", "mu_limbs", "gamma_exp",
          "gamma_limbs", "lambda_sign", "lambda_exp", "lambda_limbs", "lambda_f64", "trunc_err_f64", "seconds",
          "status", "gamma_nc", "message"]


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
def test_instance_layout_matches_header():
    from paper_1810_01478_gb300 import Instance
    src = "#include <stdio.h>\n#include <stddef.h>\n#include \"hk.h\"\nint main(void) {\n"
    for f in FIELDS:
        src += f'  printf("%s %zu\\n", "{f}", offsetof(hk_instance, {f}));\n'
    src += '  printf("sizeof %zu\\n", sizeof(hk_instance));\n  return 0;\n}\n'
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "layout.c")
        exe = os.path.join(d, "layout")
        open(c, "w").write(src)
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split("\n")
    got = dict(line.split() for line in out if line)
    for f in FIELDS:
        assert int(got[f]) == getattr(Instance, f).offset, f
    assert int(got["sizeof"]) == ctypes.sizeof(Instance)
