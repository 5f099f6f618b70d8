"""Build libhk.so in-tree for sm_103a with nvcc (no cmake, no torch extension).

One translation unit per limb width (csrc/inst.cu with -DHK_M=<M>, the list in
csrc/widths.h) plus the C ABI (csrc/hk_abi.cu), compiled in parallel and
linked into paper_1810_01478_gb300/_build/libhk.so.
"""
import hashlib
import os
import re
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libhk.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-std=c++17", "-O3", "-lineinfo", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
         "-Xcompiler", "-fvisibility=hidden"]


def nvcc():
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found: libhk needs the CUDA toolkit to build")
    return cand


def widths():
    txt = open(os.path.join(CSRC, "widths.h")).read()
    body = re.search(r"HK_FOR_EACH_M\(X\)(.*)", txt).group(1)
    return [int(v) for v in re.findall(r"X\((\d+)\)", body)]


def _sources_digest():
    h = hashlib.sha256()
    for root in (CSRC, os.path.join(HERE, "..", "include")):
        for f in sorted(os.listdir(root)):
            if f.endswith((".cu", ".cuh", ".h")):
                h.update(f.encode())
                h.update(open(os.path.join(root, f), "rb").read())
    h.update(" ".join(ARCH + FLAGS).encode())
    return h.hexdigest()


def build(verbose=False, jobs=None, out_dir=None, defines=()):
    """Compile libhk.so unless an up-to-date one exists; returns its path.

    out_dir / defines: an alternative build directory and extra -D flags
    (used to compare kernel variants side by side)."""
    out = out_dir or OUT
    lib = os.path.join(out, "libhk.so")
    os.makedirs(out, exist_ok=True)
    extra_flags = ["-D" + d for d in defines]
    digest = _sources_digest() + " ".join(extra_flags)
    stamp = os.path.join(out, "libhk.digest")
    if os.path.exists(lib) and os.path.exists(stamp) and open(stamp).read() == digest:
        return lib
    cc = nvcc()
    jobs = jobs or max(2, os.cpu_count() or 2)
    units = [("hk_abi", os.path.join(CSRC, "hk_abi.cu"), []), ("hk_noalloc", os.path.join(CSRC, "hk_noalloc.cu"), [])]
    units += [(f"inst_m{m}", os.path.join(CSRC, "inst.cu"), [f"-DHK_M={m}"]) for m in widths()]

    def compile_one(u):
        name, src, extra = u
        obj = os.path.join(out, name + ".o")
        cmd = [cc] + ARCH + FLAGS + extra_flags + extra + ["-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {name}:\n{r.stderr}")
        if verbose:
            print(name, "ok", file=sys.stderr)
        return obj

    # the heaviest widths first
    units.sort(key=lambda u: -int(u[2][0].split("=")[1]) if u[2] else 0)
    with ThreadPoolExecutor(jobs) as ex:
        objs = list(ex.map(compile_one, units))
    tmp = lib + ".tmp"
    cmd = [cc] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart", "-lpthread"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, lib)
    with open(stamp, "w") as f:
        f.write(digest)
    return lib


if __name__ == "__main__":
    print(build(verbose=True))
