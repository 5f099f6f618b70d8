"""Builds the C++/OpenMP oracle (oracle/cpp/hk_oracle.cpp) into oracle/_build.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``): the program is run by
tests/ and by bench.py's CPU-baseline legs, never by the library.  Plain g++
with OpenMP; no architecture-specific flags, so the same source builds on
x86-64 and on Arm hosts.
"""
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "cpp", "hk_oracle.cpp")
OUT = os.path.join(HERE, "_build")
EXE = os.path.join(OUT, "hk_oracle")


def build():
    """Compile hk_oracle unless an up-to-date binary exists; returns its path."""
    os.makedirs(OUT, exist_ok=True)
    if os.path.exists(EXE) and os.path.getmtime(EXE) >= os.path.getmtime(SRC):
        return EXE
    cxx = shutil.which("g++") or "g++"
    cmd = [cxx, "-O2", "-std=c++17", "-fopenmp", SRC, "-o", EXE + ".tmp"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("building the C++ oracle failed:\n" + r.stderr)
    os.replace(EXE + ".tmp", EXE)
    return EXE


if __name__ == "__main__":
    print(build())
