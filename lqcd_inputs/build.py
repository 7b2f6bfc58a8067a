"""Compile lqcd_inputs/philox.c into lqcd_inputs/libphilox.so (gcc, OpenMP).

    python lqcd_inputs/build.py

philox.py uses the compiled words when this library is present and its own numpy rounds
otherwise; both give the same 32-bit words (tests/test_inputs.py checks them against each other
and against the published known answers).
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "philox.c")
LIB = os.path.join(HERE, "libphilox.so")


def build(force=False):
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    subprocess.run(["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", SRC, "-o", LIB, "-lm"], check=True)
    return LIB


if __name__ == "__main__":
    print(build("--force" in sys.argv))
