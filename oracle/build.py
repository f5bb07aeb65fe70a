"""Compile the C oracle (oracle.c) into liboracle.so beside it.

Test infrastructure: the tests, the smoke check and the bench's CPU-baseline
leg load the result; the library's product path never does.  ISO C mode keeps
floating-point contraction off, so the oracle rounds the same way on x86-64
and on AArch64.
"""
from __future__ import annotations

import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "oracle.c")
LIB = os.path.join(HERE, "liboracle.so")


def build(force: bool = False) -> str:
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    base = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-shared", "-fPIC"]
    tmp = LIB + ".tmp"
    try:
        subprocess.check_call(base + ["-fopenmp", SRC, "-o", tmp, "-lm"])
    except subprocess.CalledProcessError:
        # a toolchain without OpenMP still builds the (single-threaded) oracle
        subprocess.check_call(base + [SRC, "-o", tmp, "-lm"])
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True))
