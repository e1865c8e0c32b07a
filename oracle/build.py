"""Compiles the CPU oracle (pipnn_oracle.c) into liborc.so beside this file.

TEST INFRASTRUCTURE: the oracle library is built so that the test suite, the smoke check and the
benchmark's CPU-baseline leg can load it; nothing on the product path uses it.

Flags: -ffp-contract=off keeps every binary32 operation exactly as written (the oracle's fused
multiply-adds are explicit fmaf calls and nothing else may be fused); OpenMP parallelises the
outer loops over points, leaves and nodes, whose iterations are independent.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "pipnn_oracle.c")
LIB = os.path.join(HERE, "liborc.so")


def build(force: bool = False) -> str:
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-fno-fast-math", "-Wall", "-Wno-unused-function", "-o", tmp, SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
