"""Builds the FP64 CPU oracle (``oracle.c``) into ``liboracle.so`` with gcc.

Test infrastructure: the shared library is loaded by the test suite, the smoke
check and the benchmark's CPU-baseline leg only.
"""
from __future__ import annotations

import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "oracle.c")
LIB = os.path.join(HERE, "liboracle.so")


def build(force: bool = False) -> str:
    """Compiles the oracle when the library is missing or older than its source.

    ``-ffp-contract=off`` keeps gcc from fusing multiply-adds, so every
    expression rounds as written.  OpenMP parallelises the collision loop over
    rows; the result does not depend on the thread count.
    """
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
           "-fPIC", "-shared", "-Wall", "-Wextra", "-o", tmp, SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True))
