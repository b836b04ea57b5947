"""Compile the C oracle into ``oracle/liboracle.so`` (plain gcc, no BLAS).

Test infrastructure only.  ``-ffp-contract=off`` keeps the arithmetic exactly
as written (no fused multiply-add contraction) so the oracle gives the same
bits on x86-64 and aarch64 hosts.  ``-fopenmp`` enables the optional
OpenMP loop over slices of the parallel predictor (off unless
``set_threads`` asks for more than one thread).
"""
from __future__ import annotations

import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "oracle.c")
LIB = os.path.join(HERE, "liboracle.so")


def build(force: bool = False) -> str:
    deps = [SRC, os.path.join(HERE, "oracle.h")]
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= max(os.path.getmtime(p) for p in deps):
        return LIB
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared", "-Wall",
           SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True))
