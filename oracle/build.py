"""Compile the CPU oracle (plain C) into a shared library next to this file.

Test infrastructure: the library's product path never builds or loads it.
Flags: -O2, no vector intrinsics, no fused multiply-add contraction, so the
same source gives the same results on x86_64 and aarch64 hosts. -fopenmp
turns on the row-loop pragmas (used to time the oracle on all host cores);
where the compiler has no OpenMP the pragmas are left out and the oracle runs
on one thread with the same results.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "stereo_oracle.c")
LIB = os.path.join(HERE, "liboracle.so")


def build(force: bool = False) -> str:
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
           "-o", LIB + ".tmp", SRC, "-lm"]
    if subprocess.run(cmd[:1] + ["-fopenmp"] + cmd[1:], stdout=subprocess.DEVNULL,
                      stderr=subprocess.DEVNULL).returncode != 0:
        subprocess.run(cmd, check=True)
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
