"""Compile the oracle's C core (kkt_dense.c) into oracle/_kkt_dense.so.

Test infrastructure only (see oracle/__init__.py).  Plain gcc, -O2, no fast-math, OpenMP
over independent (sample, component) problems.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "kkt_dense.c")
LIB = os.path.join(HERE, "_kkt_dense.so")


def build(force: bool = False) -> str:
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= os.path.getmtime(SRC)):
        return LIB
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-fno-fast-math",
           SRC, "-o", LIB + ".tmp", "-lm"]
    subprocess.check_call(cmd)
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
