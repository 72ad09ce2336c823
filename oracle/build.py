"""Compile the FP64 CPU oracle (test infrastructure) into oracle/liboracle.so.

Plain g++ with IEEE arithmetic (no fast-math, no FMA contraction) so that the
oracle's FP64 sums are the sequential sums its source states.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "kann_oracle.cpp")
LIB = os.path.join(HERE, "liboracle.so")


def compile_source(src: str, out: str) -> str:
    """Compile an oracle source file into the shared library `out` (the
    oracle's own flags; the tests also build copies with planted mistakes)."""
    cmd = ["g++", "-std=c++17", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
           "-shared", "-fPIC", "-o", out, src]
    subprocess.check_call(cmd)
    return out


def build(force: bool = False) -> str:
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    tmp = LIB + ".tmp%d" % os.getpid()
    compile_source(SRC, tmp)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
