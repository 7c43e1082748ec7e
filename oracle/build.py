"""Compile the plain-C FEAST oracle (test infrastructure only).

Builds ``oracle/_build/liboracle.so`` with gcc.  ``-fcx-limited-range`` gives
textbook complex multiply/divide (no Annex-G inf/NaN recovery calls);
OpenMP spreads the independent contour nodes over host threads (the guide's
second level of parallelism) and nothing else.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "liboracle.so")
SRC = [os.path.join(HERE, "feast_oracle.c")]


def build(force: bool = False) -> str:
    hdr = os.path.join(HERE, "feast_oracle.h")
    newest = max(os.path.getmtime(p) for p in SRC + [hdr])
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= newest:
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-std=gnu11", "-O2", "-fPIC", "-shared", "-fopenmp",
           "-fcx-limited-range", "-o", tmp] + SRC + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True))
