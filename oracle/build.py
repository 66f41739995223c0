"""Builds the CPU oracle (test infrastructure) into oracle/liboracle.so.

Strict IEEE single/double arithmetic: no fast-math, no FMA contraction, so the FP32
mirror's operation order is exactly the written one.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SOURCES = ["mirror32.cpp", "forward64.cpp", "adjoint64.cpp"]
HEADERS = ["oracle.h", "oracle_internal.h"]
LIB = os.path.join(HERE, "liboracle.so")


def stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(os.path.join(HERE, f)) > t for f in SOURCES + HEADERS)


def build(force: bool = False) -> str:
    if not force and not stale():
        return LIB
    cmd = ["g++", "-std=c++17", "-O2", "-fPIC", "-shared", "-pthread", "-ffp-contract=off",
           "-fno-fast-math", "-Wall", "-Wno-unused-function", "-o", LIB + ".tmp"]
    cmd += [os.path.join(HERE, f) for f in SOURCES]
    subprocess.run(cmd, check=True)
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
