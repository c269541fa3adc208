"""Build the FP64 CPU oracle (test infrastructure only) into oracle/liboracle.so.

The oracle is plain C++17 compiled with -ffp-contract=off so that every
addition and multiplication is rounded separately, in source order.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
LIB = os.path.join(HERE, "liboracle.so")
SOURCES = ["oracle.cpp"]
HEADERS = ["real.hpp", "euler.hpp", "reconstruct.hpp", "riemann.hpp", "schemes.hpp"]


def needs_build() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(os.path.join(HERE, f)) > t for f in SOURCES + HEADERS)


def build(force: bool = False) -> str:
    if force or needs_build():
        tmp = LIB + ".tmp%d" % os.getpid()
        cmd = ["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
               "-o", tmp] + [os.path.join(HERE, s) for s in SOURCES]
        subprocess.run(cmd, check=True)
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
