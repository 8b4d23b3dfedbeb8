"""Compile the FP64 CPU oracle (test infrastructure) into oracle/liboracle.so.

g++ with OpenMP and no floating-point contraction, so the oracle rounds the
same way on x86-64 and on aarch64 hosts.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SOURCES = ["or_table.cpp", "or_fill.cpp"]
LIB = os.path.join(HERE, "liboracle.so")


def needs_build():
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = SOURCES + ["oracle.h", "or_types.h"]
    return any(os.path.getmtime(os.path.join(HERE, s)) > t for s in deps)


def build(force=False):
    if not force and not needs_build():
        return LIB
    cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-o", LIB + ".tmp"] + [os.path.join(HERE, s) for s in SOURCES]
    subprocess.run(cmd, check=True)
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
