"""Build the CPU oracle shared library (test infrastructure only).

Compiles ``hn_oracle.cpp`` with the host C++ compiler into ``liboracle.so`` next to it.  Plain
``-O2`` with floating-point contraction off, so every operation of the oracle rounds as written.
Runs on x86_64 and aarch64 alike (no architecture flags).
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "hn_oracle.cpp")
LIB = os.path.join(HERE, "liboracle.so")


def build(force: bool = False) -> str:
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= os.path.getmtime(SRC)):
        return LIB
    cxx = os.environ.get("CXX", "g++")
    tmp = LIB + ".%d.tmp" % os.getpid()
    cmd = [cxx, "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c++17", "-shared", "-fPIC",
           "-o", tmp, SRC]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
