"""Builds liboracle.so from cox_oracle.cpp with the host C++ compiler.

Part of the oracle (test infrastructure).  Plain g++, no CUDA, no flags that
depend on the host CPU, so it builds the same on x86_64 and aarch64.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "cox_oracle.cpp")


def lib_path() -> str:
    return os.path.join(HERE, "liboracle.so")


def build(force: bool = False) -> str:
    out = lib_path()
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(SRC):
        return out
    cxx = os.environ.get("CXX", "g++")
    tmp = out + f".tmp{os.getpid()}"
    cmd = [cxx, "-O2", "-std=c++17", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-pthread", "-Wall", "-o", tmp, SRC]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
