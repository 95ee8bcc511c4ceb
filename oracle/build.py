"""Builds the oracle's shared library (test infrastructure only).

Plain g++, FP contraction off so that the FP32 instantiation rounds every
operation separately, OpenMP over patches.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
LIB = os.path.join(HERE, "liboracle.so")
SOURCES = ["capi.cpp"]
HEADERS = ["codec.hpp", "entropy.hpp", "mlp.hpp", "schemes.hpp", "sim.hpp", "sim3.hpp", "wavelet.hpp"]


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(os.path.join(HERE, f)) > t for f in SOURCES + HEADERS)


def build_oracle(force: bool = False) -> str:
    if force or _stale():
        cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
               "-fno-fast-math", "-Wall", "-o", LIB + ".tmp"] + [os.path.join(HERE, s) for s in SOURCES]
        subprocess.check_call(cmd)
        os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build_oracle(force="--force" in sys.argv))
