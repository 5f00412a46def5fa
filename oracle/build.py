"""Build the FP64 CPU oracle (test infrastructure only) into oracle/lib/liboracle.so.

Plain g++ with OpenMP; no CUDA.  Called by __graft_entry__.build() and, on
demand, by oracle.oracle when the library is missing.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_DIR = os.path.join(HERE, "lib")
LIB_PATH = os.path.join(LIB_DIR, "liboracle.so")
SOURCES = [os.path.join(HERE, "fr_oracle.cpp")]


def build(force: bool = False) -> str:
    """Compile the oracle if it is missing or older than its sources."""
    os.makedirs(LIB_DIR, exist_ok=True)
    newest = max(os.path.getmtime(s) for s in SOURCES + [os.path.join(HERE, "fr_oracle.h")])
    if not force and os.path.exists(LIB_PATH) and os.path.getmtime(LIB_PATH) >= newest:
        return LIB_PATH
    tmp = LIB_PATH + ".tmp.%d" % os.getpid()
    cmd = ["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
           "-o", tmp] + SOURCES
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB_PATH)
    return LIB_PATH


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
