"""Build the FP64 CPU oracle (test infrastructure) into oracle/_build/.

The oracle is plain C compiled with -O3 -ffp-contract=off so that the
compiler never fuses a multiply and an add: every rounding happens where the
source says.  No -march=native: the library is built on one machine and
loaded on another (the GPU machine's host), whose CPU may lack instructions of
the build machine's; -O3 alone changes no rounding (no reassociation without
-ffast-math).  It is independent of the CUDA library and is only loaded by the tests,
the smoke check and the benchmark's CPU-baseline leg.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "rmhd_oracle.c")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "librmhd_oracle.so")


def build(force: bool = False) -> str:
    os.makedirs(OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= max(os.path.getmtime(SRC),
                                             os.path.getmtime(os.path.join(HERE, "rmhd_oracle.h")))):
        return LIB
    cmd = ["gcc", "-O3", "-std=c99", "-ffp-contract=off", "-fno-fast-math",
           "-fPIC", "-shared", "-Wall", "-Wextra", "-o", LIB, SRC, "-lm"]
    subprocess.check_call(cmd)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
