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


TANGENT_LIB = os.path.join(OUT_DIR, "librmhd_oracle_tangent.so")


def _stale(lib, deps):
    return not os.path.exists(lib) or os.path.getmtime(lib) < max(
        os.path.getmtime(os.path.join(HERE, f)) for f in deps)


def build(force: bool = False) -> str:
    os.makedirs(OUT_DIR, exist_ok=True)
    if force or _stale(LIB, ("rmhd_oracle.c", "rmhd_oracle.h")):
        cmd = ["gcc", "-O3", "-std=c99", "-ffp-contract=off", "-fno-fast-math",
               "-fPIC", "-shared", "-Wall", "-Wextra", "-o", LIB, SRC, "-lm"]
        subprocess.check_call(cmd)
    return LIB


def build_tangent(force: bool = False) -> str:
    """The tangent-linear build: the same source compiled as C++ with the
    arithmetic on tangent numbers (tangent.h), same flags otherwise; the
    values it computes are those of the plain build, operation for
    operation."""
    os.makedirs(OUT_DIR, exist_ok=True)
    if force or _stale(TANGENT_LIB, ("rmhd_oracle.c", "rmhd_oracle.h", "tangent.h")):
        cmd = ["g++", "-O3", "-std=c++17", "-x", "c++", "-DORC_TANGENT", "-ffp-contract=off",
               "-fno-fast-math", "-fPIC", "-shared", "-Wall", "-Wextra",
               "-Wno-class-memaccess", "-o", TANGENT_LIB, SRC, "-lm"]
        subprocess.check_call(cmd)
    return TANGENT_LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
    print(build_tangent(force="--force" in sys.argv))
