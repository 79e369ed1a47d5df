"""Build the CUDA library (sm_103a) in-tree: paper_2510_18968_b300/librmhd.so.

The translation units are compiled in parallel (one per metric / precision
combination of the step, one for the adjoint, one for the API and one for
the allocation-free entry point) and linked into one shared library."""
import concurrent.futures as cf
import glob
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "librmhd.so")
OBJ_DIR = os.path.join(HERE, "_build")
SOURCES = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
HEADERS = sorted(glob.glob(os.path.join(CSRC, "*.cuh"))) + [
    os.path.join(os.path.dirname(HERE), "include", "rmhd.h")]

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17"] + ARCH + ["-lineinfo", "-Xcompiler", "-fPIC",
                                              "--expt-relaxed-constexpr"]


def _obj(src):
    return os.path.join(OBJ_DIR, os.path.splitext(os.path.basename(src))[0] + ".o")


def _compile(src, verbose):
    cmd = ["nvcc"] + NVCC_FLAGS + (["-Xptxas", "-v"] if verbose else []) + [
        "-c", src, "-o", _obj(src)]
    r = subprocess.run(cmd, capture_output=True, text=True)
    return src, r.returncode, r.stdout + r.stderr


def build(force=False, verbose=False):
    deps_mtime = max(os.path.getmtime(f) for f in SOURCES + HEADERS)
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= deps_mtime:
        return LIB
    os.makedirs(OBJ_DIR, exist_ok=True)
    hdr_mtime = max(os.path.getmtime(f) for f in HEADERS)
    todo = [s for s in SOURCES if force or not os.path.exists(_obj(s))
            or os.path.getmtime(_obj(s)) < max(os.path.getmtime(s), hdr_mtime)]
    with cf.ThreadPoolExecutor(max_workers=max(1, min(len(todo), os.cpu_count() or 1))) as ex:
        for src, rc, out in ex.map(lambda s: _compile(s, verbose), todo):
            if verbose or rc:
                sys.stderr.write(out)
            if rc:
                raise subprocess.CalledProcessError(rc, "nvcc -c " + src)
    subprocess.check_call(["nvcc"] + ARCH + ["-shared", "-o", LIB] + [_obj(s) for s in SOURCES])
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
