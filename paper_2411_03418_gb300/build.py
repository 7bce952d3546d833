"""In-tree build of libmarfa (CUDA, sm_103a) with nvcc; no cmake, no setuptools.

The translation units are compiled in parallel and linked into
``paper_2411_03418_gb300/_build/libmarfa.so``. Host code is compiled with
``-ffp-contract=off`` so that the FP64 centre and width arithmetic rounds the same
way on x86-64 and aarch64 hosts. ``build(debug=True)`` makes the MARFA_DEBUG variant,
``_build/libmarfa_debug.so``, whose kernels check their indexed accesses and report a
failed check through the call's return code instead of trapping.
"""
from __future__ import annotations

import hashlib
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libmarfa.so")
LIB_DEBUG = os.path.join(BUILD, "libmarfa_debug.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
SOURCES = ["marfa_api.cu", "marfa_kernels.cu", "marfa_mlp.cu"]
DEPS = SOURCES + ["marfa_internal.cuh", "mlp.cuh", "ownership.cuh", "voigt.cuh", "voigt_tables.inc"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-std=c++17", "-O3", "-lineinfo", "-Xcompiler", "-fPIC,-ffp-contract=off,-pthread", "-I", INCLUDE]


def _nvcc() -> str:
    p = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(p):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libmarfa")
    return p


def _stamp(flags) -> str:
    h = hashlib.sha256()
    for f in DEPS + [os.path.join("..", "..", "include", "marfa.h")]:
        with open(os.path.join(CSRC, f), "rb") as fh:
            h.update(fh.read())
    h.update(" ".join(ARCH + flags).encode())
    h.update(os.uname().machine.encode())
    return h.hexdigest()


def build(force: bool = False, verbose: bool = False, debug: bool = False) -> str:
    """Compile libmarfa (debug: the MARFA_DEBUG variant) if its sources changed since the
    last build; return its path."""
    os.makedirs(BUILD, exist_ok=True)
    lib = LIB_DEBUG if debug else LIB
    flags = FLAGS + (["-DMARFA_DEBUG"] if debug else [])
    tag = "_debug" if debug else ""
    stamp_file = os.path.join(BUILD, "stamp" + tag)
    stamp = _stamp(flags)
    if not force and os.path.exists(lib) and os.path.exists(stamp_file):
        if open(stamp_file).read().strip() == stamp:
            return lib
    nvcc = _nvcc()

    def compile_one(src):
        obj = os.path.join(BUILD, src.replace(".cu", tag + ".o"))
        cmd = [nvcc, *ARCH, *flags, "-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        if verbose:
            sys.stdout.write(r.stdout + r.stderr)
        return obj

    with ThreadPoolExecutor(len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = lib + ".tmp"
    cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-lpthread"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)
    with open(stamp_file, "w") as f:
        f.write(stamp)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, debug="--debug" in sys.argv))
