"""Build the sm_103a CUDA library ``liblbm_gb300.so`` in-tree (nvcc, no cmake).

Translation units compile in parallel (one per phase count plus the C ABI), then
link into one shared library next to this file.
"""
from __future__ import annotations

import concurrent.futures as cf
import hashlib
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "liblbm_gb300.so")
LIB_CHECK = os.path.join(HERE, "liblbm_gb300_check.so")  # -DLBM_CHECK_BOUNDS debug variant
UNITS = [f"lbm_kernels_n{n}_{p}.cu" for n in (2, 3, 4) for p in ("fp64", "fp32", "fp16s", "bf16s", "df64")] + ["lbm_capi.cu", "lbm_batch_capi.cu", "lbm_adjoint_capi.cu", "lbm_noalloc.cu", "lbm_slab.cu", "lbm_peak.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-std=c++17", "-O3", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2"]


def _nvcc() -> str:
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build liblbm_gb300.so")
    return nvcc


def _sources_digest(extra=()) -> str:
    h = hashlib.sha256()
    for d in (CSRC, os.path.join(ROOT, "include")):
        for name in sorted(os.listdir(d)):
            if name.endswith((".cu", ".cuh", ".h", ".hpp")):
                with open(os.path.join(d, name), "rb") as fh:
                    h.update(name.encode() + fh.read())
    h.update(" ".join(ARCH + FLAGS + list(extra)).encode())
    return h.hexdigest()


def kernel_digest() -> str:
    """Digest of what the device kernels are compiled from: the headers of csrc/ and the
    kernel units lbm_kernels_*.cu (the C ABI units and include/lbm.h are host code that
    no kernel includes), with comments removed, and the compiler flags.  Measured
    per-kernel counts are tied to it."""
    import re
    h = hashlib.sha256()
    for name in sorted(os.listdir(CSRC)):
        if name.endswith(".cuh") or (name.startswith("lbm_kernels_") and name.endswith(".cu")):
            with open(os.path.join(CSRC, name)) as fh:
                text = fh.read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            text = re.sub(r"//[^\n]*", "", text)
            text = "\n".join(line.rstrip() for line in text.splitlines() if line.strip())
            h.update(name.encode() + text.encode())
    h.update(" ".join(ARCH + FLAGS).encode())
    return h.hexdigest()


def build(force: bool = False, verbose: bool = False, check_bounds: bool = False) -> str:
    """Compile (if sources changed) and return the path of liblbm_gb300.so.

    check_bounds=True builds the debug variant liblbm_gb300_check.so instead, in which
    every global access of the kernels is bounds-checked (see lbm_debug_bounds)."""
    extra = ["-DLBM_CHECK_BOUNDS"] if check_bounds else []
    lib_path = LIB_CHECK if check_bounds else LIB
    bdir = os.path.join(BUILD, "check" if check_bounds else "release")
    os.makedirs(bdir, exist_ok=True)
    stamp = os.path.join(bdir, "digest")
    digest = _sources_digest(extra)
    if not force and os.path.exists(lib_path) and os.path.exists(stamp):
        with open(stamp) as fh:
            if fh.read().strip() == digest:
                return lib_path
    nvcc = _nvcc()

    def compile_one(unit):
        obj = os.path.join(bdir, unit.replace(".cu", ".o"))
        cmd = [nvcc] + FLAGS + extra + ARCH + ["-I", os.path.join(ROOT, "include"), "-c", os.path.join(CSRC, unit),
                                               "-o", obj]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {unit}:\n{r.stderr}")
        return obj, r.stderr

    with cf.ThreadPoolExecutor(max_workers=min(len(UNITS), os.cpu_count() or 4)) as ex:
        results = list(ex.map(compile_one, UNITS))
    if verbose:
        for _, log in results:
            print(log)
    tmp = lib_path + ".tmp"
    cmd = [nvcc] + ARCH + ["-shared", "-o", tmp] + [o for o, _ in results] + ["-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, lib_path)
    with open(stamp, "w") as fh:
        fh.write(digest)
    return lib_path


if __name__ == "__main__":
    print(build(force=True, verbose=True))
