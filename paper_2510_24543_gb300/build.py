"""In-tree build of libegpe.so for sm_103a (nvcc, parallel per translation unit).

``build()`` compiles the CUDA sources under ``csrc/`` to objects in ``_build/``
(repo root, git-ignored) and links ``paper_2510_24543_gb300/libegpe.so``.  A
stamp of the source hashes skips the work when nothing changed.
"""
from __future__ import annotations

import hashlib
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(ROOT, "_build")
LIB = os.path.join(PKG, "libegpe.so")
UNITS = ["capi.cu", "engine_f64.cu", "engine_f32.cu", "engine_mr_f64.cu", "engine_mr_f32.cu", "engine_mr5_f64.cu",
         "engine_mr5_f32.cu", "engine_big_f64.cu", "engine_big_f32.cu"]
# The FP32-field engine flushes denormals and uses the approximate (MUFU)
# divide and square root: values below 1e-38 carry no weight in any sum of that
# path, and its fields are accurate to ~1e-7 anyway.  The FP64 engine keeps
# IEEE division and square root.
_FP32_FLAGS = ["-ftz=true", "-prec-div=false", "-prec-sqrt=false"]
UNIT_FLAGS = {u: _FP32_FLAGS for u in UNITS if u.endswith("f32.cu")}
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I" + INCLUDE]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libegpe.so")


def _digest() -> str:
    h = hashlib.sha256()
    for d in (CSRC, INCLUDE):
        for name in sorted(os.listdir(d)):
            if name.endswith((".cu", ".cuh", ".h")):
                with open(os.path.join(d, name), "rb") as f:
                    h.update(name.encode() + f.read())
    # flags without the machine-specific include path, so the digest names the
    # sources and options alone (it stamps profiles taken on another machine)
    h.update(" ".join(ARCH + [f for f in FLAGS if not f.startswith("-I")]).encode())
    h.update(repr(sorted(UNIT_FLAGS.items())).encode())
    return h.hexdigest()


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile (if needed) and return the path of libegpe.so."""
    os.makedirs(BUILD, exist_ok=True)
    stamp = os.path.join(BUILD, "libegpe.stamp")
    dig = _digest()
    if not force and os.path.exists(LIB) and os.path.exists(stamp):
        with open(stamp) as f:
            if f.read().strip() == dig:
                return LIB
    nvcc = _nvcc()

    def compile_unit(unit):
        src = os.path.join(CSRC, unit)
        obj = os.path.join(BUILD, unit.replace(".cu", ".o"))
        cmd = [nvcc] + ARCH + FLAGS + UNIT_FLAGS.get(unit, []) + ["-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {unit}:\n{r.stdout}\n{r.stderr}")
        if verbose:
            sys.stderr.write(r.stderr)
        return obj

    with ThreadPoolExecutor(max_workers=len(UNITS)) as ex:
        objs = list(ex.map(compile_unit, UNITS))
    tmp = LIB + ".tmp"
    cmd = [nvcc] + ARCH + ["-shared", "-o", tmp] + objs
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    with open(stamp, "w") as f:
        f.write(dig)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
