"""Compile the CUDA library (libsph_gb300.so) for sm_103a with nvcc.

Six translation units compiled in parallel, linked as a shared library
with the static CUDA runtime.  Run as ``python -m paper_2207_11328_gb300._build``
or through ``__graft_entry__.build()``.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(HERE, "libsph_gb300.so")
OBJDIR = os.path.join(ROOT, "_build")
SOURCES = ["sph_api.cu", "neighbors.cu", "forces.cu", "forces_models.cu", "adjoint.cu", "measure.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# The interaction kernels contract only the FMAs written as fmaf(): with the
# compiler free to fuse a separate multiply and add, launch shapes with
# different register caps could round differently, and every shape (and a
# batched scene against the same scene alone) must give the same bits.
EXTRA = {"forces.cu": ["-fmad=false"], "forces_models.cu": ["-fmad=false"]}


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build the library")


def _flags(extra=()):
    return ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC,
                   *extra]


def _compile(nvcc, src, obj, verbose_ptxas=False):
    extra = EXTRA.get(src, []) + (["-Xptxas", "-v"] if verbose_ptxas else [])
    cmd = [nvcc, *_flags(extra), "-c", os.path.join(CSRC, src), "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stderr}")
    return r.stderr


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(INCLUDE, "sph.h")]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose_ptxas: bool = False) -> str:
    if not force and not _stale():
        return LIB
    nvcc = _nvcc()
    os.makedirs(OBJDIR, exist_ok=True)
    objs = [os.path.join(OBJDIR, s.replace(".cu", ".o")) for s in SOURCES]
    with cf.ThreadPoolExecutor(len(SOURCES)) as ex:
        logs = list(ex.map(lambda a: _compile(nvcc, a[0], a[1], verbose_ptxas), zip(SOURCES, objs)))
    if verbose_ptxas:
        for s, log in zip(SOURCES, logs):
            sys.stderr.write(f"== {s}\n{log}")
    tmp = LIB + f".tmp{os.getpid()}"
    r = subprocess.run([nvcc, *ARCH, "-shared", "-o", tmp, *objs], capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose_ptxas="-v" in sys.argv))
