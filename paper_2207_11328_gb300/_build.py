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
LIB_CHECKED = os.path.join(HERE, "libsph_gb300_checked.so")  # -DSPH_CHECKED: bounds checks, canaries
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


def _compile(nvcc, src, obj, verbose_ptxas=False, checked=False):
    extra = EXTRA.get(src, []) + (["-Xptxas", "-v"] if verbose_ptxas else []) + (["-DSPH_CHECKED"] if checked else [])
    cmd = [nvcc, *_flags(extra), "-c", os.path.join(CSRC, src), "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stderr}")
    return r.stderr


def _stale(lib=LIB) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(INCLUDE, "sph.h")]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose_ptxas: bool = False, checked: bool = False) -> str:
    """Build the library (checked=True: the variant compiled with SPH_CHECKED)."""
    lib = LIB_CHECKED if checked else LIB
    if not force and not _stale(lib):
        return lib
    nvcc = _nvcc()
    objdir = os.path.join(OBJDIR, "checked") if checked else OBJDIR
    os.makedirs(objdir, exist_ok=True)
    objs = [os.path.join(objdir, s.replace(".cu", ".o")) for s in SOURCES]
    with cf.ThreadPoolExecutor(len(SOURCES)) as ex:
        logs = list(ex.map(lambda a: _compile(nvcc, a[0], a[1], verbose_ptxas, checked), zip(SOURCES, objs)))
    if verbose_ptxas:
        for s, log in zip(SOURCES, logs):
            sys.stderr.write(f"== {s}\n{log}")
    tmp = lib + f".tmp{os.getpid()}"
    r = subprocess.run([nvcc, *ARCH, "-shared", "-o", tmp, *objs], capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


def build_all(force: bool = False) -> list:
    """Both libraries, compiled concurrently."""
    with cf.ThreadPoolExecutor(2) as ex:
        return list(ex.map(lambda c: build(force=force, checked=c), (False, True)))


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose_ptxas="-v" in sys.argv, checked="--checked" in sys.argv))
