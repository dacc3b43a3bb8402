"""Build the CUDA library libsdc_gb300.so in-tree for sm_103a with nvcc.

Each source is compiled to an object in parallel, then linked into one shared
library next to this file.  Objects go to ``_build/`` (git-ignored).

``build(checked=True)`` builds libsdc_gb300_checked.so from the same sources with
SDC_CHECKED=1: every gathered index in the kernels is tested against its bound,
and an index outside it makes the call return SDC_E_INVALID instead of reading
out of bounds (a debugging build; objects in ``_build/checked``).  Setting
SDC_GB300_LIB to its path makes the binding load it.
"""

from __future__ import annotations

import concurrent.futures as cf
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
ROOT = os.path.dirname(HERE)
INCLUDE = os.path.join(ROOT, "include")
OBJDIR = os.path.join(ROOT, "_build")
LIB = os.path.join(HERE, "libsdc_gb300.so")
CHECKED_LIB = os.path.join(HERE, "libsdc_gb300_checked.so")
SOURCES = ["api.cu", "assembly.cu", "step.cu", "adjoint.cu", "emi.cu", "coarse.cu", "noalloc.cu",
           "radau.cpp"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-I", INCLUDE,
         "--expt-relaxed-constexpr"]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.isabs(cand) and os.path.exists(cand) or not os.path.isabs(cand)):
            return cand
    return "nvcc"


def _deps():
    out = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    out.append(os.path.join(INCLUDE, "sdc.h"))
    return out


def _stale(target, deps) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, checked: bool = False) -> str:
    lib = CHECKED_LIB if checked else LIB
    objdir = os.path.join(OBJDIR, "checked") if checked else OBJDIR
    os.makedirs(objdir, exist_ok=True)
    deps = _deps()
    if not force and not _stale(lib, deps):
        return lib
    nvcc = _nvcc()
    flags = FLAGS + (["-DSDC_CHECKED=1"] if checked else [])

    def compile_one(src):
        obj = os.path.join(objdir, os.path.splitext(src)[0] + ".o")
        cmd = [nvcc, *ARCH, *flags, "-c", os.path.join(CSRC, src), "-o", obj]
        if src.endswith(".cpp"):
            cmd = [nvcc, *flags, "-x", "c++", "-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            print(" ".join(cmd))
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s%s" % (src, r.stdout, r.stderr))
        return obj

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = lib + ".tmp%d" % os.getpid()
    cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s%s" % (r.stdout, r.stderr))
    os.replace(tmp, lib)
    return lib


def build_all(force: bool = False) -> list:
    """The library and its checked build, compiled side by side."""
    with cf.ThreadPoolExecutor(max_workers=2) as ex:
        futs = [ex.submit(build, force, False, c) for c in (False, True)]
        return [f.result() for f in futs]


if __name__ == "__main__":
    print(build(force=True, verbose=True))
