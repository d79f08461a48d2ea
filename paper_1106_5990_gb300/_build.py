"""Compile the CUDA C-ABI library in-tree: paper_1106_5990_gb300/_lib/libamgd.so.

One translation unit per source file, compiled in parallel by nvcc for
sm_103a only, then linked into a shared library with the CUDA runtime linked
statically (the library has no torch dependency).
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
LIBDIR = os.path.join(HERE, "_lib")
LIB = os.path.join(LIBDIR, "libamgd.so")
# the checked build: every gather index of the sweep and distance kernels is
# bounds-tested in the kernel (AMGD_CHECKS); for tests, loaded with AMGD_CHECKED=1
LIB_CHECKED = os.path.join(LIBDIR, "libamgd_checked.so")
SOURCES = ["amgd_api.cu", "k_relax.cu", "k_edge.cu", "k_edge_f64.cu", "k_edge_f32.cu",
           "k_edge_f32c.cu", "k_edge_bf16.cu", "k_edge_bf16c.cu", "k_init.cu", "k_compact.cu",
           "amgd_noalloc.cu", "k_adjoint.cu", "k_interp.cu", "k_cr.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
         "-Xcompiler", "-Wall"]


def nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libamgd.so")


def _deps_mtime() -> float:
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files.append(os.path.join(os.path.dirname(HERE), "include", "amgd.h"))
    files.append(os.path.abspath(__file__))
    return max(os.path.getmtime(f) for f in files)


def build(force: bool = False, verbose: bool = False, extra: list | None = None,
          checked: bool = False) -> str:
    os.makedirs(LIBDIR, exist_ok=True)
    lib = LIB_CHECKED if checked else LIB
    if not force and os.path.exists(lib) and os.path.getmtime(lib) >= _deps_mtime():
        return lib
    cc = nvcc()
    objdir = os.path.join(LIBDIR, "obj_checked" if checked else "obj")
    os.makedirs(objdir, exist_ok=True)
    extra = list(extra or []) + (["-DAMGD_CHECKS=1"] if checked else [])

    def compile_one(src):
        obj = os.path.join(objdir, os.path.splitext(src)[0] + ".o")
        cmd = [cc, *ARCH, *FLAGS, *extra, "-c", os.path.join(CSRC, src), "-o", obj]
        p = subprocess.run(cmd, capture_output=True, text=True)
        return src, obj, p

    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        results = list(ex.map(compile_one, SOURCES))
    errs = [(s, p) for s, _, p in results if p.returncode != 0]
    for s, _, p in results:
        if verbose and (p.stdout or p.stderr):
            sys.stderr.write("== %s\n%s%s" % (s, p.stdout, p.stderr))
    if errs:
        msg = "\n".join("== %s\n%s%s" % (s, p.stdout, p.stderr) for s, p in errs)
        raise RuntimeError("nvcc failed:\n" + msg)
    tmp = lib + ".%d.tmp" % os.getpid()
    cmd = [cc, *ARCH, "-shared", "-o", tmp] + [o for _, o, _ in results] + ["-cudart", "static"]
    p = subprocess.run(cmd, capture_output=True, text=True)
    if p.returncode != 0:
        raise RuntimeError("link failed:\n" + p.stdout + p.stderr)
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, checked="--checked" in sys.argv,
                extra=["-Xptxas", "-v"] if "--ptxas" in sys.argv else None))
