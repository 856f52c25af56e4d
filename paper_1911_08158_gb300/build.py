"""Compile the CUDA library in-tree: paper_1911_08158_gb300/_build/libads_gb300.so.

nvcc for sm_103a only (-gencode arch=compute_103a,code=sm_103a), one object
per translation unit compiled in parallel, then one shared library linked
against the shared CUDA runtime.  Cross-compiles without a GPU.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libads_gb300.so")
SOURCES = ["rhs_f32.cu", "rhs_f32_s33.cu", "rhs_f32_s44.cu", "rhs_f64.cu", "rhs_f64_s33.cu", "rhs_f64_s44.cu",
           "col_f32.cu", "col_f64.cu", "kernels.cu", "api.cpp", "setup1d.cpp",
           "noalloc.cu", "peaks.cu", "rhs_el_f32.cu", "rhs_el_f32_s33.cu", "rhs_el_f32_s44.cu", "rhs_el_f64.cu",
           "rhs_el_f64_s33.cu", "rhs_el_f64_s44.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(ROOT, "include", "ads.h")]
    return any(os.path.getmtime(p) > t for p in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and not _stale():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    nv = nvcc()
    common = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-I", os.path.join(ROOT, "include"),
              "-I", CSRC]

    def compile_one(src):
        obj = os.path.join(BUILD, src + ".o")
        cmd = [nv] + ARCH + common + ["-c", os.path.join(CSRC, src), "-o", obj]
        if src.endswith(".cu"):
            cmd += ["-Xptxas", "-v"] if verbose else []
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (src, r.stdout, r.stderr))
        return obj, r.stderr

    with cf.ThreadPoolExecutor(len(SOURCES)) as ex:
        results = list(ex.map(compile_one, SOURCES))
    if verbose:
        for _, err in results:
            print(err)
    tmp = LIB + ".tmp.%d" % os.getpid()
    cmd = [nv] + ARCH + ["-shared", "--cudart", "shared", "-o", tmp] + [o for o, _ in results]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s\n%s" % (r.stdout, r.stderr))
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    import sys
    print(build(force=True, verbose="-v" in sys.argv))
