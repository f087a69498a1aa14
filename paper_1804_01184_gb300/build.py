"""Builds libfwi.so in-tree with nvcc for sm_103a (GB300).

``python -m paper_1804_01184_gb300.build`` or ``build()``; the library lands in
``paper_1804_01184_gb300/_build/libfwi.so`` (git-ignored).  One translation unit, one
-gencode, so a fresh build takes well under a minute.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libfwi.so")
# the debug build: every global access of the time-step kernels bounds-checked (-DFWI_CHECKED)
LIB_CHECKED = os.path.join(OUT_DIR, "libfwi_checked.so")
SOURCES = [os.path.join(CSRC, "fwi_api.cu"), os.path.join(CSRC, "fwi_noalloc.cu")]
# every file the translation units include: a change to any of them rebuilds the library
DEP_SUFFIXES = (".cuh", ".cu", ".h", ".inc")
DEPS = SOURCES + sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(DEP_SUFFIXES)) + \
    sorted(os.path.join(ROOT, "include", f) for f in os.listdir(os.path.join(ROOT, "include")) if f.endswith(".h"))
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc():
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libfwi.so")
    return cand


def cuda_lib_dir():
    base = os.path.dirname(os.path.dirname(os.path.realpath(nvcc())))
    for sub in ("lib64", "lib", "targets/sbsa-linux/lib", "targets/x86_64-linux/lib"):
        p = os.path.join(base, sub)
        if os.path.exists(os.path.join(p, "libcudart.so")) or os.path.exists(p):
            return p
    return os.path.join(base, "lib64")


def up_to_date(lib=None):
    lib = LIB if lib is None else lib
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(p) <= t for p in DEPS)


def _command(out, extra):
    return [nvcc(), *ARCH, "-O3", "-lineinfo", "-std=c++17", "-shared", "-Xcompiler", "-fPIC",
            "-cudart", "shared", "-Xlinker", f"-rpath,{cuda_lib_dir()}", "-I", os.path.join(ROOT, "include"),
            *extra, *SOURCES, "-o", out]


def build(force: bool = False, verbose: bool = False, extra=(), checked: bool = False) -> str:
    """Builds libfwi.so (and, with checked=True, also libfwi_checked.so, the two in parallel);
    returns the path of libfwi.so."""
    todo = [(LIB, list(extra))]
    if checked:
        todo.append((LIB_CHECKED, list(extra) + ["-DFWI_CHECKED"]))
    todo = [(lib, ex) for lib, ex in todo if force or not up_to_date(lib)]
    if not todo:
        return LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    procs = []
    for lib, ex in todo:
        tmp = lib + f".tmp{os.getpid()}"
        cmd = _command(tmp, ex)
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        procs.append((lib, tmp, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True)))
    for lib, tmp, p in procs:
        out, err = p.communicate()
        if p.returncode != 0:
            raise RuntimeError(f"nvcc failed ({p.returncode}) for {os.path.basename(lib)}:\n{out}\n{err}")
        if verbose and err:
            print(err, file=sys.stderr)
        os.replace(tmp, lib)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, checked="--checked" in sys.argv,
                extra=("-Xptxas", "-v") if "--ptxas" in sys.argv else ()))
