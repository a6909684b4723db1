"""Build the C-ABI shared library in-tree with nvcc (sm_103a only).

    python -m paper_2606_03989_gb300.build [--verbose-ptxas]

Produces paper_2606_03989_gb300/lib/libpixvod.so (git-ignored). The library
links the CUDA runtime statically and has no dependency on PyTorch.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
LIBDIR = os.path.join(PKG, "lib")
LIB = os.path.join(LIBDIR, "libpixvod.so")
ARCH = "-gencode=arch=compute_103a,code=sm_103a"


def nvcc_path() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the PixVOD CUDA library cannot be built")


def sources():
    return [os.path.join(CSRC, f) for f in ("pixvod.cu", "pixvod_adjoint.cu", "pixvod_static.cu")]


def build(verbose_ptxas: bool = False, force: bool = False) -> str:
    os.makedirs(LIBDIR, exist_ok=True)
    deps = sources() + [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    deps.append(os.path.join(ROOT, "include", "pixvod.h"))
    if not force and os.path.exists(LIB) and all(os.path.getmtime(LIB) >= os.path.getmtime(d) for d in deps):
        return LIB
    tmp = LIB + ".tmp.%d" % os.getpid()
    nvcc = nvcc_path()
    # one object per translation unit, compiled in parallel, then one link
    objs, procs = [], []
    for src in sources():
        obj = os.path.join(LIBDIR, os.path.basename(src) + ".%d.o" % os.getpid())
        cmd = [nvcc, ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-c",
               "-I", os.path.join(ROOT, "include"), "-o", obj, src]
        if verbose_ptxas:
            cmd += ["-Xptxas", "-v"]
        objs.append(obj)
        procs.append(subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
    errors, logs = [], []
    for src, pr in zip(sources(), procs):
        out, err = pr.communicate()
        logs.append(err)
        if pr.returncode != 0:
            errors.append("%s:\n%s%s" % (src, out, err))
    try:
        if errors:
            raise RuntimeError("nvcc failed:\n" + "\n".join(errors))
        res = subprocess.run([nvcc, ARCH, "-shared", "-o", tmp] + objs, capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError("nvcc link failed:\n" + res.stdout + res.stderr)
    finally:
        for obj in objs:
            if os.path.exists(obj):
                os.remove(obj)
    if verbose_ptxas:
        sys.stderr.write("".join(logs))
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(verbose_ptxas="--verbose-ptxas" in sys.argv, force=True))
