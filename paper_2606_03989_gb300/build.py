"""Build the C-ABI shared library in-tree with nvcc (sm_103a only).

    python -m paper_2606_03989_gb300.build [--verbose-ptxas]

Produces paper_2606_03989_gb300/lib/libpixvod.so and its checked variant
lib/libpixvod_checked.so (compiled with PIXVOD_CHECKED: bounds-checked indices,
NaN in the out-of-image lanes of ragged tiles; for tests), both git-ignored.
The libraries link the CUDA runtime statically and have no dependency on
PyTorch.
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
LIB_CHECKED = os.path.join(LIBDIR, "libpixvod_checked.so")
ARCH = "-gencode=arch=compute_103a,code=sm_103a"


def nvcc_path() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the PixVOD CUDA library cannot be built")


def sources():
    return [os.path.join(CSRC, f) for f in ("pixvod.cu", "pixvod_adjoint.cu", "pixvod_static.cu")]


def build(verbose_ptxas: bool = False, force: bool = False) -> str:
    """Build both libraries (the plain one and the checked one) if any source is
    newer; returns the plain library's path."""
    os.makedirs(LIBDIR, exist_ok=True)
    deps = sources() + [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    deps.append(os.path.join(ROOT, "include", "pixvod.h"))
    targets = [(LIB, []), (LIB_CHECKED, ["-DPIXVOD_CHECKED"])]
    stale = [(lib, flags) for lib, flags in targets
             if force or not os.path.exists(lib) or any(os.path.getmtime(lib) < os.path.getmtime(d) for d in deps)]
    if not stale:
        return LIB
    nvcc = nvcc_path()
    # one object per translation unit and library, all compiled in parallel, then one link each
    jobs = []
    for lib, flags in stale:
        for src in sources():
            obj = os.path.join(LIBDIR, "%s.%s.%d.o" % (os.path.basename(lib), os.path.basename(src), os.getpid()))
            cmd = [nvcc, ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-c",
                   "-I", os.path.join(ROOT, "include"), "-o", obj, src] + flags
            if verbose_ptxas and not flags:
                cmd += ["-Xptxas", "-v"]
            jobs.append((lib, src, obj, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.PIPE,
                                                         text=True)))
    errors, logs = [], []
    for lib, src, obj, pr in jobs:
        out, err = pr.communicate()
        logs.append(err)
        if pr.returncode != 0:
            errors.append("%s (%s):\n%s%s" % (src, os.path.basename(lib), out, err))
    try:
        if errors:
            raise RuntimeError("nvcc failed:\n" + "\n".join(errors))
        for lib, _ in stale:
            tmp = lib + ".tmp.%d" % os.getpid()
            objs = [obj for l2, _, obj, _ in jobs if l2 == lib]
            res = subprocess.run([nvcc, ARCH, "-shared", "-o", tmp] + objs, capture_output=True, text=True)
            if res.returncode != 0:
                raise RuntimeError("nvcc link failed:\n" + res.stdout + res.stderr)
            os.replace(tmp, lib)
    finally:
        for _, _, obj, _ in jobs:
            if os.path.exists(obj):
                os.remove(obj)
    if verbose_ptxas:
        sys.stderr.write("".join(logs))
    return LIB


if __name__ == "__main__":
    print(build(verbose_ptxas="--verbose-ptxas" in sys.argv, force=True))
