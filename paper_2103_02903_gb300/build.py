"""Build of the CUDA library ``libmrlbm.so`` (sm_103a) from ``csrc/``.

Each translation unit is compiled in parallel with nvcc for
``-gencode arch=compute_103a,code=sm_103a`` and the objects are linked into
one shared library next to this file.  The library exports the C-ABI of
``include/mr_lbm.h`` and links only the CUDA runtime.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libmrlbm.so")
SOURCES = ["mr_api.cu", "mr_encode.cu", "mr_mesh.cu", "mr_stream.cu", "mr_noalloc.cu", "mr_adjoint.cu",
           "mr_exact.cu", "mr_wide.cu"]
HEADERS = ["mr_internal.cuh", "mr_common.cuh", "mr_handle.cuh", "mr_schemes.cuh", "mr_wide.cuh"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc():
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libmrlbm.so")


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, s) for s in SOURCES + HEADERS]
    deps.append(os.path.join(ROOT, "include", "mr_lbm.h"))
    deps.append(os.path.abspath(__file__))
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and not _stale():
        return LIB
    nvcc = _nvcc()
    os.makedirs(BUILD, exist_ok=True)
    common = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                     "-I", os.path.join(ROOT, "include")]
    if verbose:
        common += ["-Xptxas", "-v"]
    procs = []
    objs = []
    for s in SOURCES:
        obj = os.path.join(BUILD, s.replace(".cu", ".o"))
        objs.append(obj)
        cmd = [nvcc, "-c", os.path.join(CSRC, s), "-o", obj] + common
        procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    errors = []
    for cmd, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0 or verbose:
            (errors if p.returncode != 0 else [sys.stdout]).append(out.decode()) if p.returncode != 0 \
                else sys.stdout.write(out.decode())
    if errors:
        raise RuntimeError("nvcc failed:\n" + "\n".join(errors))
    tmp = LIB + ".tmp%d" % os.getpid()
    subprocess.run([nvcc, "-shared"] + ARCH + ["-o", tmp] + objs + ["-lcudart"], check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose="-v" in sys.argv))
