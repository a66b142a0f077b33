"""Build of the CUDA library ``_lib/libdugks.so`` for sm_103a (GB300).

nvcc with ``-gencode arch=compute_103a,code=sm_103a``: the 2-D translation
unit (``dugks_api.cu``) and the 3-D one (``dugks3d_api.cu``) compile to
objects in parallel and link into one shared library; it is rebuilt when a
source or a header is newer than it.
"""
from __future__ import annotations

import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
LIBDIR = os.path.join(HERE, "_lib")
LIB = os.path.join(LIBDIR, "libdugks.so")
SOURCES = [os.path.join(CSRC, "dugks_api.cu"), os.path.join(CSRC, "dugks3d_api.cu")]
DEPS = SOURCES + [os.path.join(CSRC, f) for f in ("dugks_device.cuh", "dugks_kernels.cuh", "dugks_step_vp.cuh", "dugks_adjoint.cuh",
                                                  "dugks_batch.cuh", "dugks3d_kernels.cuh", "dugks3d_halves.cuh", "dugks_adjoint_rows.cuh")] + [
    os.path.join(ROOT, "include", "dugks.h"), os.path.join(ROOT, "include", "dugks3d.h")]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    return "nvcc"


def stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(d) > t for d in DEPS)


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and not stale():
        return LIB
    os.makedirs(LIBDIR, exist_ok=True)
    tag = f".tmp{os.getpid()}"
    objs, procs = [], []
    for src in SOURCES:
        obj = os.path.join(LIBDIR, os.path.basename(src) + tag + ".o")
        cmd = [nvcc(), *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-c", "-o", obj, src]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        objs.append(obj)
        procs.append((cmd, subprocess.Popen(cmd)))
    failed = [cmd for cmd, pr in procs if pr.wait() != 0]
    if failed:
        raise subprocess.CalledProcessError(1, failed[0])
    tmp = LIB + tag
    subprocess.check_call([nvcc(), *ARCH, "-shared", "-o", tmp, *objs])
    for obj in objs:
        os.remove(obj)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
