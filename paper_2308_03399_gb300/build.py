"""Build libsv.so (CUDA kernels + C++ runtime) in-tree for sm_103a with nvcc.

The two translation units compile in parallel; the result lands in
paper_2308_03399_gb300/_build/libsv.so.  Nothing is installed elsewhere.
"""
from __future__ import annotations

import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libsv.so")
SOURCES = ["sv_kernels.cu", "sv_reg_c64.cu", "sv_reg_c64x.cu", "sv_reg_c128.cu", "sv_runtime.cu", "sv_noalloc.cu",
           "sv_mlp.cu", "sv_dm.cu"]
HEADERS = ["sv_internal.h", "sv_sample.cuh", os.path.join("..", "..", "include", "sv.h"), "sv_common.cuh", "sv_pass_reg.cuh", "sv_pass_whole.cuh"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2"]


def nvcc() -> str:
    p = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(p):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libsv")
    return p


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, s) for s in SOURCES + HEADERS]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and not _stale():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    cc = nvcc()
    objs, procs = [], []
    for s in SOURCES:
        obj = os.path.join(BUILD, s.replace(".cu", ".o"))
        cmd = [cc, *ARCH, *FLAGS, "-c", os.path.join(CSRC, s), "-o", obj]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        procs.append((subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True), cmd))
        objs.append(obj)
    for p, cmd in procs:
        out, _ = p.communicate()
        if p.returncode != 0:
            raise RuntimeError(f"nvcc failed ({' '.join(cmd)}):\n{out}")
        if verbose and out:
            print(out)
    tmp = LIB + f".{os.getpid()}.tmp"
    subprocess.check_call([cc, *ARCH, "-shared", *objs, "-o", tmp])
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
