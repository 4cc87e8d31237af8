"""Compile libheom.so in-tree for sm_103a (nvcc for the kernels, g++ for the host code).

Usage: ``python paper_2306_07522_gb300/build.py`` or ``__graft_entry__.build()`` (this file is
run by path, not imported as a submodule, because the package refuses to import before
libheom.so exists). The
translation units compile in parallel; objects go to ``_build/`` next to this file.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "libheom.so")
BUILD = os.path.join(HERE, "_build")
ARCH = "-gencode=arch=compute_103a,code=sm_103a"

CU_SOURCES = ["heom_apply.cu", "heom_solvers.cu", "heom_noalloc.cu", "heom_shifted.cu",
              "heom_persist.cu", "heom_mlp.cu", "heom_arnoldi.cu"]
CPP_SOURCES = ["heom_host.cpp"]


def _cuda_home() -> str:
    for cand in (os.environ.get("CUDA_HOME"), "/usr/local/cuda"):
        if cand and os.path.exists(os.path.join(cand, "bin", "nvcc")):
            return cand
    nvcc = shutil.which("nvcc")
    if nvcc:
        return os.path.dirname(os.path.dirname(nvcc))
    raise RuntimeError("nvcc not found: set CUDA_HOME")


def build(verbose: bool = False, ptxas_info: bool = False) -> str:
    cuda = _cuda_home()
    nvcc = os.path.join(cuda, "bin", "nvcc")
    os.makedirs(BUILD, exist_ok=True)
    jobs, objs = [], []
    for src in CU_SOURCES:
        obj = os.path.join(BUILD, src.replace(".cu", ".o"))
        cmd = [nvcc, "-c", os.path.join(CSRC, src), "-o", obj, ARCH, "-O3", "-std=c++17",
               "-lineinfo", "-Xcompiler", "-fPIC,-O2"]
        if ptxas_info:
            cmd.append("-Xptxas=-v")
        jobs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
        objs.append(obj)
    for src in CPP_SOURCES:
        obj = os.path.join(BUILD, src.replace(".cpp", ".o"))
        cmd = ["g++", "-c", os.path.join(CSRC, src), "-o", obj, "-O2", "-std=c++17", "-fPIC",
               "-I" + os.path.join(cuda, "include")]
        jobs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
        objs.append(obj)
    failed = []
    for cmd, proc in jobs:
        out, _ = proc.communicate()
        text = out.decode(errors="replace")
        if verbose or ptxas_info or proc.returncode != 0:
            sys.stdout.write(text)
        if proc.returncode != 0:
            failed.append(" ".join(cmd))
    if failed:
        raise RuntimeError("compilation failed:\n" + "\n".join(failed))
    tmp = OUT + ".tmp"
    link = [nvcc, "-shared", "-o", tmp, *objs, ARCH, "-lcudart"]
    res = subprocess.run(link, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)
    if res.returncode != 0:
        raise RuntimeError("link failed:\n" + res.stdout.decode(errors="replace"))
    os.replace(tmp, OUT)
    return OUT


if __name__ == "__main__":
    print(build(verbose=True, ptxas_info="--ptxas" in sys.argv))
