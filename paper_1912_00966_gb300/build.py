"""Build libeat.so in-tree: nvcc for the .cu sources (sm_103a only), g++ for the host
preprocessing, compiled in parallel and linked into one shared library."""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libeat.so")

CUDA_HOME = os.environ.get("CUDA_HOME", "/usr/local/cuda")
NVCC = os.path.join(CUDA_HOME, "bin", "nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]

CU_SOURCES = ["eat_kernels.cu", "eat_api.cu", "eat_server.cu", "eat_ladder.cu"]
CPP_SOURCES = ["eat_build.cpp"]
HEADERS = ["eat_internal.h", "eat_launch.h", "eat_device.cuh"]


def _sources():
    return ([os.path.join(CSRC, s) for s in CU_SOURCES + CPP_SOURCES + HEADERS]
            + [os.path.join(INCLUDE, "eat.h")])


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(s) > t for s in _sources())


def build(force: bool = False, verbose: bool = False, ptxas_verbose: bool = False) -> str:
    if not force and not _stale():
        return LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    inc = ["-I", INCLUDE, "-I", CSRC, "-I", os.path.join(CUDA_HOME, "include")]
    jobs = []
    objs = []
    for s in CU_SOURCES:
        obj = os.path.join(OUT_DIR, s + ".o")
        cmd = [NVCC, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
               "-Xcompiler", "-O2", *inc, "-c", os.path.join(CSRC, s), "-o", obj]
        if ptxas_verbose:
            cmd.insert(1, "-Xptxas=-v")
        jobs.append(cmd)
        objs.append(obj)
    for s in CPP_SOURCES:
        obj = os.path.join(OUT_DIR, s + ".o")
        cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-pthread", *inc, "-c",
               os.path.join(CSRC, s), "-o", obj]
        jobs.append(cmd)
        objs.append(obj)
    procs = []
    for cmd in jobs:
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        procs.append(subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT))
    failed = []
    for cmd, p in zip(jobs, procs):
        out, _ = p.communicate()
        text = out.decode(errors="replace")
        if p.returncode != 0:
            failed.append((cmd, text))
        elif text.strip() and (verbose or ptxas_verbose):
            print(text, file=sys.stderr)
    if failed:
        msg = "\n\n".join(" ".join(c) + "\n" + t for c, t in failed)
        raise RuntimeError("libeat build failed:\n" + msg)
    tmp = LIB + f".{os.getpid()}.tmp"
    link = [NVCC, *ARCH, "-shared", "-Xcompiler", "-pthread", "-o", tmp, *objs]
    if verbose:
        print(" ".join(link), file=sys.stderr)
    subprocess.check_call(link)
    os.replace(tmp, LIB)
    return LIB


def clean() -> None:
    shutil.rmtree(OUT_DIR, ignore_errors=True)
    if os.path.exists(LIB):
        os.remove(LIB)


if __name__ == "__main__":
    print(build(force=True, verbose=True, ptxas_verbose="-v" in sys.argv))
