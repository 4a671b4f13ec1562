"""Builds the in-tree shared library libqtensor.so for sm_103a with nvcc.

Every translation unit is compiled in parallel, then linked into
paper_2012_02430_gb300/_lib/libqtensor.so (git-ignored). Host code is plain
C++17 (no intrinsics, no -march), so the same sources build on x86-64 and Arm.
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
LIB = os.path.join(LIBDIR, "libqtensor.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")

SOURCES = ["api.cpp", "host_graph.cpp", "host_schedule.cpp", "engine.cu", "noalloc.cu",
           "energy_host.cpp", "energy.cu", "learn.cpp", "mlp.cu", "gemm.cu", "umma.cu"]
GENCODE = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc_path() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found")
    return cand


def _compile(src: str, obj: str, nvcc: str) -> tuple[str, int, str]:
    cmd = [nvcc, *GENCODE, "-lineinfo", "-O3", "-std=c++17", "-I", INCLUDE,
           "-Xcompiler", "-fPIC,-O3,-Wall", "-c", os.path.join(CSRC, src), "-o", obj]
    if src.endswith(".cu"):
        cmd[1:1] = ["-Xptxas", "-v"] if os.environ.get("QT_PTXAS_VERBOSE") else []
    r = subprocess.run(cmd, capture_output=True, text=True)
    return src, r.returncode, r.stdout + r.stderr


def build(force: bool = False, verbose: bool = False) -> str:
    """Compiles and links the library; returns its path. Rebuilds when a source is newer."""
    os.makedirs(LIBDIR, exist_ok=True)
    deps = [os.path.join(CSRC, s) for s in SOURCES]
    deps += [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".h")]
    deps.append(os.path.join(INCLUDE, "qtensor.h"))
    if not force and os.path.exists(LIB):
        t = os.path.getmtime(LIB)
        if all(os.path.getmtime(d) <= t for d in deps):
            return LIB
    nvcc = nvcc_path()
    objdir = os.path.join(LIBDIR, "obj")
    os.makedirs(objdir, exist_ok=True)
    jobs = []
    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        for s in SOURCES:
            obj = os.path.join(objdir, os.path.splitext(s)[0] + ".o")
            jobs.append(ex.submit(_compile, s, obj, nvcc))
    objs = []
    for j in jobs:
        src, rc, out = j.result()
        if verbose and out.strip():
            print(out, file=sys.stderr)
        if rc != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{out}")
        objs.append(os.path.join(objdir, os.path.splitext(src)[0] + ".o"))
    tmp = LIB + ".tmp"
    cmd = [nvcc, *GENCODE, "-shared", "-o", tmp, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n" + r.stdout + r.stderr)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
