"""Build libarx.so in-tree for sm_103a (GB300).

    python -m paper_2306_11006_gb300.build [--force]

Every translation unit is compiled in parallel (one nvcc per blind-rotation
shape family, one for the other kernels, one per host file) and linked into
paper_2306_11006_gb300/libarx.so with the CUDA runtime linked statically.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libarx.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CU = ["br_h1.cu", "br_h2.cu", "br_h3.cu", "br_h4.cu", "br_h6.cu", "br_cluster.cu", "br_cluster4.cu", "br_cluster8.cu", "br_cluster16.cu", "kernels.cu", "noalloc.cu", "probe.cu", "watchdog.cu"]
CPP = ["engine.cpp", "serve.cpp", "twiddles.cpp", "client.cpp"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _sources():
    hdrs = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    hdrs.append(os.path.join(HERE, "..", "include", "arx.h"))
    return hdrs


def _stale(obj: str, src: str, hdrs) -> bool:
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(p) > t for p in [src, *hdrs])


def _compile(args):
    cmd, src = args
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"compiling {src} failed:\n{r.stdout}\n{r.stderr}")
    return r.stderr


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(OUT_DIR, exist_ok=True)
    nv = nvcc()
    hdrs = _sources()
    jobs, objs = [], []
    common = ["-O3", "-std=c++17", "-Xcompiler", "-fPIC", "-I", CSRC]
    for f in CU:
        src, obj = os.path.join(CSRC, f), os.path.join(OUT_DIR, f + ".o")
        objs.append(obj)
        if force or _stale(obj, src, hdrs):
            jobs.append(([nv, *ARCH, "-lineinfo", *common, "-c", src, "-o", obj], src))
    for f in CPP:
        src, obj = os.path.join(CSRC, f), os.path.join(OUT_DIR, f + ".o")
        objs.append(obj)
        if force or _stale(obj, src, hdrs):
            jobs.append(([nv, *common, "-x", "c++", "-c", src, "-o", obj], src))
    with ThreadPoolExecutor(max_workers=max(1, min(len(jobs), os.cpu_count() or 1))) as ex:
        for msg in ex.map(_compile, jobs):
            if verbose and msg:
                print(msg, file=sys.stderr)
    if force or jobs or not os.path.exists(LIB):
        tmp = LIB + f".{os.getpid()}.tmp"
        cmd = [nv, *ARCH, "-shared", "-o", tmp, *objs, "-lpthread"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"linking libarx.so failed:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
