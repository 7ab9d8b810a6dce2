"""Build libwost.so (CUDA, sm_103a) in-tree with nvcc.

Each translation unit is compiled in parallel, then linked into
paper_2410_18944_gb300/_build/libwost.so (CUDA runtime linked statically).
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libwost.so")
SOURCES = ["scene.cu", "walk.cu", "guided.cu", "wavefront.cu", "batch.cu", "train.cu", "capi.cu", "diag.cu", "noalloc.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "--expt-relaxed-constexpr", "-Xcompiler", "-fPIC"]


def _nvcc():
    p = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    return p


def _deps():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files.append(os.path.join(os.path.dirname(HERE), "include", "wost.h"))
    return files


def build(force: bool = False, verbose: bool = False, extra_flags=None) -> str:
    os.makedirs(OUT, exist_ok=True)
    newest = max(os.path.getmtime(f) for f in _deps())
    stamp = os.path.join(OUT, "flags.txt")
    want = " ".join(os.environ.get("WOST_NVCC_FLAGS", "").split())
    have = open(stamp).read() if os.path.exists(stamp) else ""
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= newest and have == want:
        return LIB
    nvcc = _nvcc()
    # WOST_NVCC_FLAGS: extra compile flags for tuning experiments (e.g.
    # "-DWOST_BVH_LEAF=8"); part of the dependency check via the stamp file
    env_flags = os.environ.get("WOST_NVCC_FLAGS", "").split()
    flags = FLAGS + list(extra_flags or []) + env_flags

    def compile_one(src):
        obj = os.path.join(OUT, src.replace(".cu", ".o"))
        cmd = [nvcc] + ARCH + flags + ["-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        if verbose and (r.stdout or r.stderr):
            sys.stderr.write(r.stdout + r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [nvcc] + ARCH + ["-shared", "-o", tmp] + objs
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    with open(stamp, "w") as fh:
        fh.write(want)
    return LIB


if __name__ == "__main__":
    force = "--force" in sys.argv
    verbose = "-v" in sys.argv
    extra = ["-Xptxas", "-v"] if "--ptxas" in sys.argv else None
    print(build(force=force, verbose=verbose or bool(extra), extra_flags=extra))
