"""In-tree build of libpolyclean.so for sm_103a (nvcc, no cmake).

Each .cu of csrc/ is compiled in parallel to _build/<name>.o, then linked into
paper_2406_01342_gb300/libpolyclean.so. A translation unit is rebuilt when
it, or any header it can include, is newer than its object file.
"""
from __future__ import annotations

import concurrent.futures
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(ROOT, "_build")
LIB = os.path.join(PKG, "libpolyclean.so")

SOURCES = ["common", "plan", "grid", "grid_tc", "grid_win", "degrid_win", "fft", "sparse", "gram_tc", "select", "apgd", "solve", "serve", "dict", "degrid", "noalloc", "fft_big", "reweight_op"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CFLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", f"-I{INCLUDE}",
          "-Xcompiler", "-Wall"]


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA 13 toolkit is required to build libpolyclean.so")


def _headers_mtime() -> float:
    paths = [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE) if f.endswith(".h")]
    paths += [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".inc"))]
    return max(os.path.getmtime(p) for p in paths)


def _compile(nvcc: str, name: str, hdr_mtime: float, verbose: bool) -> str:
    src = os.path.join(CSRC, name + ".cu")
    obj = os.path.join(BUILD, name + ".o")
    if os.path.exists(obj) and os.path.getmtime(obj) >= max(os.path.getmtime(src), hdr_mtime):
        return obj
    cmd = [nvcc, *ARCH, *CFLAGS, "-c", src, "-o", obj]
    if verbose:
        print(" ".join(cmd), flush=True)
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"nvcc failed on {name}.cu:\n{res.stdout}\n{res.stderr}")
    return obj


def build(verbose: bool = False, force: bool = False) -> str:
    """Compile every CUDA source and link libpolyclean.so. Returns the library path."""
    nvcc = _nvcc()
    os.makedirs(BUILD, exist_ok=True)
    if force:
        for name in SOURCES:
            obj = os.path.join(BUILD, name + ".o")
            if os.path.exists(obj):
                os.remove(obj)
    hdr = _headers_mtime()
    with concurrent.futures.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(lambda n: _compile(nvcc, n, hdr, verbose), SOURCES))
    newest = max(os.path.getmtime(o) for o in objs)
    if not os.path.exists(LIB) or os.path.getmtime(LIB) < newest:
        cmd = [nvcc, *ARCH, "-shared", "-o", LIB + ".tmp", *objs, "-ldl"]   # -ldl: the NVTX loader
        if verbose:
            print(" ".join(cmd), flush=True)
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError(f"link failed:\n{res.stdout}\n{res.stderr}")
        os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv, force="-f" in sys.argv))
