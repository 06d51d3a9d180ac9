"""Builds libcrkfr.so in-tree for sm_103a with nvcc.

    python -m paper_2512_08611_gb300.build

Each translation unit is compiled by its own nvcc process (in parallel), then
linked into ``paper_2512_08611_gb300/lib/libcrkfr.so`` with the CUDA runtime
linked statically.  Rebuilds only when a source or header is newer than the
library.
"""
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIBDIR = os.path.join(HERE, "lib")
LIBNAME = "libcrkfr.so"

SOURCES = ["api.cu", "kernels_1d.cu", "kernels_2d.cu", "kernels_imex.cu", "kernels_imex1d.cu",
           "kernels_wb.cu", "kernels_wb1d.cu",
           "kernels_limit.cu", "kernels_limit2d.cu", "kernels_limit2d_wb.cu", "noalloc.cu", "batch.cu",
           "kernels_adj2d.cu", "probe.cu", "basis.cpp"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC,-O2", "-I", INCLUDE, "-I", CSRC]


def nvcc():
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.isabs(cand) and os.path.exists(cand) or not os.path.isabs(cand)):
            return cand
    return "nvcc"


def library_path():
    return os.path.join(LIBDIR, LIBNAME)


def _inputs():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files.append(os.path.join(INCLUDE, "crkfr.h"))
    return files


def up_to_date():
    lib = library_path()
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(f) <= t for f in _inputs())


def _compile(src, verbose):
    obj = os.path.join(BUILD, os.path.splitext(src)[0] + ".o")
    cmd = [nvcc()] + ARCH + FLAGS + ["-c", os.path.join(CSRC, src), "-o", obj]
    if src.endswith(".cpp"):
        cmd[1:1] = ["-x", "c++"]
    if verbose:
        print(" ".join(cmd), flush=True)
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
    return obj


def build_library(force=False, verbose=False):
    """Compile and link libcrkfr.so; returns its path."""
    if not force and up_to_date():
        return library_path()
    os.makedirs(BUILD, exist_ok=True)
    os.makedirs(LIBDIR, exist_ok=True)
    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(lambda s: _compile(s, verbose), SOURCES))
    tmp = library_path() + ".tmp"
    cmd = [nvcc()] + ARCH + ["-shared", "-cudart", "static", "-o", tmp] + objs
    if verbose:
        print(" ".join(cmd), flush=True)
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, library_path())
    return library_path()


if __name__ == "__main__":
    print(build_library(force="--force" in sys.argv, verbose=True))
