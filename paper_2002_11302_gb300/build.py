"""Build libpbspgemm.so in-tree with nvcc for sm_103a (GB300).

Each translation unit is compiled in parallel, then linked into
``paper_2002_11302_gb300/libpbspgemm.so``.  Object files go to
``paper_2002_11302_gb300/_build/``.  No cmake; only nvcc.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
SRC_DIR = os.path.join(PKG, "csrc")
INC_DIR = os.path.join(ROOT, "include")
OBJ_DIR = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libpbspgemm.so")
SOURCES = ["pb_scan.cu", "pb_symbolic.cu", "pb_expand.cu", "pb_oversize.cu", "pb_binsort.cu", "pb_api.cu", "pb_batch.cu", "pb_serve.cu", "pb_determ.cu", "pb_noalloc.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I" + INC_DIR]


def nvcc() -> str:
    exe = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(exe):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libpbspgemm")
    return exe


def _deps_mtime() -> float:
    files = [os.path.join(SRC_DIR, f) for f in os.listdir(SRC_DIR)]
    files.append(os.path.join(INC_DIR, "pb_spgemm.h"))
    return max(os.path.getmtime(f) for f in files)


def _compile(src: str, obj_dir: str = OBJ_DIR, extra=()) -> str:
    obj = os.path.join(obj_dir, os.path.splitext(src)[0] + ".o")
    cmd = [nvcc(), *ARCH, *FLAGS, *extra, "-c", os.path.join(SRC_DIR, src), "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed on {src}:\n{r.stderr}")
    return obj


def build(force: bool = False, lib: str = LIB, obj_dir: str = OBJ_DIR, defines=()) -> str:
    """Compile and link the library if any source is newer than it; return its path.

    ``defines`` (e.g. ("PB_EXPAND_UNROLL=4",)) override tuning macros; use a
    separate ``lib``/``obj_dir`` for such variants.
    """
    if not force and os.path.exists(lib) and os.path.getmtime(lib) >= _deps_mtime():
        return lib
    os.makedirs(obj_dir, exist_ok=True)
    extra = ["-D" + d for d in defines]
    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(lambda s: _compile(s, obj_dir, extra), SOURCES))
    tmp = lib + f".tmp{os.getpid()}"
    r = subprocess.run([nvcc(), *ARCH, "-shared", "-o", tmp, *objs], capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force=True))
