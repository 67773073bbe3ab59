"""Build libvsz.so in-tree with nvcc for sm_103a.

The translation units are compiled in parallel, then linked into one shared
library next to this file.  The CUDA runtime is linked statically (nvcc's
default), so the library shares the process's primary CUDA context with
PyTorch without depending on which libcudart PyTorch ships.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD_DIR = os.path.join(HERE, "_build")
LIB_PATH = os.path.join(HERE, "libvsz.so")

SOURCES = ["api.cu", "k_misc.cu", "k_batch.cu", "k_rank1.cu", "k_rank2.cu", "k_rank3.cu", "k_tuner.cu",
           "k_huffman.cu", "k_shard.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-std=c++17", "-O3", "-lineinfo", "-fmad=false", "-Xcompiler", "-fPIC",
              "-Xcompiler", "-fvisibility=hidden"]


def _nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libvsz")
    return cand


def _deps() -> list[str]:
    out = [os.path.join(INCLUDE, "vsz.h")]
    for f in os.listdir(CSRC):
        if f.endswith((".cu", ".cuh")):
            out.append(os.path.join(CSRC, f))
    return out


def is_stale() -> bool:
    """The library is missing or older than one of its sources."""
    if not os.path.exists(LIB_PATH):
        return True
    t = os.path.getmtime(LIB_PATH)
    return any(os.path.getmtime(d) > t for d in _deps())


def build(force: bool = False, verbose: bool = False, out: str | None = None,
          defines: tuple = (), build_dir: str | None = None) -> str:
    """Compile (if needed) and return the path of the library.  `defines`
    (e.g. ("VSZ_ND_ROWS=4",)) set the compile-time tile-shape knobs; `out`
    and `build_dir` place a variant build elsewhere."""
    lib_path = out or LIB_PATH
    bdir = build_dir or BUILD_DIR
    if not force and not defines and out is None and not is_stale():
        return LIB_PATH
    nvcc = _nvcc()
    os.makedirs(bdir, exist_ok=True)
    dflags = [f"-D{d}" for d in defines]

    def compile_one(src: str) -> str:
        """nvcc of one translation unit; the object's path."""
        obj = os.path.join(bdir, src.replace(".cu", ".o"))
        cmd = [nvcc, *ARCH, *NVCC_FLAGS, *dflags, f"-I{INCLUDE}", "-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stderr[-4000:]}")
        if verbose and r.stderr:
            print(r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = lib_path + f".tmp{os.getpid()}"
    cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc link failed:\n{r.stderr[-4000:]}")
    os.replace(tmp, lib_path)
    return lib_path


if __name__ == "__main__":
    print(build(force=True, verbose=True))
