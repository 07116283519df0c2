"""Builds libbsort.so in-tree with nvcc for sm_103a (GB300).

Each CUDA translation unit compiles in parallel to an object file, then one
link step makes the shared library.  The CUDA runtime is linked statically so
the library needs only the NVIDIA driver at run time.
"""
from __future__ import annotations

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libbsort.so")
INCLUDE = os.path.join(ROOT, "include")

SOURCES = ["k_tokenize1p.cu", "k_scatter.cu", "k_sort.cu", "k_sort2.cu", "k_tile_g2.cu", "k_tile_g4.cu",
           "k_tile_g8.cu", "k_strip_noalloc.cu", "k_dedupe.cu", "k_dedupe_hash.cu", "k_order.cu", "k_layout.cu",
           "bsort_api.cu", "bsort_serve.cu"]
HEADERS = ["bsort_dev.cuh", "tok_common.cuh", "swar.h", "sort_common.cuh", "tile_sort2.cuh", "dedupe.cuh",
           "layout_bounds.h"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr", *ARCH]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.isabs(cand) and os.path.exists(cand) or not os.path.isabs(cand)):
            return cand
    return "nvcc"


def _stale(target: str, deps: list[str]) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, extra_flags: list[str] | None = None,
          out_dir: str | None = None) -> str:
    """Compile (when stale) and link libbsort.so; returns its path.  extra_flags
    and out_dir build a variant elsewhere (tuning sweeps)."""
    out_dir = out_dir or OUT_DIR
    lib = os.path.join(out_dir, "libbsort.so")
    os.makedirs(out_dir, exist_ok=True)
    headers = [os.path.join(CSRC, h) for h in HEADERS] + [os.path.join(INCLUDE, "bsort.h"), __file__]
    flags = NVCC_FLAGS + (extra_flags or [])
    objs = []

    def compile_one(src: str) -> str:
        s = os.path.join(CSRC, src)
        o = os.path.join(out_dir, src.replace(".cu", ".o"))
        if force or _stale(o, [s] + headers):
            cmd = [nvcc(), *flags, "-I", INCLUDE, "-I", CSRC, "-c", s, "-o", o + ".tmp"]
            if verbose:
                print(" ".join(cmd), file=sys.stderr)
            subprocess.check_call(cmd)
            os.replace(o + ".tmp", o)
        return o

    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    if force or _stale(lib, objs):
        tmp = lib + f".{os.getpid()}.tmp"
        subprocess.check_call([nvcc(), *ARCH, "-shared", "-Xcompiler", "-fPIC", *objs, "-o", tmp])
        os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
