"""ORACLE — test infrastructure, not product code.

Python access to the plain CPU oracle in ``bsort_oracle.cpp`` (the paper's
strip / bucket-by-length / bubble-sort-per-bucket method, Sections II and III
of arXiv 1407.6603).  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package; the CUDA library
never does.

Parity of every function here is pinned by ``tests/test_oracle_pins.py``
(hand-worked cases, brute force over permutations, invariants, the bubble
sort's n(n-1)/2 comparison bound) and ``tests/test_oracle_mutants.py``
(planted mistakes that the pins must catch).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
SOURCE = os.path.join(_HERE, "bsort_oracle.cpp")
_LIB_PATH = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

CXXFLAGS = ["-O2", "-std=c++17", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared"]


class _Result(ctypes.Structure):
    _fields_ = [
        ("max_len", ctypes.c_uint32),
        ("n_words", ctypes.c_uint64),
        ("stream_bytes", ctypes.c_uint64),
        ("counts", ctypes.POINTER(ctypes.c_uint64)),
        ("offsets", ctypes.POINTER(ctypes.c_uint32)),
        ("stream", ctypes.POINTER(ctypes.c_uint8)),
        ("compares", ctypes.c_uint64),
        ("swaps", ctypes.c_uint64),
    ]


def compile_library(source: str, out_path: str) -> str:
    """Compile an oracle source file into a shared library (g++, OpenMP)."""
    os.makedirs(os.path.dirname(out_path), exist_ok=True)
    tmp = out_path + f".{os.getpid()}.tmp"
    subprocess.check_call(["g++", *CXXFLAGS, source, "-o", tmp])
    os.replace(tmp, out_path)
    return out_path


def build(force: bool = False) -> str:
    with _lock:
        if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(SOURCE):
            return _LIB_PATH
        return compile_library(SOURCE, _LIB_PATH)


def bind(path: str):
    """Load an oracle library and declare its entry points."""
    lib = ctypes.CDLL(path)
    for name in ("oracle_bubble", "oracle_stable"):
        f = getattr(lib, name)
        f.restype = ctypes.c_int
        f.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int, ctypes.POINTER(_Result)]
    for name in ("oracle_bubble_order", "oracle_stable_order"):
        f = getattr(lib, name)
        f.restype = ctypes.c_int
        f.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int, ctypes.c_int, ctypes.POINTER(_Result)]
    lib.oracle_tokenize.restype = ctypes.c_int64
    lib.oracle_tokenize.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.POINTER(ctypes.c_void_p),
                                    ctypes.POINTER(ctypes.c_void_p)]
    lib.oracle_free.restype = None
    lib.oracle_free.argtypes = [ctypes.POINTER(_Result)]
    lib.oracle_free_buffer.restype = None
    lib.oracle_free_buffer.argtypes = [ctypes.c_void_p]
    lib.oracle_max_threads.restype = ctypes.c_int
    return lib


def _load():
    global _lib
    if _lib is None:
        _lib = bind(build())
    return _lib


def _as_u8(data) -> np.ndarray:
    if isinstance(data, (bytes, bytearray, memoryview)):
        return np.frombuffer(bytes(data), dtype=np.uint8)
    a = np.ascontiguousarray(data, dtype=np.uint8)
    return a.reshape(-1)


def _run(lib, fname: str, data, nthreads: int, order: int | None = None) -> dict:
    a = _as_u8(data)
    r = _Result()
    f = getattr(lib, fname)
    ptr = a.ctypes.data if a.size else None
    rc = (f(ptr, a.size, int(nthreads), ctypes.byref(r)) if order is None
          else f(ptr, a.size, int(order), int(nthreads), ctypes.byref(r)))
    try:
        if rc != 0:
            raise RuntimeError(f"{fname} failed with code {rc}")
        n = int(r.n_words)
        out = {
            "max_len": int(r.max_len),
            "n_words": n,
            "stream_bytes": int(r.stream_bytes),
            "counts": np.ctypeslib.as_array(r.counts, shape=(r.max_len + 1,)).copy(),
            "offsets": np.ctypeslib.as_array(r.offsets, shape=(n + 1,)).copy(),
            "stream": (np.ctypeslib.as_array(r.stream, shape=(int(r.stream_bytes),)).copy()
                       if r.stream_bytes else np.zeros(0, np.uint8)),
        }
        if fname == "oracle_bubble":
            out["compares"] = int(r.compares)
            out["swaps"] = int(r.swaps)
        return out
    finally:
        lib.oracle_free(ctypes.byref(r))


def bubble(data, nthreads: int = 1, lib=None) -> dict:
    """O1: bubble sort per length bucket (OpenMP over buckets with ``nthreads``)."""
    return _run(lib or _load(), "oracle_bubble", data, nthreads)


def stable(data, nthreads: int = 1, lib=None) -> dict:
    """O2: std::stable_sort by (length, bytes), grouped per length bucket."""
    return _run(lib or _load(), "oracle_stable", data, nthreads)


# Orders (the boundary's bsort_order): 0 ASCII per length bucket (the
# paper's Section III step 4), 1 folded (alphabetic, case ignored, ties in
# ASCII order) per length bucket, 2 whole-file ASCII order without length
# buckets (Table 1, row 2), 3 length buckets in input order (Table 1, row 3).
ORDER_ASCII, ORDER_FOLDED, ORDER_WHOLE, ORDER_LENGTH = 0, 1, 2, 3


def bubble_order(data, order: int, nthreads: int = 1, lib=None) -> dict:
    """O1 in any order: bubble sort with the order's comparison."""
    return _run(lib or _load(), "oracle_bubble_order", data, nthreads, order)


def stable_order(data, order: int, nthreads: int = 1, lib=None) -> dict:
    """O2 in any order: std::stable_sort with the order's comparison."""
    return _run(lib or _load(), "oracle_stable_order", data, nthreads, order)


def tokenize(data, lib=None) -> list[bytes]:
    """Phase 1 alone: the stripped words in input order."""
    lib = lib or _load()
    a = _as_u8(data)
    letters = ctypes.c_void_p()
    lengths = ctypes.c_void_p()
    n = lib.oracle_tokenize(a.ctypes.data if a.size else None, a.size, ctypes.byref(letters),
                            ctypes.byref(lengths))
    try:
        if n < 0:
            raise RuntimeError(f"oracle_tokenize failed with code {n}")
        lens = np.ctypeslib.as_array(ctypes.cast(lengths, ctypes.POINTER(ctypes.c_uint32)), shape=(max(n, 1),))[:n]
        total = int(lens.sum()) if n else 0
        buf = (bytes(np.ctypeslib.as_array(ctypes.cast(letters, ctypes.POINTER(ctypes.c_uint8)), shape=(total,)))
               if total else b"")
        out, pos = [], 0
        for L in lens.tolist():
            out.append(buf[pos:pos + L])
            pos += L
        return out
    finally:
        lib.oracle_free_buffer(letters)
        lib.oracle_free_buffer(lengths)


def words_of(result: dict) -> list[bytes]:
    """Split an oracle (or boundary) result's stream back into its words."""
    s = bytes(np.asarray(result["stream"], dtype=np.uint8))
    off = np.asarray(result["offsets"]).tolist()
    return [s[off[i]:off[i + 1]] for i in range(len(off) - 1)]


def max_threads() -> int:
    return int(_load().oracle_max_threads())
