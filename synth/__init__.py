"""Seeded synthetic text: the input documents for tests, the bench and smoke.

This package produces bytes only; it holds none of the sorting method's
arithmetic, so both the CPU oracle and the CUDA path can take its output as
plain input.  The documents stand in for the paper's Hamlet text files
(Section II, 190 KB and 1.38 MB), which are not available: seeded English-like
text with a Zipf token draw, see ``textgen.c`` for the recipe.

Workloads (sizes in bytes, binary units as in the paper's "190 KB"):

* ``plain_190k``  194,560 B, V=4,000,   len 1+Poisson(3.7) in [1,20], seed 0
* ``plain_1m38``  1,447,000 B, V=12,000, len 1+Poisson(3.7) in [1,20], seed 1
* ``plain_256m``  268,435,456 B, V=500,000, len 1+Poisson(5.5) in [1,40], seed 2
* ``batch_4096``  4,096 documents, document i log-uniform in [1 KiB, 4 MiB],
  V log-uniform in [500, 100,000], len 1+Poisson(3.7) in [1,24], seed 3+i
* ``serve``       Poisson arrivals at 2,000/s for 60 s, documents log-uniform
  in [1 KiB, 16 MiB], V in [2,000, 200,000], len 1+Poisson(4.5) in [1,32], seed 4
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "_build", "libsynth.so")
_lock = threading.Lock()
_lib = None

ZIPF_S = 1.07
P_CAP = 0.12
P_PUNCT = 0.10

# Stream tags: keep workloads apart that share a seed number.
TAG_PLAIN = 1
TAG_BATCH = 3
TAG_SERVE = 5
TAG_FUZZ = 7


@dataclass(frozen=True)
class Plain:
    name: str
    nbytes: int
    vocab: int
    lam: float
    lmax: int
    seed: int


PLAIN = {
    "plain_190k": Plain("plain_190k", 194_560, 4_000, 3.7, 20, 0),
    "plain_1m38": Plain("plain_1m38", 1_447_000, 12_000, 3.7, 20, 1),
    "plain_256m": Plain("plain_256m", 268_435_456, 500_000, 5.5, 40, 2),
}

BATCH = dict(name="batch_4096", ndocs=4096, nmin=1024, nmax=4 << 20, vmin=500, vmax=100_000,
             lam=3.7, lmax=24, seed0=3)
SERVE = dict(name="serve", rate=2000.0, seconds=60.0, nmin=1024, nmax=16 << 20, vmin=2_000,
             vmax=200_000, lam=4.5, lmax=32, seed=4)


def build(force: bool = False) -> str:
    """Compile ``textgen.c`` into ``_build/libsynth.so`` (plain C, no OpenMP)."""
    with _lock:
        src = os.path.join(_HERE, "textgen.c")
        if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(src):
            return _LIB_PATH
        os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
                               src, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB_PATH)
        return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        lib.synth_text.restype = ctypes.c_int
        lib.synth_text.argtypes = [ctypes.c_uint32, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint32,
                                   ctypes.c_double, ctypes.c_uint32, ctypes.c_double, ctypes.c_double,
                                   ctypes.c_double, ctypes.c_void_p]
        lib.synth_doc_shape.restype = None
        lib.synth_doc_shape.argtypes = [ctypes.c_uint32, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64,
                                        ctypes.c_uint32, ctypes.c_uint32, ctypes.POINTER(ctypes.c_uint64),
                                        ctypes.POINTER(ctypes.c_uint32)]
        lib.synth_arrivals.restype = None
        lib.synth_arrivals.argtypes = [ctypes.c_uint32, ctypes.c_uint64, ctypes.c_double, ctypes.c_uint64,
                                       ctypes.c_void_p]
        _lib = lib
    return _lib


def text(tag: int, seed: int, nbytes: int, vocab: int, lam: float, lmax: int, out: np.ndarray | None = None,
         zipf_s: float = ZIPF_S, p_cap: float = P_CAP, p_punct: float = P_PUNCT) -> np.ndarray:
    """Return ``nbytes`` of generated text as a uint8 array (written into ``out`` if given)."""
    lib = _load()
    if out is None:
        out = np.empty(nbytes, dtype=np.uint8)
    assert out.dtype == np.uint8 and out.flags.c_contiguous and out.size >= nbytes
    rc = lib.synth_text(tag, seed, nbytes, vocab, lam, lmax, zipf_s, p_cap, p_punct,
                        out.ctypes.data if nbytes else None)
    if rc != 0:
        raise RuntimeError(f"synth_text failed with code {rc}")
    return out[:nbytes]


def plain(name: str) -> np.ndarray:
    """One of the single-document workloads, by name."""
    c = PLAIN[name]
    return text(TAG_PLAIN, c.seed, c.nbytes, c.vocab, c.lam, c.lmax)


def doc_shape(tag: int, seed: int, nmin: int, nmax: int, vmin: int, vmax: int) -> tuple[int, int]:
    lib = _load()
    n = ctypes.c_uint64()
    v = ctypes.c_uint32()
    lib.synth_doc_shape(tag, seed, nmin, nmax, vmin, vmax, ctypes.byref(n), ctypes.byref(v))
    return int(n.value), int(v.value)


def batch_shapes(ndocs: int | None = None) -> list[tuple[int, int, int]]:
    """(seed, nbytes, vocab) of the first ``ndocs`` documents of the batch workload."""
    b = BATCH
    nd = b["ndocs"] if ndocs is None else ndocs
    out = []
    for i in range(nd):
        seed = b["seed0"] + i
        n, v = doc_shape(TAG_BATCH, seed, b["nmin"], b["nmax"], b["vmin"], b["vmax"])
        out.append((seed, n, v))
    return out


def batch_doc(seed: int, nbytes: int, vocab: int, out: np.ndarray | None = None) -> np.ndarray:
    b = BATCH
    return text(TAG_BATCH, seed, nbytes, vocab, b["lam"], b["lmax"], out=out)


def batch(ndocs: int | None = None, threads: int = 8) -> list[np.ndarray]:
    """The batch workload's documents (generated on ``threads`` host threads)."""
    from concurrent.futures import ThreadPoolExecutor

    shapes = batch_shapes(ndocs)
    with ThreadPoolExecutor(max_workers=threads) as ex:
        return list(ex.map(lambda s: batch_doc(*s), shapes))


def arrivals(count: int, rate: float | None = None, seed: int | None = None) -> np.ndarray:
    """Poisson arrival times (seconds from start) of the request stream."""
    lib = _load()
    out = np.empty(count, dtype=np.float64)
    lib.synth_arrivals(TAG_SERVE, SERVE["seed"] if seed is None else seed,
                       SERVE["rate"] if rate is None else rate, count, out.ctypes.data)
    return out


def serve_doc_shape(i: int) -> tuple[int, int]:
    s = SERVE
    return doc_shape(TAG_SERVE, (s["seed"] << 32) + i, s["nmin"], s["nmax"], s["vmin"], s["vmax"])


def serve_doc(i: int) -> np.ndarray:
    s = SERVE
    n, v = serve_doc_shape(i)
    return text(TAG_SERVE, (s["seed"] << 32) + i, n, v, s["lam"], s["lmax"])
