"""Python binding of libbsort, the GB300 length-bucketed word sort.

The method (arXiv 1407.6603, Section II, three pre-processing phases): strip
every non-letter from a text, bucket its words by length with shorter buckets
first, and sort each bucket into ASCII order.  All of it runs in the CUDA
kernels of ``libbsort.so``; this module only marshals arguments through the C
ABI of ``include/bsort.h`` and has the same entry point names.  There is no
CPU fallback: ``load()`` raises when the library has not been built.

PyTorch is used here only for device memory and streams (``text_device``
takes a CUDA tensor and the current torch stream).
"""
from __future__ import annotations

import ctypes
import threading
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libbsort.so")

BSORT_OK = 0
BSORT_E_INVAL = 1
BSORT_E_NOMEM = 2
BSORT_E_CUDA = 3
BSORT_E_TOO_LARGE = 4
BSORT_E_WORD_TOO_LONG = 5
BSORT_E_TIMEOUT = 6
BSORT_E_BUSY = 7
STATUS_NAMES = {0: "OK", 1: "E_INVAL", 2: "E_NOMEM", 3: "E_CUDA", 4: "E_TOO_LARGE", 5: "E_WORD_TOO_LONG",
                6: "E_TIMEOUT", 7: "E_BUSY"}


class bsort_config(ctypes.Structure):
    _fields_ = [("l_cap", ctypes.c_uint32), ("want_offsets", ctypes.c_int32), ("device", ctypes.c_int32),
                ("profile", ctypes.c_int32), ("wait_limit", ctypes.c_uint64), ("tune_table", ctypes.c_char_p),
                ("order", ctypes.c_uint32), ("key_pack", ctypes.c_uint32)]


# bsort_order and bsort_key_pack
ORDER_ASCII, ORDER_FOLDED, ORDER_WHOLE, ORDER_LENGTH = 0, 1, 2, 3
KEYS_BYTES, KEYS_LETTERS6 = 0, 1


class bsort_kernel_stat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char_p), ("launches", ctypes.c_uint64), ("ms", ctypes.c_double),
                ("bytes", ctypes.c_double), ("key_levels", ctypes.c_double)]


class bsort_trace_rec(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char_p), ("start_ms", ctypes.c_double), ("end_ms", ctypes.c_double),
                ("bytes", ctypes.c_double), ("stream", ctypes.c_uint32), ("variant", ctypes.c_uint32),
                ("kernels", ctypes.c_uint32), ("reserved", ctypes.c_uint32)]


class bsort_result(ctypes.Structure):
    _fields_ = [("max_len", ctypes.c_uint32), ("status", ctypes.c_uint32), ("n_words", ctypes.c_uint64),
                ("stream_bytes", ctypes.c_uint64), ("counts", ctypes.c_void_p), ("offsets", ctypes.c_void_p),
                ("stream", ctypes.c_void_p)]


class bsort_serve_config(ctypes.Structure):
    _fields_ = [("hbm_budget", ctypes.c_uint64), ("workers", ctypes.c_uint32), ("max_batch_docs", ctypes.c_uint32)]


class BsortError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"bsort {STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


_lib = None


def build(force: bool = False) -> str:
    from . import builder as _b

    return _b.build(force=force)


def load(path: str | None = None):
    """Load libbsort.so.  Raises if it is missing: there is no fallback path."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"libbsort.so not found at {p}: run build() (nvcc, sm_103a) first")
    lib = ctypes.CDLL(p)
    ctx_p = ctypes.c_void_p
    lib.bsort_config_default.restype = None
    lib.bsort_config_default.argtypes = [ctypes.POINTER(bsort_config)]
    lib.bsort_create.restype = ctypes.c_int
    lib.bsort_create.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(bsort_config)]
    lib.bsort_destroy.restype = None
    lib.bsort_destroy.argtypes = [ctx_p]
    lib.bsort_last_error.restype = ctypes.c_char_p
    lib.bsort_last_error.argtypes = [ctx_p]
    lib.bsort_text.restype = ctypes.c_int
    lib.bsort_text.argtypes = [ctx_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.POINTER(bsort_result)]
    lib.bsort_text_device.restype = ctypes.c_int
    lib.bsort_text_device.argtypes = [ctx_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p,
                                      ctypes.POINTER(bsort_result)]
    lib.bsort_batch.restype = ctypes.c_int
    lib.bsort_batch.argtypes = [ctx_p, ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_size_t),
                                ctypes.c_size_t, ctypes.POINTER(bsort_result)]
    lib.bsort_batch_device.restype = ctypes.c_int
    lib.bsort_batch_device.argtypes = [ctx_p, ctypes.c_void_p, ctypes.POINTER(ctypes.c_uint64),
                                       ctypes.POINTER(ctypes.c_uint64), ctypes.c_size_t, ctypes.c_void_p,
                                       ctypes.POINTER(bsort_result)]
    lib.bsort_result_release.restype = None
    lib.bsort_result_release.argtypes = [ctx_p, ctypes.POINTER(bsort_result)]
    lib.bsort_profile_read.restype = ctypes.c_int
    lib.bsort_profile_read.argtypes = [ctx_p, ctypes.POINTER(bsort_kernel_stat), ctypes.c_int]
    lib.bsort_trace_read.restype = ctypes.c_int
    lib.bsort_trace_read.argtypes = [ctx_p, ctypes.POINTER(bsort_trace_rec), ctypes.c_int]
    lib.bsort_launch_count.restype = ctypes.c_uint64
    lib.bsort_launch_count.argtypes = [ctx_p]
    lib.bsort_context_config.restype = ctypes.c_int
    lib.bsort_context_config.argtypes = [ctx_p, ctypes.POINTER(bsort_config)]
    lib.bsort_serve_config_default.restype = None
    lib.bsort_serve_config_default.argtypes = [ctypes.POINTER(bsort_serve_config)]
    lib.bsort_serve_start.restype = ctypes.c_int
    lib.bsort_serve_start.argtypes = [ctx_p, ctypes.POINTER(bsort_serve_config)]
    lib.bsort_submit.restype = ctypes.c_int
    lib.bsort_submit.argtypes = [ctx_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_uint64]
    lib.bsort_submit_borrowed.restype = ctypes.c_int
    lib.bsort_submit_borrowed.argtypes = [ctx_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_uint64]
    lib.bsort_poll.restype = ctypes.c_size_t
    lib.bsort_poll.argtypes = [ctx_p, ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(bsort_result),
                               ctypes.POINTER(ctypes.c_uint64), ctypes.c_size_t]
    lib.bsort_serve_pending.restype = ctypes.c_size_t
    lib.bsort_serve_pending.argtypes = [ctx_p]
    lib.bsort_serve_stop.restype = ctypes.c_int
    lib.bsort_serve_stop.argtypes = [ctx_p]
    lib.bsort_device_finish.restype = ctypes.c_int
    lib.bsort_device_finish.argtypes = [ctx_p, ctypes.c_void_p]
    lib.bsort_strip_noalloc.restype = ctypes.c_int
    lib.bsort_strip_noalloc.argtypes = [ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_void_p, ctypes.c_void_p]
    if path is None:
        _lib = lib
    return lib


# ---- thin wrappers with the C names ----

def bsort_config_default() -> bsort_config:
    cfg = bsort_config()
    load().bsort_config_default(ctypes.byref(cfg))
    return cfg


def bsort_create(cfg: bsort_config | None = None) -> ctypes.c_void_p:
    lib = load()
    h = ctypes.c_void_p()
    st = lib.bsort_create(ctypes.byref(h), ctypes.byref(cfg) if cfg is not None else None)
    if st != BSORT_OK:
        raise BsortError(st, "bsort_create failed")
    return h


def bsort_destroy(h) -> None:
    load().bsort_destroy(h)


def bsort_last_error(h) -> str:
    return load().bsort_last_error(h).decode(errors="replace")


def _as_u8(data) -> np.ndarray:
    if isinstance(data, (bytes, bytearray, memoryview)):
        return np.frombuffer(bytes(data), dtype=np.uint8)
    return np.ascontiguousarray(data, dtype=np.uint8).reshape(-1)


def bsort_text(h, data) -> bsort_result:
    a = _as_u8(data)
    res = bsort_result()
    st = load().bsort_text(h, a.ctypes.data if a.size else None, a.size, ctypes.byref(res))
    if st != BSORT_OK:
        raise BsortError(st, bsort_last_error(h))
    return res


def bsort_text_device(h, ptr: int, nbytes: int, stream: int) -> bsort_result:
    res = bsort_result()
    st = load().bsort_text_device(h, ptr if nbytes else None, nbytes, stream or None, ctypes.byref(res))
    if st != BSORT_OK:
        raise BsortError(st, bsort_last_error(h))
    return res


def bsort_batch(h, docs: list) -> tuple[int, list[bsort_result]]:
    arrs = [_as_u8(d) for d in docs]
    n = len(arrs)
    ptrs = (ctypes.c_void_p * max(n, 1))(*[a.ctypes.data if a.size else None for a in arrs])
    lens = (ctypes.c_size_t * max(n, 1))(*[a.size for a in arrs])
    outs = (bsort_result * max(n, 1))()
    st = load().bsort_batch(h, ptrs, lens, n, outs)
    return st, [outs[i] for i in range(n)]


def bsort_batch_device(h, base_ptr: int, offs, lens, stream: int) -> tuple[int, list[bsort_result]]:
    n = len(offs)
    o = (ctypes.c_uint64 * max(n, 1))(*[int(x) for x in offs])
    ln = (ctypes.c_uint64 * max(n, 1))(*[int(x) for x in lens])
    outs = (bsort_result * max(n, 1))()
    st = load().bsort_batch_device(h, base_ptr or None, o, ln, n, stream or None, outs)
    return st, [outs[i] for i in range(n)]


def bsort_device_finish(h, stream: int) -> int:
    """Waits for the last device call's work on ``stream``; its bsort_status
    (BSORT_E_TIMEOUT when a bounded wait of the sort kernels ran out)."""
    return int(load().bsort_device_finish(h, stream or None))


def bsort_result_release(h, res: bsort_result) -> None:
    load().bsort_result_release(h, ctypes.byref(res))


def bsort_profile_read(h) -> dict:
    """Per kernel family: {name: (launches, ms, algorithmic bytes, key-levels)} since the last read."""
    arr = (bsort_kernel_stat * 16)()
    k = load().bsort_profile_read(h, arr, 16)
    if k < 0:
        raise BsortError(BSORT_E_CUDA, "bsort_profile_read failed")
    return {arr[i].name.decode(): (int(arr[i].launches), float(arr[i].ms), float(arr[i].bytes),
                                   float(arr[i].key_levels)) for i in range(k)}


def bsort_trace_read(h) -> list[tuple[str, float, float, float, int]]:
    """Traced launches since the last profile read, in launch order:
    (family, start ms, end ms, algorithmic bytes, stream, variant)."""
    lib = load()
    n = lib.bsort_trace_read(h, None, 0)
    if n < 0:
        raise BsortError(BSORT_E_CUDA, "bsort_trace_read failed")
    arr = (bsort_trace_rec * max(n, 1))()
    n = lib.bsort_trace_read(h, arr, n)
    if n < 0:
        raise BsortError(BSORT_E_CUDA, "bsort_trace_read failed")
    return [(arr[i].name.decode(), arr[i].start_ms, arr[i].end_ms, arr[i].bytes, int(arr[i].stream),
             int(arr[i].variant), int(arr[i].kernels)) for i in range(n)]


def bsort_launch_count(h) -> int:
    return int(load().bsort_launch_count(h))


def bsort_serve_start(h, hbm_budget: int = 0, workers: int = 0, max_batch_docs: int = 0) -> None:
    cfg = bsort_serve_config()
    load().bsort_serve_config_default(ctypes.byref(cfg))
    if hbm_budget:
        cfg.hbm_budget = hbm_budget
    if workers:
        cfg.workers = workers
    if max_batch_docs:
        cfg.max_batch_docs = max_batch_docs
    st = load().bsort_serve_start(h, ctypes.byref(cfg))
    if st != BSORT_OK:
        raise BsortError(st, "bsort_serve_start failed")


def bsort_submit(h, data, tag: int) -> int:
    a = _as_u8(data)
    return int(load().bsort_submit(h, a.ctypes.data if a.size else None, a.size, tag))


def bsort_submit_borrowed(h, data, tag: int) -> int:
    """data (a uint8 array) must stay alive and unchanged until the request's
    result is polled (Context.submit(borrow=True) keeps the reference)."""
    a = _as_u8(data)
    return int(load().bsort_submit_borrowed(h, a.ctypes.data if a.size else None, a.size, tag))


def bsort_poll(h, max_results: int = 256, want_offsets: bool = True, copy: bool = True) -> list:
    """Finished requests: [(tag, result, latency_ns)].  copy=True: the results
    are copied out and released at once.  copy=False: each result is a
    ViewResult over the server's page-locked buffers, valid until it is passed
    to bsort_result_release (Context.release), which must follow."""
    tags = (ctypes.c_uint64 * max_results)()
    outs = (bsort_result * max_results)()
    lat = (ctypes.c_uint64 * max_results)()
    lib = load()
    k = int(lib.bsort_poll(h, tags, outs, lat, max_results))
    got = []
    for i in range(k):
        r = bsort_result.from_buffer_copy(outs[i])
        if copy:
            res = _host_result(r, want_offsets)
            lib.bsort_result_release(h, ctypes.byref(r))
        else:
            res = ViewResult(r, want_offsets)
        got.append((int(tags[i]), res, int(lat[i])))
    return got


def bsort_serve_pending(h) -> int:
    return int(load().bsort_serve_pending(h))


def bsort_serve_stop(h) -> None:
    st = load().bsort_serve_stop(h)
    if st != BSORT_OK:
        raise BsortError(st, "bsort_serve_stop failed")


NOALLOC_MAX_BYTES = (64 << 20) - 16


def bsort_strip_noalloc(ptr: int, nbytes: int, stream: int, letters_ptr: int, starts_ptr: int,
                        totals_ptr: int) -> int:
    """Strip + tokenize one device document into caller-provided device
    buffers without allocating; returns the bsort_status of the call."""
    return int(load().bsort_strip_noalloc(ptr or None, nbytes, stream or None, letters_ptr or None,
                                          starts_ptr or None, totals_ptr or None))


# ---- convenience layer ----

@dataclass
class Result:
    max_len: int
    n_words: int
    stream_bytes: int
    counts: np.ndarray
    offsets: np.ndarray | None
    stream: np.ndarray
    status: int = 0

    def words(self) -> list[bytes]:
        s = self.stream.tobytes()
        off = self.offsets.tolist()
        return [s[off[i]:off[i + 1]] for i in range(len(off) - 1)]


def _host_array(ptr, ctype, count, dtype, copy: bool) -> np.ndarray:
    if count == 0 or not ptr:  # empty, or a failed document (zeroed result)
        return np.zeros(0, dtype=dtype)
    v = np.ctypeslib.as_array(ctypes.cast(ptr, ctypes.POINTER(ctype)), shape=(count,))
    return v.copy() if copy else v


class ViewResult:
    """A host result whose arrays are views of page-locked buffers, made on
    first access: the context's (valid until the next call on the context) or,
    from poll(copy=False), the server's (valid until Context.release).  Same
    fields as Result."""

    __slots__ = ("_r", "_want_offsets", "max_len", "n_words", "stream_bytes", "status", "_cache")

    def __init__(self, r: bsort_result, want_offsets: bool):
        self._r = r
        self._want_offsets = want_offsets
        self.max_len = int(r.max_len)
        self.n_words = int(r.n_words)
        self.stream_bytes = int(r.stream_bytes)
        self.status = int(r.status)
        self._cache = {}

    @property
    def counts(self) -> np.ndarray:
        if "c" not in self._cache:
            self._cache["c"] = _host_array(self._r.counts, ctypes.c_uint64, self.max_len + 1, np.uint64, False)
        return self._cache["c"]

    @property
    def offsets(self) -> np.ndarray | None:
        if not self._want_offsets:
            return None
        if "o" not in self._cache:
            self._cache["o"] = _host_array(self._r.offsets, ctypes.c_uint32, self.n_words + 1, np.uint32, False)
        return self._cache["o"]

    @property
    def stream(self) -> np.ndarray:
        if "s" not in self._cache:
            self._cache["s"] = _host_array(self._r.stream, ctypes.c_uint8, self.stream_bytes, np.uint8, False)
        return self._cache["s"]

    words = Result.words


def _host_result(r: bsort_result, want_offsets: bool, copy: bool = True):
    """copy=False gives a ViewResult over the context's page-locked result
    buffers, valid until the next call on the context."""
    if not copy:
        return ViewResult(r, want_offsets)
    n = int(r.n_words)
    ml = int(r.max_len)
    return Result(
        max_len=ml, n_words=n, stream_bytes=int(r.stream_bytes),
        counts=_host_array(r.counts, ctypes.c_uint64, ml + 1, np.uint64, True),
        offsets=_host_array(r.offsets, ctypes.c_uint32, n + 1, np.uint32, True) if want_offsets else None,
        stream=_host_array(r.stream, ctypes.c_uint8, int(r.stream_bytes), np.uint8, True),
        status=int(r.status),
    )


class _DevView:
    """A device buffer owned by the context, seen through __cuda_array_interface__."""

    def __init__(self, ptr: int, count: int, typestr: str):
        self.__cuda_array_interface__ = {"shape": (count,), "typestr": typestr, "data": (ptr or 0, False),
                                         "version": 3, "strides": None, "stream": None}


def pinned_empty(nbytes: int) -> np.ndarray:
    """A page-locked host uint8 array (torch's pinned allocator), which
    bsort_text / bsort_batch read in place."""
    import torch

    return torch.empty(max(nbytes, 1), dtype=torch.uint8, pin_memory=True).numpy()[:nbytes]


def pack_host(docs: list, pinned: bool = True) -> list[np.ndarray]:
    """Copies documents back to back into one (page-locked) host buffer and
    returns views of it, the layout bsort_batch moves in one copy."""
    lens = [len(d) for d in docs]
    buf = pinned_empty(sum(lens)) if pinned else np.empty(sum(lens), np.uint8)
    out, pos = [], 0
    for d, n in zip(docs, lens):
        buf[pos:pos + n] = _as_u8(d)
        out.append(buf[pos:pos + n])
        pos += n
    return out


class Context:
    """Owns a bsort context (CUDA stream, device arena, pinned host buffers)."""

    def __init__(self, l_cap: int = 255, want_offsets: bool = True, device: int = -1, wait_limit: int = 0,
                 profile: bool = False, tune_table: str | None = None, order: int = ORDER_ASCII,
                 key_pack: int = KEYS_BYTES):
        """tune_table: None for the built-in tuning, else the text of a tune
        table (see bsort_config.tune_table; autotune.py writes one).  order:
        the result's order (ORDER_*); key_pack: the sort keys' encoding
        (KEYS_*, the same result)."""
        cfg = bsort_config_default()
        cfg.order = order
        cfg.key_pack = key_pack
        cfg.l_cap = l_cap
        cfg.want_offsets = 1 if want_offsets else 0
        cfg.device = device
        cfg.profile = 1 if profile else 0
        cfg.wait_limit = wait_limit
        self._tune = tune_table.encode() if tune_table is not None else None
        cfg.tune_table = self._tune
        self.want_offsets = want_offsets
        self._borrowed = {}  # tag -> array of a borrowed request not yet polled
        self._borrow_lock = threading.Lock()
        self._h = bsort_create(cfg)

    def close(self) -> None:
        if getattr(self, "_h", None):
            bsort_destroy(self._h)
            self._h = None
        self._borrowed = {}

    def __del__(self):
        self.close()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def handle(self):
        return self._h

    def text(self, data, copy: bool = True) -> Result:
        """Host bytes in, host result out (synchronous).  copy=False returns
        views of the context's result buffers, valid until its next call."""
        return _host_result(bsort_text(self._h, data), self.want_offsets, copy)

    def text_device_raw(self, tensor, stream=None) -> bsort_result:
        """Device tensor in (uint8, contiguous); device pointers out, valid once
        ``stream`` (default: torch's current stream) reaches this point."""
        import torch

        assert tensor.is_cuda and tensor.dtype == torch.uint8 and tensor.is_contiguous()
        s = stream if stream is not None else torch.cuda.current_stream(tensor.device)
        return bsort_text_device(self._h, tensor.data_ptr(), tensor.numel(), s.cuda_stream)

    def text_device(self, tensor, stream=None, clone: bool = True) -> dict:
        """As text_device_raw, returning torch tensors (copies unless clone=False)."""
        import torch

        r = self.text_device_raw(tensor, stream)
        n, ml = int(r.n_words), int(r.max_len)
        dev = tensor.device

        def view(ptr, count, typestr, dtype):
            if count == 0:
                return torch.zeros(0, dtype=dtype, device=dev)
            t = torch.as_tensor(_DevView(ptr, count, typestr), device=dev)
            return t.clone() if clone else t

        with torch.cuda.stream(stream if stream is not None else torch.cuda.current_stream(dev)):
            out = {
                "max_len": ml, "n_words": n, "stream_bytes": int(r.stream_bytes),
                # signed views: torch handles int64/int32 everywhere (values < 2^31 here)
                "counts": view(r.counts, ml + 1, "<i8", torch.int64),
                "offsets": view(r.offsets, n + 1, "<i4", torch.int32) if self.want_offsets else None,
                "stream": view(r.stream, int(r.stream_bytes), "|u1", torch.uint8),
            }
        return out

    def batch_device_raw(self, base, offs, lens, stream=None) -> tuple[int, list[bsort_result]]:
        """Documents packed in one CUDA uint8 tensor at host-listed offsets;
        device pointers out (valid once ``stream`` reaches this point)."""
        import torch

        assert base.is_cuda and base.dtype == torch.uint8 and base.is_contiguous()
        s = stream if stream is not None else torch.cuda.current_stream(base.device)
        return bsort_batch_device(self._h, base.data_ptr() if base.numel() else 0, offs, lens, s.cuda_stream)

    def batch_device(self, base, offs, lens, stream=None) -> tuple[int, list[dict]]:
        """As batch_device_raw, with each document's outputs copied to torch tensors."""
        import torch

        st, rs = self.batch_device_raw(base, offs, lens, stream)
        dev = base.device

        def view(ptr, count, typestr, dtype):
            if count == 0 or not ptr:
                return torch.zeros(0, dtype=dtype, device=dev)
            return torch.as_tensor(_DevView(ptr, count, typestr), device=dev).clone()

        out = []
        with torch.cuda.stream(stream if stream is not None else torch.cuda.current_stream(dev)):
            for r in rs:
                n, ml = int(r.n_words), int(r.max_len)
                out.append({"status": int(r.status), "max_len": ml, "n_words": n, "stream_bytes": int(r.stream_bytes),
                            "counts": view(r.counts, ml + 1, "<i8", torch.int64),
                            "offsets": view(r.offsets, n + 1, "<i4", torch.int32) if self.want_offsets else None,
                            "stream": view(r.stream, int(r.stream_bytes), "|u1", torch.uint8)})
        return st, out

    def batch(self, docs: list, copy: bool = True) -> tuple[int, list[Result]]:
        """Many host documents in one pass.  Views of one buffer, back to back
        (as pack_host() makes them), move as one copy; copy=False as in text()."""
        st, rs = bsort_batch(self._h, docs)
        return st, [_host_result(r, self.want_offsets, copy) for r in rs]

    def last_error(self) -> str:
        return bsort_last_error(self._h)

    def device_finish(self, stream=None) -> int:
        """Status of the last device call's work (waits for ``stream``, default
        torch's current stream)."""
        import torch

        s = stream if stream is not None else torch.cuda.current_stream()
        return bsort_device_finish(self._h, s.cuda_stream)

    def serve_start(self, hbm_budget: int = 0, workers: int = 0, max_batch_docs: int = 0) -> None:
        bsort_serve_start(self._h, hbm_budget, workers, max_batch_docs)

    def submit(self, data, tag: int, borrow: bool = False) -> int:
        """Queues a document.  borrow=True: no copy; the array (page-locked
        ones are read in place by the copy engine) is kept referenced here
        until its tag's result is polled."""
        if not borrow:
            return bsort_submit(self._h, data, tag)
        a = _as_u8(data)
        with self._borrow_lock:
            self._borrowed[tag] = a
        st = bsort_submit_borrowed(self._h, a, tag)
        if st != BSORT_OK:
            with self._borrow_lock:
                self._borrowed.pop(tag, None)
        return st

    def poll(self, max_results: int = 256, copy: bool = True) -> list:
        got = bsort_poll(self._h, max_results, self.want_offsets, copy)
        if self._borrowed:
            with self._borrow_lock:
                for tag, _, _ in got:
                    self._borrowed.pop(tag, None)
        return got

    def release(self, res) -> None:
        """Ends a served result's hold on the server's buffers (a ViewResult
        from poll(copy=False)); its arrays must not be used afterwards."""
        bsort_result_release(self._h, res._r)

    def serve_pending(self) -> int:
        return bsort_serve_pending(self._h)

    def serve_stop(self) -> None:
        bsort_serve_stop(self._h)

    def profile_read(self) -> dict:
        return bsort_profile_read(self._h)

    def trace_read(self) -> list:
        return bsort_trace_read(self._h)

    def launch_count(self) -> int:
        return bsort_launch_count(self._h)
