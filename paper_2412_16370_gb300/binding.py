"""Thin ctypes binding of ``libpospopcnt.so`` (C ABI: ``include/pospopcnt.h``).

Argument marshalling only: every function forwards to the entry point of the
same name, passing raw pointers (``tensor.data_ptr()`` for torch tensors,
``array.ctypes.data`` for numpy arrays), sizes and the CUDA stream handle, and
raises ``PospopError`` on a nonzero status.  There is no CPU fallback: if the
library is missing, every call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libpospopcnt.so")

POSPOP_OK = 0
POSPOP_EINVAL = -1
POSPOP_EPTR = -2
POSPOP_ECUDA = -3
POSPOP_ENOMEM = -4
POSPOP_ETIMEDOUT = -5
POSPOP_EBUSY = -6
POSPOP_ERANGE = -7

_lock = threading.Lock()
_lib = None


class PospopError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"pospopcnt error {code}: {msg}")
        self.code = code


_u64p = ctypes.POINTER(ctypes.c_uint64)
_vp = ctypes.c_void_p
_sz = ctypes.c_size_t
_int = ctypes.c_int

_SIGNATURES = {
    "pospopcnt_strerror": ([_int], ctypes.c_char_p),
    "pospopcnt_init": ([_int], _int),
    "pospopcnt_shutdown": ([], None),
    "pospopcnt_u8": ([_vp, _vp, _sz], _int),
    "pospopcnt_u16": ([_vp, _vp, _sz], _int),
    "pospopcnt_u32": ([_vp, _vp, _sz], _int),
    "pospopcnt_u64": ([_vp, _vp, _sz], _int),
    "pospopcnt_async": ([_int, _vp, _vp, _sz, _vp], _int),
    "pospopcnt_batch": ([_int, _vp, _vp, _vp, _sz, _vp], _int),
    "pospopcnt_batch_noalloc": ([_int, _vp, _vp, _vp, _sz, _vp], _int),
    "pospopcnt_gather": ([_int, _vp, _vp, _vp, _sz, _vp], _int),
    "pospopcnt_multi": ([_sz, _vp, _vp, _vp, _vp, _vp], _int),
    "pospopcnt_masked": ([_int, _vp, _vp, _sz, _vp, _vp], _int),
    "pospopcnt_batch_status": ([_vp], _int),
    "pospopcnt_reserve": ([_sz, _vp], _int),
    "pospopcnt_host": ([_int, _vp, _vp, _sz], _int),
    "pospopcnt_roofline_read": ([_vp, _sz, _vp, _vp], _int),
    "pospopcnt_plan": ([_int, _sz, ctypes.POINTER(ctypes.c_uint32)], _int),
    "pospopcnt_autotune": ([_sz, ctypes.c_char_p], _int),
    "pospopcnt_tune_load": ([ctypes.c_char_p], _int),
    "pospopcnt_tune_describe": ([ctypes.c_char_p, _sz], _int),
    "pospopcnt_tune_check": ([ctypes.c_char_p, ctypes.POINTER(_int)], _int),
    "pospopcnt_batch_graph_create": ([_int, _vp, _vp, _vp, _sz, _vp, ctypes.POINTER(_vp)], _int),
    "pospopcnt_graph_launch": ([_vp, _vp], _int),
    "pospopcnt_graph_status": ([_vp], _int),
    "pospopcnt_graph_workspace": ([_vp, ctypes.POINTER(_vp), ctypes.POINTER(_sz)], _int),
    "pospopcnt_graph_destroy": ([_vp], _int),
    "pospopcnt_launch_count": ([], ctypes.c_uint64),
    "pospop_server_create": ([_sz, _int, _int, ctypes.POINTER(_vp)], _int),
    "pospop_server_submit": ([_vp, _int, _vp, _sz, _vp, ctypes.POINTER(ctypes.c_uint64)], _int),
    "pospop_server_create_pooled": ([_sz, _int, _int, ctypes.POINTER(_vp)], _int),
    "pospop_server_submit_host": ([_vp, _int, _vp, _sz, _vp, ctypes.POINTER(ctypes.c_uint64)],
                                  _int),
    "pospop_server_pool_stats": ([_vp, ctypes.POINTER(ctypes.c_uint64)], _int),
    "pospop_server_poll": ([_vp, _vp, _int, _int], _int),
    "pospop_server_drain": ([_vp, _int], _int),
    "pospop_server_stats": ([_vp, ctypes.POINTER(ctypes.c_uint64)], _int),
    "pospop_server_run_trace": ([_vp, _sz, _vp, _vp, _vp, _vp, _vp, _vp, _int], _int),
    "pospop_server_destroy": ([_vp], _int),
}


class Completion(ctypes.Structure):
    """pospop_completion."""
    _fields_ = [("id", ctypes.c_uint64), ("status", ctypes.c_int32), ("w", ctypes.c_int32),
                ("nbytes", ctypes.c_uint64), ("t_submit_ns", ctypes.c_int64),
                ("t_admit_ns", ctypes.c_int64), ("t_launch_ns", ctypes.c_int64),
                ("t_done_ns", ctypes.c_int64)]


COMPLETION_DTYPE = [("id", "<u8"), ("status", "<i4"), ("w", "<i4"), ("nbytes", "<u8"),
                    ("t_submit_ns", "<i8"), ("t_admit_ns", "<i8"), ("t_launch_ns", "<i8"),
                    ("t_done_ns", "<i8")]


def lib():
    """The loaded library (raises if it has not been built)."""
    global _lib
    loaded = _lib
    if loaded is not None:       # set once, never cleared: no lock on the hot path
        return loaded
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(
                    f"{LIB_PATH} is missing: build it with "
                    "`python -m paper_2412_16370_gb300.build` (there is no CPU fallback)")
            L = ctypes.CDLL(LIB_PATH)
            for name, (args, res) in _SIGNATURES.items():
                fn = getattr(L, name)
                fn.argtypes = args
                fn.restype = res
            _lib = L
        return _lib


def strerror(code: int) -> str:
    return lib().pospopcnt_strerror(code).decode()


def _check(rc: int) -> int:
    if rc != POSPOP_OK:
        raise PospopError(rc, strerror(rc))
    return rc


def _ptr(x) -> int | None:
    """Raw address of a torch tensor, numpy array, int or None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if hasattr(x, "ctypes"):
        return x.ctypes.data
    raise TypeError(f"cannot take the address of {type(x).__name__}")


def _nbytes(x) -> int:
    if hasattr(x, "element_size"):
        return x.numel() * x.element_size()
    return int(x.nbytes)


def _stream(stream) -> int | None:
    """A cudaStream_t handle: None means torch's current stream on the current device."""
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream or None
    if isinstance(stream, int):
        return stream or None
    return stream.cuda_stream or None


def init(device: int = 0) -> None:
    _check(lib().pospopcnt_init(device))


def shutdown() -> None:
    lib().pospopcnt_shutdown()


def _typed(w: int, counts, words, n):
    if n is None:
        n = _nbytes(words) // (w // 8)
    fn = getattr(lib(), f"pospopcnt_u{w}")
    return _check(fn(_ptr(counts), _ptr(words), n))


def pospopcnt_u8(counts, words, n=None):
    return _typed(8, counts, words, n)


def pospopcnt_u16(counts, words, n=None):
    return _typed(16, counts, words, n)


def pospopcnt_u32(counts, words, n=None):
    return _typed(32, counts, words, n)


def pospopcnt_u64(counts, words, n=None):
    return _typed(64, counts, words, n)


def pospopcnt_async(w: int, counts, data, nbytes=None, stream=None):
    if nbytes is None:
        nbytes = _nbytes(data)
    return _check(lib().pospopcnt_async(w, _ptr(counts), _ptr(data), nbytes, _stream(stream)))


def pospopcnt_batch(w: int, counts, base, offsets, m=None, stream=None):
    if m is None:
        m = offsets.numel() - 1 if hasattr(offsets, "numel") else len(offsets) - 1
    return _check(lib().pospopcnt_batch(w, _ptr(counts), _ptr(base), _ptr(offsets), m,
                                        _stream(stream)))


def pospopcnt_batch_noalloc(w: int, counts, base, offsets, m=None, stream=None):
    """pospopcnt_batch without any device allocation (m <= 65535; see the header)."""
    if m is None:
        m = offsets.numel() - 1 if hasattr(offsets, "numel") else len(offsets) - 1
    return _check(lib().pospopcnt_batch_noalloc(w, _ptr(counts), _ptr(base), _ptr(offsets), m,
                                                _stream(stream)))


def pospopcnt_multi(widths, counts, ptrs, nbytes, stream=None):
    """Several independent counts in one launch: widths[i], counter address
    counts[i], input address ptrs[i] and length nbytes[i] (sequences of
    ints, or tensors / arrays for the addresses)."""
    import numpy as np
    n = len(widths)
    w = np.ascontiguousarray(widths, dtype=np.int32)
    c = np.ascontiguousarray([_ptr(x) for x in counts], dtype=np.uint64)
    p = np.ascontiguousarray([_ptr(x) for x in ptrs], dtype=np.uint64)
    nb = np.ascontiguousarray(nbytes, dtype=np.uint64)
    if not (len(c) == len(p) == len(nb) == n):
        raise ValueError("widths, counts, ptrs and nbytes differ in length")
    return _check(lib().pospopcnt_multi(n, w.ctypes.data, c.ctypes.data, p.ctypes.data,
                                        nb.ctypes.data, _stream(stream)))


def pospopcnt_gather(w: int, counts, ptrs, lens, n=None, stream=None):
    """Count n device regions (device arrays of start addresses and lengths) into one counter array."""
    if n is None:
        n = ptrs.numel() if hasattr(ptrs, "numel") else len(ptrs)
    return _check(lib().pospopcnt_gather(w, _ptr(counts), _ptr(ptrs), _ptr(lens), n,
                                         _stream(stream)))


def pospopcnt_masked(w: int, counts, words, n: int, select, stream=None):
    """Count the n words whose bit in the selection bitmap is set (device pointers)."""
    return _check(lib().pospopcnt_masked(w, _ptr(counts), _ptr(words), n, _ptr(select),
                                         _stream(stream)))


def pospopcnt_batch_status(stream=None) -> int:
    """Status of the last batch call on ``stream`` (0 or a negative code; does not raise)."""
    return lib().pospopcnt_batch_status(_stream(stream))


def pospopcnt_reserve(m_max: int, stream=None):
    return _check(lib().pospopcnt_reserve(m_max, _stream(stream)))


def pospopcnt_host(w: int, counts, data, nbytes=None):
    if nbytes is None:
        nbytes = _nbytes(data)
    return _check(lib().pospopcnt_host(w, _ptr(counts), _ptr(data), nbytes))


def pospopcnt_roofline_read(data, sum_out, nbytes=None, stream=None):
    if nbytes is None:
        nbytes = _nbytes(data)
    return _check(lib().pospopcnt_roofline_read(_ptr(data), nbytes, _ptr(sum_out),
                                                _stream(stream)))


PLAN_FIELDS = ("grid", "block", "depth", "hint", "size_class", "rows", "launches", "ctas_per_sm")


def pospopcnt_plan(w: int, nbytes: int) -> dict:
    out = (ctypes.c_uint32 * 8)()
    _check(lib().pospopcnt_plan(w, nbytes, out))
    return dict(zip(PLAN_FIELDS, list(out)))


def pospopcnt_autotune(max_bytes: int = 0, path: str | None = None):
    return _check(lib().pospopcnt_autotune(max_bytes, path.encode() if path else None))


def pospopcnt_tune_load(path: str):
    return _check(lib().pospopcnt_tune_load(path.encode()))


def pospopcnt_tune_check(path: str) -> int:
    """0 if the tune file parses, else the 1-based number of its first bad
    line (no GPU needed); raises if the file cannot be read."""
    line = _int(0)
    rc = lib().pospopcnt_tune_check(path.encode(), ctypes.byref(line))
    if rc != POSPOP_OK and line.value == 0:
        raise PospopError(rc, f"cannot read {path}")
    return line.value


def pospopcnt_tune_describe() -> str:
    buf = ctypes.create_string_buffer(8192)
    _check(lib().pospopcnt_tune_describe(buf, len(buf)))
    return buf.value.decode()


def pospopcnt_batch_graph_create(w: int, counts, base, offsets, m=None, stream=None) -> int:
    if m is None:
        m = offsets.numel() - 1 if hasattr(offsets, "numel") else len(offsets) - 1
    h = _vp()
    _check(lib().pospopcnt_batch_graph_create(w, _ptr(counts), _ptr(base), _ptr(offsets), m,
                                              _stream(stream), ctypes.byref(h)))
    return h.value


def pospopcnt_graph_launch(graph: int, stream=None):
    return _check(lib().pospopcnt_graph_launch(graph, _stream(stream)))


def pospopcnt_graph_status(graph: int) -> int:
    """Status of the graph's last replay (0 or a negative code; does not raise)."""
    return lib().pospopcnt_graph_status(graph)


def pospopcnt_graph_workspace(graph: int) -> tuple[int, int]:
    """(device address, bytes) of the graph's own scratch memory."""
    addr, size = _vp(), _sz()
    _check(lib().pospopcnt_graph_workspace(graph, ctypes.byref(addr), ctypes.byref(size)))
    return addr.value or 0, size.value


def pospopcnt_graph_destroy(graph: int):
    return _check(lib().pospopcnt_graph_destroy(graph))


def pospopcnt_launch_count() -> int:
    return int(lib().pospopcnt_launch_count())


# --- serving -----------------------------------------------------------------
def pospop_server_create(mem_budget: int, max_inflight: int = 4096, max_batches: int = 4) -> int:
    h = _vp()
    _check(lib().pospop_server_create(mem_budget, max_inflight, max_batches, ctypes.byref(h)))
    return h.value


def pospop_server_create_pooled(mem_budget: int, max_inflight: int = 4096,
                                max_batches: int = 4) -> int:
    """A server with a device staging pool of mem_budget bytes for host input."""
    h = _vp()
    _check(lib().pospop_server_create_pooled(mem_budget, max_inflight, max_batches,
                                             ctypes.byref(h)))
    return h.value


def pospop_server_submit_host(server: int, w: int, data, nbytes=None, result=None) -> int:
    """Queue a request whose input is host memory (numpy array, CPU tensor or address)."""
    if nbytes is None:
        nbytes = _nbytes(data)
    rid = ctypes.c_uint64()
    _check(lib().pospop_server_submit_host(server, w, _ptr(data), nbytes, _ptr(result),
                                           ctypes.byref(rid)))
    return rid.value


def pospop_server_pool_stats(server: int) -> tuple[int, int, int]:
    """(pool bytes, bytes held now, most bytes ever held at once)."""
    out = (ctypes.c_uint64 * 3)()
    _check(lib().pospop_server_pool_stats(server, out))
    return tuple(int(x) for x in out)


def pospop_server_submit(server: int, w: int, data, nbytes=None, result=None) -> int:
    if nbytes is None:
        nbytes = _nbytes(data)
    rid = ctypes.c_uint64()
    _check(lib().pospop_server_submit(server, w, _ptr(data), nbytes, _ptr(result),
                                      ctypes.byref(rid)))
    return rid.value


def pospop_server_poll(server: int, max_records: int = 1024, timeout_ms: int = 1000) -> list:
    """Finished requests' records (an empty list on timeout)."""
    buf = (Completion * max_records)()
    n = lib().pospop_server_poll(server, buf, max_records, timeout_ms)
    if n == POSPOP_ETIMEDOUT:
        return []
    _check(n if n < 0 else 0)
    return [buf[i] for i in range(n)]


def pospop_server_drain(server: int, timeout_ms: int = 60000) -> int:
    """POSPOP_OK, or POSPOP_ETIMEDOUT (does not raise on a timeout)."""
    rc = lib().pospop_server_drain(server, timeout_ms)
    if rc not in (POSPOP_OK, POSPOP_ETIMEDOUT):
        _check(rc)
    return rc


def pospop_server_stats(server: int) -> dict:
    out = (ctypes.c_uint64 * 6)()
    _check(lib().pospop_server_stats(server, out))
    keys = ("submitted", "finished", "waiting", "inflight", "inflight_bytes", "loop_error")
    vals = list(out)
    vals[5] = ctypes.c_int64(vals[5]).value
    return dict(zip(keys, vals))


def pospop_server_run_trace(server: int, arrival_ns, w, ptrs, nbytes, results, timeout_ms=600000):
    """Replay a request trace natively; returns the completion records (numpy structured array)."""
    import numpy as np
    n = len(arrival_ns)
    arrival_ns = np.ascontiguousarray(arrival_ns, dtype=np.int64)
    w = np.ascontiguousarray(w, dtype=np.int32)
    ptrs = np.ascontiguousarray(ptrs, dtype=np.uint64)
    nbytes = np.ascontiguousarray(nbytes, dtype=np.uint64)
    out = np.zeros(n, dtype=COMPLETION_DTYPE)
    _check(lib().pospop_server_run_trace(server, n, arrival_ns.ctypes.data, w.ctypes.data,
                                         ptrs.ctypes.data, nbytes.ctypes.data, _ptr(results),
                                         out.ctypes.data, timeout_ms))
    return out


def pospop_server_destroy(server: int):
    return _check(lib().pospop_server_destroy(server))
