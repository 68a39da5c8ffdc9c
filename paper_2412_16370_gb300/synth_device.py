"""ctypes binding of ``libpospop_synth.so``: the device twin of ``synth``.

Fills device buffers (torch tensors) with the same bytes the numpy recipes
of ``synth`` produce, so that multi-GiB inputs are made on the device.
Input generation only; nothing here counts.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import synth

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libpospop_synth.so")

_lock = threading.Lock()
_lib = None


def lib():
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"{LIB_PATH} is missing: run `python -m paper_2412_16370_gb300.build`")
            L = ctypes.CDLL(LIB_PATH)
            vp, sz, u64 = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_uint64
            L.pospop_synth_random.argtypes = [vp, sz, u64, u64, vp]
            L.pospop_synth_bernoulli.argtypes = [vp, sz, u64, u64, u64, vp]
            L.pospop_synth_one_hot.argtypes = [vp, sz, u64, ctypes.POINTER(ctypes.c_uint32),
                                               ctypes.c_int, u64, vp]
            L.pospop_synth_fill.argtypes = [vp, sz, ctypes.c_uint8, vp]
            for f in ("pospop_synth_random", "pospop_synth_bernoulli", "pospop_synth_one_hot",
                      "pospop_synth_fill"):
                getattr(L, f).restype = ctypes.c_int
            _lib = L
        return _lib


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream or None
    if isinstance(stream, int):
        return stream or None
    return stream.cuda_stream or None


def _check(rc):
    if rc != 0:
        raise RuntimeError(f"pospop_synth error {rc}")


def _dst(t, nbytes):
    n = t.numel() * t.element_size() if nbytes is None else nbytes
    return t.data_ptr(), n


def random_(t, seed: int, start: int = 0, nbytes=None, stream=None):
    p, n = _dst(t, nbytes)
    _check(lib().pospop_synth_random(p, n, seed & (2 ** 64 - 1), start, _stream(stream)))
    return t


def bernoulli_(t, p: float, seed: int, start: int = 0, nbytes=None, stream=None):
    if p == 0.5:
        return random_(t, seed, start, nbytes, stream)
    ptr, n = _dst(t, nbytes)
    _check(lib().pospop_synth_bernoulli(ptr, n, seed & (2 ** 64 - 1), synth.bernoulli_threshold(p),
                                        start, _stream(stream)))
    return t


def one_hot_(t, seed: int, thresholds=None, start: int = 0, nbytes=None, stream=None):
    if thresholds is None:
        thresholds = synth.zipf_thresholds()
    arr = (ctypes.c_uint32 * max(1, len(thresholds)))(*thresholds)
    ptr, n = _dst(t, nbytes)
    _check(lib().pospop_synth_one_hot(ptr, n, seed & (2 ** 64 - 1), arr, len(thresholds), start,
                                      _stream(stream)))
    return t


def fill_(t, value: int, nbytes=None, stream=None):
    ptr, n = _dst(t, nbytes)
    _check(lib().pospop_synth_fill(ptr, n, value & 0xFF, _stream(stream)))
    return t
