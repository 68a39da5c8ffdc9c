"""Helpers for the GPU parity tests: device <-> host moves and comparisons."""
from __future__ import annotations

from concurrent.futures import ThreadPoolExecutor

import numpy as np
import torch

from paper_2412_16370_gb300 import binding as pp

WORD_W = (8, 16, 32, 64)


def to_dev(a: np.ndarray, dev, align_pad: int = 0) -> torch.Tensor:
    """Copy a uint8 numpy array to the device (16-byte aligned start + align_pad)."""
    t = torch.empty(a.size + align_pad + 16, dtype=torch.uint8, device=dev)
    v = t[align_pad:align_pad + a.size]
    v.copy_(torch.from_numpy(np.ascontiguousarray(a)))
    return v


def counts_np(t: torch.Tensor) -> np.ndarray:
    return t.cpu().numpy().view(np.uint64)


def gpu_count(w: int, data: torch.Tensor, stream=None) -> np.ndarray:
    c = torch.zeros(w, dtype=torch.int64, device=data.device)
    pp.pospopcnt_async(w, c, data, data.numel(), stream)
    torch.cuda.synchronize()
    return counts_np(c)


def oracle_device_bytes(orc, widths, data: torch.Tensor, chunk: int = 1 << 30, threads: int = 0):
    """Oracle counts (one array per w) of a device buffer, copied back in word-aligned chunks."""
    import os
    threads = threads or max(1, os.cpu_count() or 1)
    out = {w: np.zeros(w, dtype=np.uint64) for w in widths}
    n = data.numel()
    host = torch.empty(min(chunk, n), dtype=torch.uint8, pin_memory=True)
    for c0 in range(0, n, chunk):
        c1 = min(n, c0 + chunk)
        h = host[:c1 - c0]
        h.copy_(data[c0:c1])
        a = h.numpy()
        for w in widths:
            orc.bytes_mt(w, a, threads, counts=out[w])
    return out


def oracle_batch_parallel(orc, w: int, base: np.ndarray, offsets: np.ndarray, threads: int = 16):
    """oracle.batch over array ranges in parallel threads (ctypes releases the GIL)."""
    m = offsets.size - 1
    out = np.zeros((m, w), dtype=np.uint64)
    bounds = np.linspace(0, m, threads + 1).astype(np.int64)

    def run(k):
        a0, a1 = int(bounds[k]), int(bounds[k + 1])
        if a1 > a0:
            sub = (offsets[a0:a1 + 1] - offsets[a0]).astype(np.uint64)
            lo, hi = int(offsets[a0]), int(offsets[a1])
            orc.batch(w, base[lo:hi], sub, counts=out[a0:a1])

    with ThreadPoolExecutor(threads) as ex:
        list(ex.map(run, range(threads)))
    return out


def oracle_batch_device(orc, widths, base: torch.Tensor, offsets: np.ndarray,
                        chunk: int = 1 << 30, threads: int = 0):
    """Oracle counts of every array of a batch resident on the device: the
    arrays are copied back in runs of whole arrays of at most ``chunk`` bytes
    (an array larger than ``chunk`` is a run of its own) and each run is
    counted with oracle.batch on all host cores.  Returns {w: (m, w) uint64}."""
    import os
    threads = threads or max(1, os.cpu_count() or 1)
    m = offsets.size - 1
    out = {w: np.zeros((m, w), dtype=np.uint64) for w in widths}
    span = int(max(chunk, int(np.diff(offsets).max()) if m else 0))
    host = torch.empty(max(1, span), dtype=torch.uint8, pin_memory=True)
    a0 = 0
    while a0 < m:
        # the longest run of arrays a0 .. a1-1 within `span` bytes (at least one)
        a1 = int(np.searchsorted(offsets, offsets[a0] + span, side="right")) - 1
        a1 = min(max(a1, a0 + 1), m)
        lo, hi = int(offsets[a0]), int(offsets[a1])
        h = host[:hi - lo]
        h.copy_(base[lo:hi])
        sub = (offsets[a0:a1 + 1] - offsets[a0]).astype(np.uint64)
        for w in widths:
            out[w][a0:a1] = oracle_batch_parallel(orc, w, h.numpy(), sub, threads)
        a0 = a1
    return out
