"""CPU oracle for the positional population count (TEST INFRASTRUCTURE).

Only the test suite, ``__graft_entry__.smoke()`` and the benchmark's CPU
baseline / reference leg may import this package.  The product library never
does, and this package never imports the product library.

``pospopcnt_oracle.c`` is a plain C99 restatement of the definition
(arXiv 2412.16370, Fig. 2 and the interleaved-streams description of
Section 1); this module builds it with gcc and calls it through ctypes on
numpy arrays.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pospopcnt_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LOCK = threading.Lock()
_LIBS: dict[int, "Oracle"] = {}

WIDTHS = (1, 2, 4, 8, 16, 32, 64, 128, 256)
OK = 0
EINVAL = -1

# Planted mistakes compiled in by -DORACLE_MUTANT=k (see pospopcnt_oracle.c).
MUTANTS = {
    1: "big-endian word reading",
    2: "trailing partial word dropped",
    3: "position index off by one",
    4: "last byte skipped",
    5: "counts overwritten instead of added to",
    6: "selection bitmap read most significant bit first",
    7: "gathered regions counted as one continuous stream",
}

_CFLAGS = ["-std=c99", "-O2", "-fno-tree-vectorize", "-fPIC", "-shared", "-pthread", "-Wall"]


def lib_path(mutant: int = 0) -> str:
    name = "liboracle.so" if mutant == 0 else f"liboracle_m{mutant}.so"
    return os.path.join(_BUILD, name)


def build(mutant: int = 0, force: bool = False) -> str:
    """Compile the oracle (optionally a planted-mistake variant); return the .so path."""
    out = lib_path(mutant)
    if (not force and os.path.exists(out)
            and os.path.getmtime(out) >= os.path.getmtime(_SRC)):
        return out
    os.makedirs(_BUILD, exist_ok=True)
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", *_CFLAGS, f"-DORACLE_MUTANT={mutant}", _SRC, "-o", tmp]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


class Oracle:
    """ctypes wrapper of one oracle build."""

    def __init__(self, path: str):
        self.path = path
        lib = ctypes.CDLL(path)
        u64p = ctypes.POINTER(ctypes.c_uint64)
        vp = ctypes.c_void_p
        for name in ("oracle_pospop_u8", "oracle_pospop_u16", "oracle_pospop_u32",
                     "oracle_pospop_u64"):
            fn = getattr(lib, name)
            fn.argtypes = [u64p, vp, ctypes.c_size_t]
            fn.restype = None
        lib.oracle_pospop_bytes.argtypes = [ctypes.c_int, u64p, vp, ctypes.c_size_t]
        lib.oracle_pospop_bytes.restype = ctypes.c_int
        lib.oracle_pospop_batch.argtypes = [ctypes.c_int, u64p, vp, vp, ctypes.c_size_t]
        lib.oracle_pospop_batch.restype = ctypes.c_int
        lib.oracle_pospop_bytes_mt.argtypes = [ctypes.c_int, u64p, vp, ctypes.c_size_t,
                                               ctypes.c_int]
        lib.oracle_pospop_bytes_mt.restype = ctypes.c_int
        lib.oracle_pospop_gather.argtypes = [ctypes.c_int, u64p, vp, vp, ctypes.c_size_t]
        lib.oracle_pospop_gather.restype = ctypes.c_int
        lib.oracle_pospop_masked.argtypes = [ctypes.c_int, u64p, vp, ctypes.c_size_t, vp]
        lib.oracle_pospop_masked.restype = ctypes.c_int
        lib.oracle_mutant_id.argtypes = []
        lib.oracle_mutant_id.restype = ctypes.c_int
        self.lib = lib
        self.mutant = lib.oracle_mutant_id()

    @staticmethod
    def _counts(w: int, counts):
        if counts is None:
            counts = np.zeros(w, dtype=np.uint64)
        if counts.dtype != np.uint64 or not counts.flags.c_contiguous:
            raise TypeError("counts must be a C-contiguous uint64 array")
        return counts

    @staticmethod
    def _u64p(a: np.ndarray):
        return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))

    def typed(self, w: int, words: np.ndarray, counts=None) -> np.ndarray:
        """Fig. 2 over a typed word array (uint8/16/32/64 for w = 8/16/32/64)."""
        dt = {8: np.uint8, 16: np.uint16, 32: np.uint32, 64: np.uint64}[w]
        words = np.ascontiguousarray(words, dtype=dt)
        counts = self._counts(w, counts)
        fn = getattr(self.lib, f"oracle_pospop_u{w}")
        fn(self._u64p(counts), words.ctypes.data, words.size)
        return counts

    def bytes(self, w: int, data: np.ndarray, counts=None) -> np.ndarray:
        """Interleaved-stream definition over a byte array (any length)."""
        data = np.ascontiguousarray(data, dtype=np.uint8)
        counts = self._counts(w, counts)
        rc = self.lib.oracle_pospop_bytes(w, self._u64p(counts), data.ctypes.data, data.size)
        if rc != OK:
            raise ValueError(f"oracle_pospop_bytes returned {rc}")
        return counts

    def bytes_rc(self, w: int, counts: np.ndarray, ptr, nbytes: int) -> int:
        """Raw call (for argument-error checks)."""
        return self.lib.oracle_pospop_bytes(w, self._u64p(counts) if counts is not None else None,
                                            ptr, nbytes)

    def bytes_mt(self, w: int, data: np.ndarray, nthreads: int, counts=None) -> np.ndarray:
        """Timed-baseline form: Fig. 2 word loop split across ``nthreads`` threads."""
        data = np.ascontiguousarray(data, dtype=np.uint8)
        counts = self._counts(w, counts)
        rc = self.lib.oracle_pospop_bytes_mt(w, self._u64p(counts), data.ctypes.data, data.size,
                                             int(nthreads))
        if rc != OK:
            raise ValueError(f"oracle_pospop_bytes_mt returned {rc}")
        return counts

    def batch(self, w: int, base: np.ndarray, offsets: np.ndarray, counts=None) -> np.ndarray:
        """Per-array counts (shape ``(m, w)``) of arrays given by CSR byte offsets."""
        base = np.ascontiguousarray(base, dtype=np.uint8)
        offsets = np.ascontiguousarray(offsets, dtype=np.uint64)
        m = offsets.size - 1
        if counts is None:
            counts = np.zeros((m, w), dtype=np.uint64)
        rc = self.lib.oracle_pospop_batch(w, self._u64p(counts), base.ctypes.data,
                                          offsets.ctypes.data, m)
        if rc != OK:
            raise ValueError(f"oracle_pospop_batch returned {rc}")
        return counts

    def gather(self, w: int, regions, counts=None) -> np.ndarray:
        """Several byte arrays (a list of uint8 arrays) counted into one counter array."""
        regions = [np.ascontiguousarray(r, dtype=np.uint8) for r in regions]
        ptrs = np.array([r.ctypes.data if r.size else 0 for r in regions], dtype=np.uint64)
        lens = np.array([r.size for r in regions], dtype=np.uint64)
        counts = self._counts(w, counts)
        rc = self.lib.oracle_pospop_gather(w, self._u64p(counts), ptrs.ctypes.data,
                                           lens.ctypes.data, len(regions))
        if rc != OK:
            raise ValueError(f"oracle_pospop_gather returned {rc}")
        return counts

    def masked(self, w: int, words: np.ndarray, n: int, mask: np.ndarray, counts=None) -> np.ndarray:
        """Fig. 2 over the n words (little-endian bytes) whose selection bit is set."""
        words = np.ascontiguousarray(words, dtype=np.uint8)
        mask = np.ascontiguousarray(mask, dtype=np.uint8)
        if words.size < n * (w // 8) or mask.size < (n + 7) // 8:
            raise ValueError("words or mask too short")
        counts = self._counts(w, counts)
        rc = self.lib.oracle_pospop_masked(w, self._u64p(counts), words.ctypes.data, n,
                                           mask.ctypes.data)
        if rc != OK:
            raise ValueError(f"oracle_pospop_masked returned {rc}")
        return counts

    def batch_rc(self, w: int, base: np.ndarray, offsets: np.ndarray, counts: np.ndarray) -> int:
        return self.lib.oracle_pospop_batch(w, self._u64p(counts), base.ctypes.data,
                                            offsets.ctypes.data, offsets.size - 1)


def load(mutant: int = 0) -> Oracle:
    """Build (if needed) and load the oracle; ``mutant`` > 0 loads a planted-mistake build."""
    with _LOCK:
        if mutant not in _LIBS:
            _LIBS[mutant] = Oracle(build(mutant))
        return _LIBS[mutant]
