"""Seeded synthetic inputs for the positional population count.

This module only *makes inputs*; it holds no part of the counting method.
The tests, the benchmark and the oracle checks all draw their data from it,
and ``csrc/synth.cu`` is its device twin (same stream, same bytes), used to
fill multi-GiB device buffers quickly.  A GPU test checks that both produce
identical bytes.

Generator: SplitMix64 (G. L. Steele, D. Lea, C. H. Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), used counter-based: output i of
stream ``seed`` is ``mix(seed + (i + 1) * 0x9E3779B97F4A7C15)`` with the
64-bit finaliser ``z ^= z >> 30; z *= 0xBF58476D1CE4E5B9; z ^= z >> 27;
z *= 0x94D049BB133111EB; z ^= z >> 31`` (all arithmetic mod 2**64).

Recipes (the workloads of the benchmark configurations):

* ``random_bytes``: byte ``k`` of the stream is byte ``k % 8`` (little-endian)
  of output ``k // 8``: every bit i.i.d. Bernoulli(0.5).
* ``bernoulli_bytes``: bit ``b`` of byte ``k`` is set iff the top 32 bits of
  output ``8k + b`` are below ``T = round(p * 2**32)``.
* ``one_hot_bytes``: byte ``k`` has exactly bit ``c - 1`` set, where the
  category ``c`` in ``1..K`` is found by comparing the top 32 bits of output
  ``k`` with ``K - 1`` integer CDF thresholds (Zipf(s) over ``K`` classes).
* ``log_uniform_sizes``: array sizes ``floor(exp(U))`` with ``U`` uniform on
  ``[ln lo, ln(hi + 1))``, ``U`` from the top 53 bits of each output.

Every recipe takes a ``start`` so that a window of a long stream can be
regenerated on its own (sampled checks of multi-GiB device arrays).
"""
from __future__ import annotations

import math

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

#: the short/unaligned sweep's start offsets past a 16-byte boundary
SHORT_OFFSETS = tuple(range(16))

#: Zipf exponent and class count of the one-hot (batched) workload
ZIPF_S = 1.1
ZIPF_K = 8


def splitmix64(seed: int, idx: np.ndarray) -> np.ndarray:
    """Outputs ``idx`` (uint64 array) of the SplitMix64 stream ``seed``."""
    idx = np.asarray(idx, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + (idx + np.uint64(1)) * GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def random_bytes(nbytes: int, seed: int, start: int = 0) -> np.ndarray:
    """Bytes ``[start, start + nbytes)`` of the raw stream (Bernoulli(0.5) bits)."""
    if nbytes <= 0:
        return np.zeros(0, dtype=np.uint8)
    b0 = start // 8
    b1 = (start + nbytes + 7) // 8
    words = splitmix64(seed, np.arange(b0, b1, dtype=np.uint64))
    raw = words.astype("<u8").view(np.uint8)
    off = start - 8 * b0
    return raw[off:off + nbytes].copy()


def bernoulli_threshold(p: float) -> int:
    """Integer threshold ``T`` in ``[0, 2**32]`` on a 32-bit uniform: P(bit) = T / 2**32."""
    if not (0.0 <= p <= 1.0):
        raise ValueError("p must lie in [0, 1]")
    return int(min(max(round(p * 4294967296.0), 0), 4294967296))


def bernoulli_bytes(nbytes: int, p: float, seed: int, start: int = 0) -> np.ndarray:
    """Bytes whose bits are i.i.d. Bernoulli(p); p == 0.5 uses the raw stream."""
    if p == 0.5:
        return random_bytes(nbytes, seed, start)
    if nbytes <= 0:
        return np.zeros(0, dtype=np.uint8)
    t = np.uint64(bernoulli_threshold(p))
    out = np.zeros(nbytes, dtype=np.uint8)
    step = 1 << 20
    for c0 in range(0, nbytes, step):
        c1 = min(nbytes, c0 + step)
        k = np.arange(start + c0, start + c1, dtype=np.uint64)
        acc = np.zeros(c1 - c0, dtype=np.uint8)
        for b in range(8):
            u = splitmix64(seed, k * np.uint64(8) + np.uint64(b)) >> np.uint64(32)
            acc |= ((u < t).astype(np.uint8) << np.uint8(b))
        out[c0:c1] = acc
    return out


def ones_bytes(nbytes: int) -> np.ndarray:
    return np.full(max(nbytes, 0), 0xFF, dtype=np.uint8)


def zipf_thresholds(s: float = ZIPF_S, k: int = ZIPF_K) -> list[int]:
    """``k - 1`` integer thresholds on a 32-bit uniform for Zipf(s) over ``k`` classes."""
    if not (1 <= k <= 8):
        raise ValueError("k must be in 1..8 (one bit per class in a byte)")
    weights = [1.0 / (c ** s) for c in range(1, k + 1)]
    total = sum(weights)
    out, acc = [], 0.0
    for c in range(k - 1):
        acc += weights[c] / total
        out.append(int(min(math.floor(acc * 4294967296.0), 4294967295)))
    return out


def zipf_probabilities(s: float = ZIPF_S, k: int = ZIPF_K) -> list[float]:
    weights = [1.0 / (c ** s) for c in range(1, k + 1)]
    total = sum(weights)
    return [x / total for x in weights]


def one_hot_categories(nbytes: int, seed: int, thresholds=None, start: int = 0) -> np.ndarray:
    """Category index ``c - 1`` (0-based) of each byte of the one-hot stream."""
    if thresholds is None:
        thresholds = zipf_thresholds()
    if nbytes <= 0:
        return np.zeros(0, dtype=np.uint8)
    u = splitmix64(seed, np.arange(start, start + nbytes, dtype=np.uint64)) >> np.uint64(32)
    cat = np.zeros(nbytes, dtype=np.uint8)
    for t in thresholds:
        cat += (u >= np.uint64(t)).astype(np.uint8)
    return cat


def one_hot_bytes(nbytes: int, seed: int, thresholds=None, start: int = 0) -> np.ndarray:
    """One-hot bytes: exactly one of the low ``k`` bits set, class drawn by ``thresholds``."""
    cat = one_hot_categories(nbytes, seed, thresholds, start)
    return (np.uint8(1) << cat).astype(np.uint8)


def log_uniform_sizes(m: int, lo: int, hi: int, seed: int) -> np.ndarray:
    """``m`` sizes, log-uniform on ``[lo, hi]`` (int64)."""
    if not (1 <= lo <= hi):
        raise ValueError("need 1 <= lo <= hi")
    u = (splitmix64(seed, np.arange(m, dtype=np.uint64)) >> np.uint64(11)).astype(np.float64)
    u *= 2.0 ** -53
    a, b = math.log(lo), math.log(hi + 1)
    sizes = np.floor(np.exp(a + u * (b - a))).astype(np.int64)
    return np.clip(sizes, lo, hi)


def csr_offsets(sizes: np.ndarray) -> np.ndarray:
    """CSR byte offsets (``m + 1`` uint64, leading zero) of arrays stored back to back."""
    out = np.zeros(len(sizes) + 1, dtype=np.uint64)
    np.cumsum(np.asarray(sizes, dtype=np.uint64), out=out[1:])
    return out


def short_sweep_lengths() -> list[int]:
    """Byte lengths of the short/unaligned sweep: 1..256, then 2**i - 1, 2**i, 2**i + 1 for i = 9..16."""
    lens = set(range(1, 257))
    for i in range(9, 17):
        lens.update((2 ** i - 1, 2 ** i, 2 ** i + 1))
    return sorted(lens)


def case_seed(w: int, length: int, offset: int) -> int:
    """Seed of one short-sweep case: a SplitMix64 output keyed by (w, length, offset)."""
    key = (w << 40) ^ (length << 8) ^ offset
    return int(splitmix64(0x5EED5EED, np.array([key], dtype=np.uint64))[0])


def uniforms(n: int, seed: int, start: int = 0) -> np.ndarray:
    """``n`` doubles uniform on [0, 1) from the top 53 bits of each output."""
    u = splitmix64(seed, np.arange(start, start + n, dtype=np.uint64)) >> np.uint64(11)
    return u.astype(np.float64) * 2.0 ** -53


def poisson_requests(n: int, rate_per_s: float, seed: int, lo: int, hi: int,
                     widths=(8, 16, 32, 64), pool_bytes: int | None = None):
    """A Poisson request stream for the serving workload.

    Returns a dict of numpy arrays: ``arrival_s`` (cumulative exponential
    inter-arrival times at ``rate_per_s``), ``w`` (uniform over ``widths``),
    ``nbytes`` (log-uniform on ``[lo, hi]``) and ``offset`` (uniform start in a
    pool of ``pool_bytes`` bytes, any byte alignment).
    """
    u = uniforms(4 * n, seed).reshape(n, 4)
    gaps = -np.log1p(-u[:, 0]) / rate_per_s
    arrival = np.cumsum(gaps)
    w = np.asarray(widths, dtype=np.int64)[np.minimum((u[:, 1] * len(widths)).astype(np.int64),
                                                      len(widths) - 1)]
    a, b = math.log(lo), math.log(hi + 1)
    nbytes = np.clip(np.floor(np.exp(a + u[:, 2] * (b - a))).astype(np.int64), lo, hi)
    if pool_bytes is None:
        pool_bytes = hi
    span = np.maximum(pool_bytes - nbytes, 0)
    offset = np.floor(u[:, 3] * (span + 1)).astype(np.int64)
    return {"arrival_s": arrival, "w": w, "nbytes": nbytes, "offset": offset}
