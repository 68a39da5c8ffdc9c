"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

Each ``pin_*`` function takes an ``oracle.Oracle`` and returns ``None`` when
the pin holds or a short message when it fails.  The same functions run on
the default oracle build (all must hold) and on builds with a planted mistake
(at least one must fail), which shows that a plausible error in the oracle
does not slip through.

None of these re-types the oracle's loop.  The expected values come from:

* base-2 digit strings of Python integers (exhaustive single words),
* ``numpy.unpackbits(..., bitorder="little")`` reshaped to ``w`` columns and
  summed (brute force on tiny inputs: a different formulation of the same
  definition, Section 1),
* ``int.bit_count`` of the whole input as one Python integer (w = 1 and the
  Harley-Seal identity of Section 3.3: all counts add up to the popcount),
* closed forms (all-zero, all-one and single-bit inputs),
* additivity under concatenation and the add-into contract (Section 4,
  step 1 and its footnote),
* the one-hot category histogram (Section 1's GROUP BY use), counted with
  ``numpy.bincount`` from the generator's categories,
* fold consistency between widths w and 2w,
* a 6-sigma band around n*p for Bernoulli(p) bits,
* for the gathered form: each region's numpy brute force, summed (Section 4
  step 1's footnote: non-contiguous regions counted into one C), and the
  split of one array at word boundaries giving the whole array's count,
* for the selected (WHERE) form: numpy brute force (the unpacked word bits
  times the unpacked selection bits), all-ones and all-zero selections, and
  the one-hot category histogram of the selected rows.
"""
from __future__ import annotations

import numpy as np

from paper_2412_16370_gb300 import synth

ALL_W = (1, 2, 4, 8, 16, 32, 64, 128, 256)
WORD_W = (8, 16, 32, 64)


def _digits(v: int, w: int) -> np.ndarray:
    """Base-2 digits of v, least significant first, as a length-w vector."""
    s = format(v, f"0{w}b")[::-1]
    return np.array([int(c) for c in s], dtype=np.uint64)


def _unpack_counts(data: np.ndarray, w: int) -> np.ndarray:
    bits = np.unpackbits(np.asarray(data, dtype=np.uint8), bitorder="little")
    pad = (-bits.size) % w
    if pad:
        bits = np.concatenate([bits, np.zeros(pad, dtype=np.uint8)])
    return bits.reshape(-1, w).sum(axis=0, dtype=np.uint64)


def pin_exhaustive_u8(o):
    for v in range(256):
        exp = _digits(v, 8)
        got_t = o.typed(8, np.array([v], dtype=np.uint8))
        got_b = o.bytes(8, np.array([v], dtype=np.uint8))
        if not (np.array_equal(got_t, exp) and np.array_equal(got_b, exp)):
            return f"single byte {v:#04x}: typed {got_t.tolist()} bytes {got_b.tolist()}"
    return None


def pin_exhaustive_u16(o):
    vals = np.arange(65536, dtype=np.uint16)
    exp = np.array([[int(c) for c in format(v, "016b")[::-1]] for v in range(65536)],
                   dtype=np.uint64)
    # every 16-bit word as its own array of the batch form (little-endian bytes)
    base = vals.astype("<u2").view(np.uint8)
    offsets = np.arange(0, 2 * 65536 + 1, 2, dtype=np.uint64)
    got = o.batch(16, base, offsets)
    if not np.array_equal(got, exp):
        bad = int(np.nonzero((got != exp).any(axis=1))[0][0])
        return f"single u16 {bad:#06x}: {got[bad].tolist()}"
    # Fig. 2 over all 65536 words at once: each bit is set in exactly half of them
    tot = o.typed(16, vals)
    if not np.array_equal(tot, np.full(16, 32768, dtype=np.uint64)):
        return f"all u16 words: {tot.tolist()}"
    for v in (0x0001, 0x8000, 0x1234, 0xFFFF, 0xA5A5):
        if not np.array_equal(o.typed(16, np.array([v], dtype=np.uint16)), _digits(v, 16)):
            return f"typed single u16 {v:#06x}"
    return None


def pin_bruteforce_tiny(o):
    buf = synth.random_bytes(256 + 16, seed=1234)
    for off in range(16):
        for n in range(0, 257):
            data = buf[off:off + n]
            for w in ALL_W:
                got = o.bytes(w, data)
                exp = _unpack_counts(data, w)
                if not np.array_equal(got, exp):
                    return f"w={w} off={off} len={n}: {got.tolist()} != {exp.tolist()}"
    return None


def pin_popcount_sum(o):
    for n in (1, 3, 7, 15, 16, 17, 100, 255, 1000, 4097):
        data = synth.random_bytes(n, seed=77 + n)
        pc = int.from_bytes(data.tobytes(), "little").bit_count()
        for w in ALL_W:
            s = int(o.bytes(w, data).sum())
            if s != pc:
                return f"len={n} w={w}: sum {s} != popcount {pc}"
        if int(o.bytes(1, data)[0]) != pc:
            return f"w=1 len={n}"
    return None


def pin_additivity(o):
    for w in WORD_W:
        W = w // 8
        for (a, b) in ((0, 5), (W, 1), (3 * W, 2 * W + 1), (64 * W, 333), (10 * W, 0)):
            x = synth.random_bytes(a, seed=5 + a)
            y = synth.random_bytes(b, seed=9 + b)
            whole = o.bytes(w, np.concatenate([x, y]))
            parts = o.bytes(w, x) + o.bytes(w, y)
            if not np.array_equal(whole, parts):
                return f"w={w} |x|={a} |y|={b}"
            # add-into: counts passed in are added to, not replaced
            start = np.arange(w, dtype=np.uint64) * np.uint64(1000003)
            into = o.bytes(w, y, counts=start.copy())
            if not np.array_equal(into, start + o.bytes(w, y)):
                return f"add-into w={w} |y|={b}"
    return None


def pin_one_hot(o):
    th = synth.zipf_thresholds()
    for n, seed in ((1, 3), (999, 4), (65536, 5)):
        cat = synth.one_hot_categories(n, seed, th)
        data = synth.one_hot_bytes(n, seed, th)
        exp = np.bincount(cat, minlength=8).astype(np.uint64)
        if not np.array_equal(o.bytes(8, data), exp) or not np.array_equal(o.typed(8, data), exp):
            return f"one-hot n={n}"
        if int(exp.sum()) != n:
            return "one-hot generator"
    return None


def pin_closed_forms(o):
    for w in ALL_W:
        for n in (0, 1, 5, 8, 9, 64, 1001):
            if o.bytes(w, np.zeros(n, dtype=np.uint8)).any():
                return f"all-zero w={w} n={n}"
            got = o.bytes(w, synth.ones_bytes(n))
            nbits = 8 * n
            exp = np.array([nbits // w + (1 if j < nbits % w else 0) for j in range(w)],
                           dtype=np.uint64)
            if not np.array_equal(got, exp):
                return f"all-ones w={w} n={n}: {got.tolist()}"
    for w in WORD_W:
        dt = {8: np.uint8, 16: np.uint16, 32: np.uint32, 64: np.uint64}[w]
        for j in (0, 1, w // 2, w - 1):
            words = np.full(37, 1 << j, dtype=np.uint64).astype(dt)
            exp = np.zeros(w, dtype=np.uint64)
            exp[j] = 37
            if not np.array_equal(o.typed(w, words), exp):
                return f"single-bit typed w={w} j={j}"
            if not np.array_equal(o.bytes(w, words.astype(f"<u{w // 8}").view(np.uint8)), exp):
                return f"single-bit bytes w={w} j={j}"
    return None


def pin_fold(o):
    data = synth.random_bytes(32 * 1000, seed=42)
    for w in (1, 2, 4, 8, 16, 32, 64, 128):
        pw = o.bytes(w, data)
        p2 = o.bytes(2 * w, data)
        if not np.array_equal(pw, p2[:w] + p2[w:]):
            return f"fold {2 * w}->{w}"
    return None


def pin_statistical(o):
    n = 1 << 16
    for p in (0.01, 0.5, 0.99):
        data = synth.bernoulli_bytes(n, p, seed=11)
        for w in WORD_W:
            trials = 8 * n // w
            sd = (trials * p * (1 - p)) ** 0.5
            c = o.bytes(w, data).astype(np.float64)
            if np.any(np.abs(c - trials * p) > 6 * sd + 1):
                return f"Bernoulli p={p} w={w}"
    return None


def pin_typed_vs_bytes(o):
    data = synth.random_bytes(8 * 777, seed=8)
    for w in WORD_W:
        words = data.view(f"<u{w // 8}")
        if not np.array_equal(o.typed(w, words), o.bytes(w, data)):
            return f"typed vs bytes w={w}"
    return None


def pin_mt(o):
    for n in (1, 7, 1000, 65537, 1 << 20):
        data = synth.random_bytes(n, seed=n)
        for w in ALL_W:
            ref = _unpack_counts(data, w) if n <= 65537 else o.bytes(w, data)
            for t in (1, 3, 8):
                if not np.array_equal(o.bytes_mt(w, data, t), ref):
                    return f"mt w={w} n={n} threads={t}"
    return None


def pin_batch(o):
    sizes = np.array([0, 1, 2, 15, 16, 17, 0, 255, 4096, 3], dtype=np.int64)
    offs = synth.csr_offsets(sizes)
    base = synth.random_bytes(int(offs[-1]), seed=21)
    for w in ALL_W:
        got = o.batch(w, base, offs)
        for a in range(len(sizes)):
            exp = _unpack_counts(base[int(offs[a]):int(offs[a + 1])], w)
            if not np.array_equal(got[a], exp):
                return f"batch w={w} array {a}"
    bad = offs.copy()
    bad[3], bad[4] = bad[4], bad[3]
    counts = np.zeros((len(sizes), 8), dtype=np.uint64)
    if o.batch_rc(8, base, bad, counts) != -1 or counts.any():
        return "non-monotone offsets accepted"
    return None


def pin_gather(o):
    rng = np.random.default_rng(3)
    for w in ALL_W:
        lens = [0, 1, 3, 16, 17, 255, 1000, 4097, 0, 9]
        regions = [synth.random_bytes(n, seed=100 + k) for k, n in enumerate(lens)]
        exp = sum(_unpack_counts(r, w) for r in regions)
        got = o.gather(w, regions)
        if not np.array_equal(got, exp):
            return f"gather w={w}"
        W = max(1, w // 8)
        whole = synth.random_bytes(64 * W + 5, seed=7)
        cuts = sorted(set(int(c) * W for c in rng.integers(0, 64, 6)))
        pieces = [whole[a:b] for a, b in zip([0] + cuts, cuts + [whole.size])]
        if not np.array_equal(o.gather(w, pieces), _unpack_counts(whole, w)):
            return f"gather split w={w}"
    return None


def _masked_expected(w, words, n, mask):
    W = w // 8
    bits = np.unpackbits(words[:n * W], bitorder="little").reshape(n, w).astype(np.uint64)
    sel = np.unpackbits(mask, bitorder="little")[:n].astype(np.uint64)
    return (bits * sel[:, None]).sum(axis=0, dtype=np.uint64)


def pin_masked(o):
    for w in WORD_W:
        W = w // 8
        for n in (1, 7, 8, 9, 63, 64, 65, 1000):
            words = synth.random_bytes(n * W, seed=n + w)
            mask = synth.random_bytes((n + 7) // 8, seed=3 * n + w)
            if not np.array_equal(o.masked(w, words, n, mask), _masked_expected(w, words, n, mask)):
                return f"masked w={w} n={n}"
            ones = np.full((n + 7) // 8, 0xFF, dtype=np.uint8)
            if not np.array_equal(o.masked(w, words, n, ones), o.bytes(w, words)):
                return f"masked all-ones w={w} n={n}"
            if o.masked(w, words, n, np.zeros_like(ones)).any():
                return f"masked all-zero w={w} n={n}"
    th = synth.zipf_thresholds()
    n = 10000
    cats = synth.one_hot_categories(n, 9, th)
    data = synth.one_hot_bytes(n, 9, th)
    mask = synth.random_bytes((n + 7) // 8, seed=10)
    sel = np.unpackbits(mask, bitorder="little")[:n].astype(bool)
    exp = np.bincount(cats[sel], minlength=8).astype(np.uint64)
    if not np.array_equal(o.masked(8, data, n, mask), exp):
        return "masked one-hot GROUP BY"
    return None


ALL_PINS = [
    pin_exhaustive_u8, pin_exhaustive_u16, pin_bruteforce_tiny, pin_popcount_sum,
    pin_additivity, pin_one_hot, pin_closed_forms, pin_fold, pin_statistical,
    pin_typed_vs_bytes, pin_mt, pin_batch, pin_gather, pin_masked,
]

#: a fast subset used on the planted-mistake builds
QUICK_PINS = [pin_exhaustive_u8, pin_bruteforce_tiny, pin_popcount_sum, pin_additivity,
              pin_typed_vs_bytes, pin_closed_forms, pin_gather, pin_masked]
