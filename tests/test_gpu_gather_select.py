"""Gathered regions and word-selected counts on the GPU vs the CPU oracle.

pospopcnt_gather: many separate regions (unaligned, overlapping, empty) of
device memory counted into one counter array, each region its own word
stream.  pospopcnt_masked: only the words whose selection bit is set are
counted (the GROUP BY count with a WHERE bitmap), at every word phase of the
16-byte granule, across the short path, the CSA paths and the tails.
"""
import numpy as np
import pytest
import torch

from paper_2412_16370_gb300 import binding as pp
from paper_2412_16370_gb300 import synth, synth_device

from _gpu import WORD_W, counts_np

pytestmark = pytest.mark.gpu


@pytest.fixture
def tune_override(gpu, tmp_path):
    saved = tmp_path / "saved_tune.txt"
    saved.write_text(pp.pospopcnt_tune_describe())

    def install(text):
        f = tmp_path / "tune.txt"
        f.write_text(text)
        pp.pospopcnt_tune_load(str(f))

    yield install
    pp.pospopcnt_tune_load(str(saved))


def _regions(m, seed, span, hi):
    rng = np.random.default_rng(seed)
    lens = synth.log_uniform_sizes(m, 1, hi, seed=seed)
    lens[::13] = 0
    starts = rng.integers(0, span - hi, m)
    return starts.astype(np.int64), lens.astype(np.int64)


def _gather_gpu(w, buf, starts, lens):
    dev = buf.device
    ptrs = torch.from_numpy(buf.data_ptr() + starts).to(dev)
    ln = torch.from_numpy(lens).to(dev)
    c = torch.zeros(w, dtype=torch.int64, device=dev)
    pp.pospopcnt_gather(w, c, ptrs, ln, len(starts))
    torch.cuda.synchronize()
    return counts_np(c)


def test_gather_matches_oracle(gpu, orc):
    span = 64 << 20
    buf = torch.empty(span, dtype=torch.uint8, device=gpu)
    synth_device.random_(buf, 31)
    host = buf.cpu().numpy()
    for m, hi, seed in ((1, 1000, 1), (37, 5000, 2), (3000, 1 << 20, 3)):
        starts, lens = _regions(m, seed, span, hi)
        regions = [host[s:s + n] for s, n in zip(starts, lens)]
        for w in (1, 2, 4, 8, 16, 32, 64, 128, 256):
            assert np.array_equal(_gather_gpu(w, buf, starts, lens), orc.gather(w, regions)), (m, w)


def test_gather_split_array_equals_whole(gpu, orc):
    n = (5 << 20) + 3
    buf = torch.empty(n + 64, dtype=torch.uint8, device=gpu)
    synth_device.random_(buf, 77)
    data = buf[7:7 + n]
    rng = np.random.default_rng(0)
    for w in WORD_W:
        W = w // 8
        cuts = np.unique(rng.integers(1, n // W, 500) * W)
        starts = np.concatenate([[0], cuts]).astype(np.int64)
        lens = np.diff(np.concatenate([starts, [n]])).astype(np.int64)
        whole = torch.zeros(w, dtype=torch.int64, device=gpu)
        pp.pospopcnt_async(w, whole, data)
        got = _gather_gpu(w, data, starts, lens)
        assert np.array_equal(got, counts_np(whole)), w
        assert np.array_equal(got, orc.bytes(w, data.cpu().numpy())), w


def test_gather_every_variant(gpu, orc, tune_override):
    span = 8 << 20
    buf = torch.empty(span, dtype=torch.uint8, device=gpu)
    synth_device.random_(buf, 5)
    host = buf.cpu().numpy()
    starts, lens = _regions(400, 9, span, 200000)
    regions = [host[s:s + n] for s, n in zip(starts, lens)]
    widths = WORD_W + (256,)
    exp = {w: orc.gather(w, regions) for w in widths}
    for bs, minb in ((256, 2), (512, 1), (128, 4)):
        for depth in (16, 32):
            for item_rows in (1, 15, 31, 127):
                tune_override(f"batch {bs} {minb} {depth} 1 1 {item_rows} 2\n")
                for w in widths:
                    assert np.array_equal(_gather_gpu(w, buf, starts, lens), exp[w]), \
                        (bs, depth, item_rows, w)


def _masked_gpu(w, words, n, sel):
    c = torch.zeros(w, dtype=torch.int64, device=words.device)
    pp.pospopcnt_masked(w, c, words, n, sel)
    torch.cuda.synchronize()
    return counts_np(c)


def _dev_bytes(a, dev, pad=0):
    t = torch.empty(a.size + pad + 64, dtype=torch.uint8, device=dev)
    v = t[pad:pad + a.size]
    v.copy_(torch.from_numpy(np.ascontiguousarray(a)))
    return v


@pytest.mark.parametrize("w", WORD_W)
def test_masked_phases_and_sizes(gpu, orc, w):
    W = w // 8
    rng = np.random.default_rng(w)
    sizes = sorted(set([1, 2, 3, 7, 8, 9, 31, 32, 33, 100, 1000, 4095, 4096, 4097, 100003,
                        (1 << 20) + 5] + [int(x) for x in rng.integers(1, 1 << 18, 20)]))
    for n in sizes:
        phase = int(rng.integers(0, 16 // W)) * W        # word-aligned, any 16-byte phase
        words_h = synth.random_bytes(n * W, seed=n * 3 + w)
        sel_h = synth.random_bytes((n + 7) // 8, seed=n * 5 + w)
        sel_h[-1] |= 0xF0          # bits past n must not count
        words = _dev_bytes(words_h, gpu, phase)
        sel = _dev_bytes(sel_h, gpu, 0)
        assert sel.data_ptr() % 4 == 0
        exp = orc.masked(w, words_h, n, sel_h)
        assert np.array_equal(_masked_gpu(w, words, n, sel), exp), (n, phase)


def test_masked_per_warp_rows(gpu, orc, tune_override):
    """Each warp gets 1..40 rows: selection through short, CSA_15 and CSA_16+4 paths."""
    for depth in (16, 32):
        lines = [f"stream {c} 128 4 {depth} 1 1 1000000" for c in range(5)]
        tune_override("\n".join(lines) + "\n")
        for w in WORD_W:
            W = w // 8
            for k in (1, 2, 3, 4, 5, 15, 16, 17, 31, 32, 33, 40, 47):
                n = max(1, (4 * k * 512 - 3 * W) // W)
                words_h = synth.random_bytes(n * W, seed=k + w)
                sel_h = synth.random_bytes((n + 7) // 8, seed=k * 7 + w)
                words = _dev_bytes(words_h, gpu, W)
                sel = _dev_bytes(sel_h, gpu, 0)
                assert np.array_equal(_masked_gpu(w, words, n, sel),
                                      orc.masked(w, words_h, n, sel_h)), (depth, w, k)


def test_masked_closed_forms_and_group_by(gpu, orc):
    n = 3_000_001
    for w in WORD_W:
        W = w // 8
        words_h = synth.random_bytes(n * W, seed=w)
        words = _dev_bytes(words_h, gpu, 16 - W)
        ones = torch.full(((n + 7) // 8 + 8,), 0xFF, dtype=torch.uint8, device=gpu)
        zeros = torch.zeros_like(ones)
        plain = torch.zeros(w, dtype=torch.int64, device=gpu)
        pp.pospopcnt_async(w, plain, words)
        assert np.array_equal(_masked_gpu(w, words, n, ones), counts_np(plain))
        assert not _masked_gpu(w, words, n, zeros).any()
    # GROUP BY category WHERE selected
    cats = synth.one_hot_categories(n, 12)
    data = _dev_bytes(synth.one_hot_bytes(n, 12), gpu, 5)
    sel_h = synth.random_bytes((n + 7) // 8, seed=13)
    chosen = np.unpackbits(sel_h, bitorder="little")[:n].astype(bool)
    exp = np.bincount(cats[chosen], minlength=8).astype(np.uint64)
    assert np.array_equal(_masked_gpu(8, data, n, _dev_bytes(sel_h, gpu)), exp)


def test_masked_large(gpu, orc):
    n = 64 << 20     # 64 Mi words of 32 bits = 256 MiB
    words = torch.empty(4 * n, dtype=torch.uint8, device=gpu)
    synth_device.random_(words, 21)
    sel = torch.empty((n + 7) // 8, dtype=torch.uint8, device=gpu)
    synth_device.bernoulli_(sel, 0.3, 22)
    got = _masked_gpu(32, words, n, sel)
    exp = orc.masked(32, words.cpu().numpy(), n, sel.cpu().numpy())
    assert np.array_equal(got, exp)


def test_argument_errors(gpu):
    L = pp.lib()
    c = torch.zeros(64, dtype=torch.int64, device=gpu)
    d = torch.zeros(4096, dtype=torch.uint8, device=gpu)
    s = None
    assert L.pospopcnt_masked(16, c.data_ptr(), d.data_ptr() + 1, 10, d.data_ptr(), s) == pp.POSPOP_EINVAL
    assert L.pospopcnt_masked(16, c.data_ptr(), d.data_ptr(), 10, d.data_ptr() + 2, s) == pp.POSPOP_EINVAL
    assert L.pospopcnt_masked(4, c.data_ptr(), d.data_ptr(), 10, d.data_ptr(), s) == pp.POSPOP_EINVAL
    assert L.pospopcnt_masked(16, c.data_ptr(), d.data_ptr(), 0, None, s) == pp.POSPOP_OK
    assert L.pospopcnt_gather(16, c.data_ptr(), None, d.data_ptr(), 3, s) == pp.POSPOP_EINVAL
    h = np.zeros(4, dtype=np.uint64)
    assert L.pospopcnt_gather(16, c.data_ptr(), h.ctypes.data, d.data_ptr(), 3, s) == pp.POSPOP_EPTR


def test_masked_and_wide_every_tune_shape(gpu, orc, tune_override):
    """Every launch shape the tune table may choose dispatches to a kernel
    compiled for that block size (selected count and w = 256)."""
    n = 300_001
    words_h = synth.random_bytes(4 * n, seed=1)
    sel_h = synth.random_bytes((n + 7) // 8, seed=2)
    words = _dev_bytes(words_h, gpu, 4)
    sel = _dev_bytes(sel_h, gpu)
    exp32 = orc.masked(32, words_h, n, sel_h)
    exp256 = orc.bytes(256, words_h)
    for bs, minb in ((256, 2), (512, 1), (128, 4)):
        for depth in (16, 32):
            for hint in (0, 1):
                lines = [f"stream {c} {bs} {minb} {depth} {hint} 1 4" for c in range(5)]
                tune_override("\n".join(lines) + "\n")
                assert np.array_equal(_masked_gpu(32, words, n, sel), exp32), (bs, depth, hint)
                c = torch.zeros(256, dtype=torch.int64, device=gpu)
                pp.pospopcnt_async(256, c, words)
                torch.cuda.synchronize()
                assert np.array_equal(counts_np(c), exp256), (bs, depth, hint)


@pytest.mark.parametrize("w", WORD_W)
def test_masked_staged_form(gpu, orc, tune_override, w):
    """Selected counts large enough for the staged form (bulk copies into
    shared memory, at least two 16-row chunks per warp of the grid), with
    16-byte-aligned and word-aligned starts and ragged ends, for every ring
    shape and the register form (tune entry `staged k`), against the oracle,
    with bitmaps on and 4 bytes past a 16-byte boundary."""
    W = w // 8
    base_tune = pp.pospopcnt_tune_describe()
    keep = "\n".join(l for l in base_tune.splitlines() if not l.startswith("staged"))
    # 48 MiB of words: at least two 16-row chunks per warp for every ring
    # shape (the 16-warp ring needs 38 MiB)
    for extra, seed, pad in ((0, 1, 0), (3, 2, 0), ((1 << 20) // W + 1, 3, 0),
                             (5, 4, W), (0, 5, 16 - W)):
        n = (48 << 20) // W + extra
        words_h = synth.random_bytes(n * W, seed=seed * 10 + w)
        sel_h = synth.random_bytes(4 * ((n + 31) // 32), seed=seed * 10 + w + 1)
        words = _dev_bytes(words_h, gpu, pad)   # pad > 0: the start is inside a granule
        assert words.data_ptr() % 16 == pad
        exp = orc.masked(w, words_h, n, sel_h)
        sel16 = _dev_bytes(sel_h, gpu, 0)
        sel4 = _dev_bytes(sel_h, gpu, 4)
        assert sel16.data_ptr() % 16 == 0 and sel4.data_ptr() % 16 == 4
        for staged in (1, 2, 3, 0):   # the three ring shapes, then the register form
            tune_override(keep + f"\nstaged {staged}\n")
            assert np.array_equal(_masked_gpu(w, words, n, sel16), exp), (n, pad, staged)
            assert np.array_equal(_masked_gpu(w, words, n, sel4), exp), (n, pad, staged)
        assert pp.pospopcnt_batch_status() == pp.POSPOP_OK
