"""Single-array pospopcnt on the GPU vs the CPU oracle, bit-exact.

Covers the plain workload (1 MiB of uint16 words, Bernoulli(0.5), seed 0),
the short/unaligned sweep (every byte length up to 256 and 2**i - 1, 2**i,
2**i + 1 for i = 9..16, at every start offset 0..15 past a 16-byte boundary,
for w = 8, 16, 32, 64, one launch per array), sizes that put 1..40 rows of
512 B on a warp (the short path, CSA_15-only and CSA_16+4 boundaries),
widths 1, 2, 4, add-into, the host-memory path and argument errors.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2412_16370_gb300 import binding as pp
from paper_2412_16370_gb300 import synth, synth_device

from _gpu import WORD_W, counts_np, gpu_count, to_dev

pytestmark = pytest.mark.gpu


def test_plain_config_typed_and_async(gpu, orc):
    n = 524288
    host = synth.bernoulli_bytes(2 * n, 0.5, seed=0)
    words_h = host.view("<u2")
    d = to_dev(host, gpu)
    assert d.data_ptr() % 16 == 0
    exp16 = orc.typed(16, words_h)
    # Fig. 2 entry point on device pointers
    c = torch.zeros(16, dtype=torch.int64, device=gpu)
    pp.pospopcnt_u16(c, d.view(torch.int16), n)
    assert np.array_equal(counts_np(c), exp16)
    # byte-length async form
    assert np.array_equal(gpu_count(16, d), exp16)
    # the other typed entry points over the same bytes
    for w in (8, 32, 64):
        c = torch.zeros(w, dtype=torch.int64, device=gpu)
        getattr(pp, f"pospopcnt_u{w}")(c, d, 2 * n // (w // 8))
        assert np.array_equal(counts_np(c), orc.typed(w, host.view(f"<u{w // 8}"))), w


@pytest.mark.parametrize("w", WORD_W)
def test_short_unaligned_sweep(gpu, orc, w):
    lens = synth.short_sweep_lengths()
    cases = [(n, off) for n in lens for off in synth.SHORT_OFFSETS]
    slot = 16 + max(lens) + 16
    slot = (slot + 15) // 16 * 16
    host = np.zeros(slot * len(cases), dtype=np.uint8)
    for k, (n, off) in enumerate(cases):
        host[k * slot + off:k * slot + off + n] = synth.random_bytes(n, synth.case_seed(w, n, off))
    # poison the bytes around every case: they must never be counted
    mask = np.ones(host.size, dtype=bool)
    for k, (n, off) in enumerate(cases):
        mask[k * slot + off:k * slot + off + n] = False
    host[mask] = 0xFF
    d = to_dev(host, gpu)
    counts = torch.zeros((len(cases), w), dtype=torch.int64, device=gpu)
    base = d.data_ptr()
    stream = torch.cuda.current_stream()
    for k, (n, off) in enumerate(cases):
        pp.pospopcnt_async(w, counts[k], base + k * slot + off, n, stream)
    torch.cuda.synchronize()
    got = counts_np(counts)
    for k, (n, off) in enumerate(cases):
        exp = orc.bytes(w, host[k * slot + off:k * slot + off + n])
        assert np.array_equal(got[k], exp), (w, n, off)


@pytest.fixture
def tune_override(gpu, tmp_path):
    """Install test tune tables; restore the original afterwards."""
    saved = tmp_path / "saved_tune.txt"
    saved.write_text(pp.pospopcnt_tune_describe())

    def install(text):
        f = tmp_path / "tune.txt"
        f.write_text(text)
        pp.pospopcnt_tune_load(str(f))

    yield install
    pp.pospopcnt_tune_load(str(saved))


@pytest.mark.parametrize("depth", (16, 32))
@pytest.mark.parametrize("hint", (0, 1))
def test_per_warp_row_counts(gpu, orc, tune_override, depth, hint):
    """One block of 4 warps: each warp gets k = 1..40 rows of 512 B (short path,
    CSA_15 only, CSA_16+4 groups with masked and unmasked loads, tails)."""
    lines = [f"stream {c} 128 4 {depth} {hint} 1 1000000" for c in range(5)]
    tune_override("\n".join(lines) + "\n")
    assert pp.pospopcnt_plan(16, 40 * 4 * 512)["grid"] == 1
    rng = np.random.default_rng(depth + hint)
    for k in list(range(1, 41)) + [47, 48, 63, 64, 65]:
        for d in (-513, -17, -1, 0, 1, 15, 511):
            n = max(1, 4 * k * 512 + d)
            off = int(rng.integers(0, 16))
            host = synth.random_bytes(n, seed=n * 7 + off)
            dd = to_dev(host, gpu, align_pad=off)
            for w in WORD_W:
                assert np.array_equal(gpu_count(w, dd), orc.bytes(w, host)), (k, d, off, w)


def test_every_launch_variant(gpu, orc, tune_override):
    """Every kernel variant of the table, on a size spanning many rows per warp."""
    host = synth.random_bytes((3 << 20) + 333, seed=4242)
    for bs, minb in ((256, 2), (512, 1), (128, 4)):
        for depth in (16, 32):
            for hint in (0, 1):
                lines = [f"stream {c} {bs} {minb} {depth} {hint} 1 64" for c in range(5)]
                tune_override("\n".join(lines) + "\n")
                dd = to_dev(host, gpu, align_pad=9)
                for w in WORD_W:
                    assert np.array_equal(gpu_count(w, dd), orc.bytes(w, host)), (bs, depth, hint, w)


def test_random_sizes_and_offsets(gpu, orc):
    sizes = synth.log_uniform_sizes(120, 1, 64 << 20, seed=99)
    for k, n in enumerate(sizes.tolist()):
        off = k % 16
        host = synth.random_bytes(n, seed=1000 + k)
        d = to_dev(host, gpu, align_pad=off)
        w = WORD_W[k % 4]
        assert np.array_equal(gpu_count(w, d), orc.bytes(w, host)), (n, off, w)


@pytest.mark.parametrize("w", (1, 2, 4))
def test_sub_byte_widths(gpu, orc, w):
    for k, n in enumerate((1, 2, 15, 16, 17, 513, 4096, 100001, 3 << 20)):
        host = synth.random_bytes(n, seed=k)
        d = to_dev(host, gpu, align_pad=k % 16)
        assert np.array_equal(gpu_count(w, d), orc.bytes(w, host)), (w, n)


def test_add_into_and_all_ones(gpu, orc):
    for w in WORD_W:
        n = 3 * (1 << 20) + 7
        d = to_dev(synth.ones_bytes(n), gpu, align_pad=3)
        start = torch.arange(w, dtype=torch.int64, device=gpu) * 1000003
        c = start.clone()
        pp.pospopcnt_async(w, c, d, n)
        pp.pospopcnt_async(w, c, d, n)
        torch.cuda.synchronize()
        nbits = 8 * n
        per = np.array([nbits // w + (1 if j < nbits % w else 0) for j in range(w)], np.uint64)
        assert np.array_equal(counts_np(c) - counts_np(start), 2 * per)


def test_zero_and_one_hot(gpu, orc):
    d = torch.zeros(1 << 20, dtype=torch.uint8, device=gpu)
    for w in WORD_W:
        assert not gpu_count(w, d[1:]).any()
    cats = synth.one_hot_categories(1 << 20, seed=17)
    host = synth.one_hot_bytes(1 << 20, seed=17)
    exp = np.bincount(cats, minlength=8).astype(np.uint64)
    assert np.array_equal(gpu_count(8, to_dev(host, gpu)), exp)


def test_host_memory_paths(gpu, orc):
    n = (150 << 20) + 12345   # crosses the 64 MiB staging chunks
    host = synth.random_bytes(n, seed=31)
    for w in WORD_W:
        exp = orc.bytes_mt(w, host, 8)
        got = np.zeros(w, dtype=np.uint64)
        pp.pospopcnt_host(w, got, host)                  # pageable: staged copies
        assert np.array_equal(got, exp), ("pageable", w)
        pinned = torch.from_numpy(host).pin_memory()
        got2 = np.zeros(w, dtype=np.uint64)
        pp.pospopcnt_host(w, got2, pinned)               # pinned: read in place
        assert np.array_equal(got2, exp), ("pinned", w)
    # the other widths through both host paths
    pinned = torch.from_numpy(host).pin_memory()
    for w in (1, 2, 4, 128, 256):
        exp = orc.bytes_mt(w, host, 8)
        for src in (host, pinned):
            got = np.zeros(w, dtype=np.uint64)
            pp.pospopcnt_host(w, got, src)
            assert np.array_equal(got, exp), w
    # Fig. 2 entry points on plain host arrays
    words = host[:2 * 1000003].view("<u2")
    got = np.zeros(16, dtype=np.uint64)
    pp.pospopcnt_u16(got, words)
    assert np.array_equal(got, orc.typed(16, words))


def test_argument_errors(gpu):
    L = pp.lib()
    c = torch.zeros(64, dtype=torch.int64, device=gpu)
    d = torch.zeros(64, dtype=torch.uint8, device=gpu)
    s = None
    assert L.pospopcnt_async(16, c.data_ptr(), d.data_ptr(), 0, s) == pp.POSPOP_OK
    assert L.pospopcnt_async(16, None, d.data_ptr(), 8, s) == pp.POSPOP_EINVAL
    assert L.pospopcnt_async(16, c.data_ptr(), None, 8, s) == pp.POSPOP_EINVAL
    for bad_w in (0, 3, 12, 96, 512):
        assert L.pospopcnt_async(bad_w, c.data_ptr(), d.data_ptr(), 8, s) == pp.POSPOP_EINVAL
    host = np.zeros(64, dtype=np.uint8)
    assert L.pospopcnt_async(16, c.data_ptr(), host.ctypes.data, 8, s) == pp.POSPOP_EPTR
    hc = np.zeros(16, dtype=np.uint64)
    assert L.pospopcnt_u16(hc.ctypes.data, d.data_ptr(), 4) == pp.POSPOP_EPTR   # mixed kinds
    assert L.pospopcnt_u16(c.data_ptr(), None, 4) == pp.POSPOP_EINVAL
    assert L.pospopcnt_u16(c.data_ptr(), None, 0) == pp.POSPOP_OK
    torch.cuda.synchronize()
    assert not c.any()
    with pytest.raises(pp.PospopError):
        pp.pospopcnt_async(7, c, d)


def test_plan_and_launch_counter(gpu):
    before = pp.pospopcnt_launch_count()
    d = torch.zeros(1 << 20, dtype=torch.uint8, device=gpu)
    gpu_count(16, d)
    assert pp.pospopcnt_launch_count() == before + 1
    p = pp.pospopcnt_plan(16, 8 << 30)
    assert p["launches"] == 1 and p["depth"] in (16, 32) and p["grid"] >= 1
    assert p["rows"] == (8 << 30) // 512
    small = pp.pospopcnt_plan(16, 100)
    assert small["grid"] == 1 and small["size_class"] == 0


@pytest.mark.parametrize("w", (128, 256))
def test_wide_folds(gpu, orc, w):
    """w = 128 and 256 (Section 4's general maximum word size)."""
    rng = np.random.default_rng(w)
    sizes = [1, 15, 16, 17, 31, 32, 33, 255, 256, 257, 511, 512, 513, 4096, 100003, 3 << 20]
    sizes += [int(x) for x in rng.integers(1, 1 << 22, 10)]
    for k, n in enumerate(sizes):
        off = k % 16
        host = synth.random_bytes(n, seed=w + k)
        d = to_dev(host, gpu, align_pad=off)
        assert np.array_equal(gpu_count(w, d), orc.bytes(w, host)), (w, n, off)
    host = synth.random_bytes((5 << 20) + 77, seed=9)
    got = np.zeros(w, dtype=np.uint64)
    pp.pospopcnt_host(w, got, host)
    assert np.array_equal(got, orc.bytes(w, host))


@pytest.mark.parametrize("w", (128, 256))
def test_wide_folds_every_shape_and_row_count(gpu, orc, tune_override, w):
    host = synth.random_bytes((1 << 20) + 333, seed=5)
    for bs, minb, hint in ((512, 1, 0), (512, 1, 1), (256, 2, 1), (128, 4, 1)):
        lines = [f"stream {c} {bs} {minb} 16 {hint} 1 64" for c in range(5)]
        tune_override("\n".join(lines) + "\n")
        dd = to_dev(host, gpu, align_pad=7)
        assert np.array_equal(gpu_count(w, dd), orc.bytes(w, host)), (bs, hint)
    lines = [f"stream {c} 128 4 16 1 1 1000000" for c in range(5)]
    tune_override("\n".join(lines) + "\n")
    for k in (1, 2, 3, 4, 15, 16, 17, 31, 32, 33, 40):
        n = 4 * k * 512 - 5
        h = synth.random_bytes(n, seed=k)
        dd = to_dev(h, gpu, align_pad=k % 16)
        assert np.array_equal(gpu_count(w, dd), orc.bytes(w, h)), (k,)


def test_wide_folds_large(gpu, orc):
    n = 1 << 30
    d = torch.empty(n + 64, dtype=torch.uint8, device=gpu)
    synth_device.random_(d, 31337)
    data = d[3:3 + n - 11]
    host = data.cpu().numpy()
    for w in (128, 256):
        assert np.array_equal(gpu_count(w, data), orc.bytes_mt(w, host, 16)), w


def test_launch_split_overflow_guard(gpu, orc, tune_override):
    """The single-array count splits into several launches when a warp would
    take more rows than the counter bound allows (here lowered to 3 rows per
    warp, so a 2 MiB count needs many launches); results stay exact."""
    lines = [f"stream {c} 128 4 16 1 1 1" for c in range(5)] + ["split 3"]
    tune_override("\n".join(lines) + "\n")
    n = (2 << 20) + 4099
    plan = pp.pospopcnt_plan(64, n)
    assert plan["launches"] > 1, plan
    host = synth.random_bytes(n, seed=123)
    d = to_dev(host, gpu, align_pad=11)
    before = pp.pospopcnt_launch_count()
    for w in (8, 64, 256):
        assert np.array_equal(gpu_count(w, d), orc.bytes(w, host)), w
    assert pp.pospopcnt_launch_count() - before == 3 * plan["launches"]
    # the selected count splits the same way
    W = 4
    nw = n // W
    sel_h = synth.random_bytes((nw + 31) // 32 * 4, seed=5)
    sel = to_dev(sel_h, gpu)
    c = torch.zeros(32, dtype=torch.int64, device=gpu)
    words = to_dev(host[:nw * W], gpu, align_pad=8)
    pp.pospopcnt_masked(32, c, words, nw, sel)
    torch.cuda.synchronize()
    assert np.array_equal(counts_np(c), orc.masked(32, host[:nw * W], nw, sel_h))


def test_regroup_short_path_single(gpu, orc, tune_override):
    """Single arrays whose warps get at most 3 rows, w = 8, through the
    per-lane bit regroup (tune entry `short 1`)."""
    lines = [f"stream {c} 128 4 16 1 1 {mr}" for c, mr in zip(range(5), (1, 2, 3, 3, 3))]
    tune_override("\n".join(lines) + "\nshort 1\n")
    for n in (1, 5, 16, 17, 511, 512, 513, 4 * 512 * 3 - 7, 4 * 512 * 3, 100003):
        for off in (0, 7, 15):
            host = synth.random_bytes(n, seed=n + off)
            d = to_dev(host, gpu, align_pad=off)
            for w in (8, 16):
                assert np.array_equal(gpu_count(w, d), orc.bytes(w, host)), (n, off, w)
