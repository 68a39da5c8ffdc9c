"""Batched pospopcnt (CSR offsets, one persistent launch) vs the CPU oracle.

The ragged one-hot workload: uint8 arrays, each byte with exactly one of 8
bits set (Zipf(1.1) categories), sizes log-uniform on 1 B .. 4 MiB,
concatenated back to back (so starts are unaligned).  A 20000-array subset
(every w) and the full 200000-array batch (about 55 GB; w = 8 and 16) are
checked against the oracle on every array.  Also: every kernel variant and
work-item size, zero-length arrays, decreasing offsets, and CUDA-graph
replay, including a graph's own workspace outliving later calls.
"""
import numpy as np
import pytest
import torch

from paper_2412_16370_gb300 import binding as pp
from paper_2412_16370_gb300 import synth, synth_device

from _gpu import WORD_W, counts_np, oracle_batch_device, oracle_batch_parallel

pytestmark = pytest.mark.gpu

ONE_HOT_SEED = 4
SIZE_SEED = 3


def _one_hot_batch(dev, m):
    sizes = synth.log_uniform_sizes(m, 1, 4 << 20, seed=SIZE_SEED)
    offs = synth.csr_offsets(sizes)
    total = int(offs[-1])
    base = torch.empty(total + 64, dtype=torch.uint8, device=dev)
    synth_device.one_hot_(base, ONE_HOT_SEED, nbytes=total)
    offs_d = torch.from_numpy(offs.view(np.int64)).to(dev)
    return sizes, offs, base, offs_d


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


def test_subset_every_array_exact(gpu, orc):
    m = 20000
    sizes, offs, base, offs_d = _one_hot_batch(gpu, m)
    host = base[:int(offs[-1])].cpu().numpy()
    # the device generator made exactly the numpy recipe's bytes (sampled windows)
    for s0 in (0, 12345, int(offs[-1]) - 4096):
        assert np.array_equal(host[s0:s0 + 4096], synth.one_hot_bytes(4096, ONE_HOT_SEED, start=s0))
    for w in WORD_W:
        counts = torch.zeros((m, w), dtype=torch.int64, device=gpu)
        pp.pospopcnt_batch(w, counts, base, offs_d, m)
        assert pp.pospopcnt_batch_status() == pp.POSPOP_OK
        got = counts_np(counts)
        exp = oracle_batch_parallel(orc, w, host, offs)
        bad = np.nonzero((got != exp).any(axis=1))[0]
        assert bad.size == 0, (w, bad[:5].tolist())
        if w == 8:
            assert np.array_equal(got.sum(axis=1), sizes.astype(np.uint64))


def test_full_batch_every_array_exact(gpu, orc):
    """The stated workload at full size: all 200000 arrays (about 55 GB),
    every array compared with the oracle at w = 8 and w = 16."""
    m = 200000
    sizes, offs, base, offs_d = _one_hot_batch(gpu, m)
    got = {}
    for w in (8, 16):
        counts = torch.zeros((m, w), dtype=torch.int64, device=gpu)
        pp.pospopcnt_batch(w, counts, base, offs_d, m)
        assert pp.pospopcnt_batch_status() == pp.POSPOP_OK
        got[w] = counts_np(counts)
        del counts
    exp = oracle_batch_device(orc, (8, 16), base, offs)
    for w in (8, 16):
        bad = np.nonzero((got[w] != exp[w]).any(axis=1))[0]
        assert bad.size == 0, (w, bad.size, bad[:5].tolist())
        # every byte has exactly one bit set: an array's counts add up to its length
        assert np.array_equal(got[w].sum(axis=1), sizes.astype(np.uint64)), w
    # the device generator made the recipe's bytes (sampled windows)
    total = int(offs[-1])
    for s0 in (0, total // 2 + 7, total - 4096):
        win = base[s0:s0 + 4096].cpu().numpy()
        assert np.array_equal(win, synth.one_hot_bytes(4096, ONE_HOT_SEED, start=s0))


def test_every_variant_and_item_size(gpu, orc, tune_override):
    sizes = synth.log_uniform_sizes(700, 1, 300000, seed=77)
    sizes[::37] = 0   # zero-length arrays in between
    offs = synth.csr_offsets(sizes)
    host = synth.random_bytes(int(offs[-1]), seed=78)
    base = torch.empty(host.size + 32, dtype=torch.uint8, device=gpu)[5:5 + host.size]
    base.copy_(torch.from_numpy(host))
    offs_d = torch.from_numpy(offs.view(np.int64)).to(gpu)
    exp = {w: orc.batch(w, host, offs) for w in WORD_W}
    for bs, minb in ((256, 2), (512, 1), (128, 4)):
        for depth in (16, 32):
            for hint in (0, 1):
                for item_rows, grab in ((1, 1), (3, 2), (15, 1), (31, 3), (47, 1), (511, 4)):
                    tune_override(f"batch {bs} {minb} {depth} {hint} 1 {item_rows} {grab}\n")
                    for w in WORD_W:
                        c = torch.zeros((len(sizes), w), dtype=torch.int64, device=gpu)
                        pp.pospopcnt_batch(w, c, base, offs_d)
                        assert pp.pospopcnt_batch_status() == pp.POSPOP_OK
                        assert np.array_equal(counts_np(c), exp[w]), (bs, depth, hint, item_rows, w)


def test_per_class_item_rows(gpu, orc, tune_override):
    """Work-item rows per array size class (tune entry batch_rows): arrays of
    every class (up to 2 KiB, 32 KiB, 1 MiB, above) in one batch, each class
    with its own item size, bit-exact for several tables and widths."""
    sizes = np.concatenate([synth.log_uniform_sizes(400, 1, 2048, seed=41),
                            synth.log_uniform_sizes(300, 2049, 32768, seed=42),
                            synth.log_uniform_sizes(100, 32769, 1 << 20, seed=43),
                            synth.log_uniform_sizes(12, (1 << 20) + 1, 6 << 20, seed=44)])
    rng = np.random.default_rng(45)
    sizes = sizes[rng.permutation(sizes.size)]
    sizes[::53] = 0
    offs = synth.csr_offsets(sizes)
    host = synth.random_bytes(int(offs[-1]), seed=46)
    base = torch.empty(host.size + 32, dtype=torch.uint8, device=gpu)[9:9 + host.size]
    base.copy_(torch.from_numpy(host))
    offs_d = torch.from_numpy(offs.view(np.int64)).to(gpu)
    exp = {w: orc.batch(w, host, offs) for w in (8, 32, 256)}
    for rows in ("1 2 3 4", "4 64 2048 4095", "2 7 100 1000", "3 31 255 63"):
        tune_override(f"batch 512 1 16 1 1 127 2\nbatch_rows {rows}\n")
        assert f"batch_rows {rows}" in pp.pospopcnt_tune_describe()
        for w in (8, 32, 256):
            c = torch.zeros((len(sizes), w), dtype=torch.int64, device=gpu)
            pp.pospopcnt_batch(w, c, base, offs_d)
            assert pp.pospopcnt_batch_status() == pp.POSPOP_OK
            assert np.array_equal(counts_np(c), exp[w]), (rows, w)


def test_short_sweep_back_to_back(gpu, orc):
    """The short/unaligned sweep's arrays laid back to back in one batch."""
    for w in WORD_W:
        lens = synth.short_sweep_lengths()
        arrays = [synth.random_bytes(n, synth.case_seed(w, n, off))
                  for n in lens for off in (0, 7, 15)]
        sizes = np.array([a.size for a in arrays], dtype=np.int64)
        offs = synth.csr_offsets(sizes)
        host = np.concatenate(arrays)
        base = torch.from_numpy(host).to(gpu)
        c = torch.zeros((len(arrays), w), dtype=torch.int64, device=gpu)
        pp.pospopcnt_batch(w, c, base, torch.from_numpy(offs.view(np.int64)).to(gpu))
        assert np.array_equal(counts_np(c), orc.batch(w, host, offs)), w


def test_sub_byte_and_wide_widths(gpu, orc):
    sizes = synth.log_uniform_sizes(500, 1, 100000, seed=5)
    offs = synth.csr_offsets(sizes)
    host = synth.random_bytes(int(offs[-1]), seed=6)
    base = torch.from_numpy(host).to(gpu)
    offs_d = torch.from_numpy(offs.view(np.int64)).to(gpu)
    for w in (1, 2, 4, 128, 256):
        c = torch.zeros((len(sizes), w), dtype=torch.int64, device=gpu)
        pp.pospopcnt_batch(w, c, base, offs_d)
        assert np.array_equal(counts_np(c), orc.batch(w, host, offs)), w


def test_decreasing_offsets_rejected(gpu):
    offs = np.array([0, 10, 30, 20, 40], dtype=np.int64)
    base = torch.ones(64, dtype=torch.uint8, device=gpu)
    c = torch.full((4, 8), 7, dtype=torch.int64, device=gpu)
    pp.pospopcnt_batch(8, c, base, torch.from_numpy(offs).to(gpu))
    assert pp.pospopcnt_batch_status() == pp.POSPOP_EINVAL
    assert (c == 7).all()
    # the status is cleared once read, and a good batch afterwards works
    offs[3] = 30
    pp.pospopcnt_batch(8, c, base, torch.from_numpy(offs).to(gpu))
    assert pp.pospopcnt_batch_status() == pp.POSPOP_OK
    assert c.sum().item() == 4 * 8 * 7 + 40


def test_graph_replay_matches_direct(gpu, orc):
    sizes = synth.log_uniform_sizes(3000, 1, 1 << 20, seed=12)
    offs = synth.csr_offsets(sizes)
    host = synth.random_bytes(int(offs[-1]), seed=13)
    base = torch.from_numpy(host).to(gpu)
    offs_d = torch.from_numpy(offs.view(np.int64)).to(gpu)
    exp = orc.batch(32, host, offs)
    s = torch.cuda.Stream()
    c = torch.zeros((len(sizes), 32), dtype=torch.int64, device=gpu)
    g = pp.pospopcnt_batch_graph_create(32, c, base, offs_d, stream=s)
    try:
        s.synchronize()
        c.zero_()
        torch.cuda.synchronize()
        for _ in range(3):
            pp.pospopcnt_graph_launch(g, s)
        s.synchronize()
        assert np.array_equal(counts_np(c), 3 * exp)
    finally:
        pp.pospopcnt_graph_destroy(g)


def test_graph_owns_its_workspace(gpu, orc):
    """A graph made by pospopcnt_batch_graph_create keeps its own scratch:
    a later, larger batch on the capture stream (which replaces that
    stream's workspace) and a shutdown of the library leave it valid."""
    m = 2000
    sizes = synth.log_uniform_sizes(m, 1, 1 << 18, seed=14)
    sizes[::97] = 0
    offs = synth.csr_offsets(sizes)
    host = synth.random_bytes(int(offs[-1]) + 7, seed=15)
    dbuf = torch.from_numpy(host).to(gpu)
    base = dbuf[7:]
    offs_d = torch.from_numpy(offs.view(np.int64)).to(gpu)
    exp = orc.batch(16, host[7:], offs)
    s = torch.cuda.Stream()
    c = torch.zeros((m, 16), dtype=torch.int64, device=gpu)
    pp.pospopcnt_batch(16, c, base, offs_d, m, s)   # the stream's own workspace exists
    s.synchronize()
    g = pp.pospopcnt_batch_graph_create(16, c, base, offs_d, stream=s)
    try:
        addr0, size0 = pp.pospopcnt_graph_workspace(g)
        assert addr0 != 0 and size0 >= 8 * (m + 1)
        s.synchronize()
        c.zero_()
        torch.cuda.synchronize()
        # a batch with many more arrays on the same stream grows (replaces)
        # the stream's workspace
        big_m = 300000
        bsz = synth.log_uniform_sizes(big_m, 1, 64, seed=16)
        boffs = synth.csr_offsets(bsz)
        bbase = torch.zeros(int(boffs[-1]) + 16, dtype=torch.uint8, device=gpu)
        bc = torch.zeros((big_m, 8), dtype=torch.int64, device=gpu)
        pp.pospopcnt_batch(8, bc, bbase, torch.from_numpy(boffs.view(np.int64)).to(gpu), big_m, s)
        assert pp.pospopcnt_batch_status(s) == pp.POSPOP_OK
        pp.pospopcnt_graph_launch(g, s)
        s.synchronize()   # replays of one graph must not overlap
        pp.pospopcnt_graph_launch(g, torch.cuda.current_stream())   # any stream
        assert pp.pospopcnt_graph_status(g) == pp.POSPOP_OK
        # and a shutdown of the library (which frees every stream workspace)
        pp.shutdown()
        pp.init(0)
        pp.pospopcnt_graph_launch(g, s)
        assert pp.pospopcnt_graph_status(g) == pp.POSPOP_OK
        torch.cuda.synchronize()
        assert np.array_equal(counts_np(c), 3 * exp)
        assert pp.pospopcnt_graph_workspace(g) == (addr0, size0)
    finally:
        pp.pospopcnt_graph_destroy(g)


def test_graph_reports_decreasing_offsets(gpu):
    offs = torch.tensor([0, 10, 30, 20, 40], dtype=torch.int64, device=gpu)
    base = torch.ones(64, dtype=torch.uint8, device=gpu)
    c = torch.full((4, 8), 7, dtype=torch.int64, device=gpu)
    s = torch.cuda.Stream()
    g = pp.pospopcnt_batch_graph_create(8, c, base, offs, 4, s)
    try:
        pp.pospopcnt_graph_launch(g, s)
        assert pp.pospopcnt_graph_status(g) == pp.POSPOP_EINVAL
        assert (c == 7).all()
        assert pp.pospopcnt_graph_status(g) == pp.POSPOP_OK   # cleared once read
        offs[3] = 30
        pp.pospopcnt_graph_launch(g, s)
        assert pp.pospopcnt_graph_status(g) == pp.POSPOP_OK
        torch.cuda.synchronize()
        assert c.sum().item() == 4 * 8 * 7 + 40
    finally:
        pp.pospopcnt_graph_destroy(g)


def test_argument_errors(gpu):
    L = pp.lib()
    c = torch.zeros(64, dtype=torch.int64, device=gpu)
    base = torch.zeros(64, dtype=torch.uint8, device=gpu)
    offs = torch.zeros(3, dtype=torch.int64, device=gpu)
    assert L.pospopcnt_batch(8, c.data_ptr(), base.data_ptr(), offs.data_ptr(), 0, None) == 0
    assert L.pospopcnt_batch(8, None, base.data_ptr(), offs.data_ptr(), 2, None) == pp.POSPOP_EINVAL
    assert L.pospopcnt_batch(9, c.data_ptr(), base.data_ptr(), offs.data_ptr(), 2, None) == pp.POSPOP_EINVAL
    assert L.pospopcnt_batch(512, c.data_ptr(), base.data_ptr(), offs.data_ptr(), 2, None) == pp.POSPOP_EINVAL
    hoffs = np.zeros(3, dtype=np.uint64)
    assert L.pospopcnt_batch(8, c.data_ptr(), base.data_ptr(), hoffs.ctypes.data, 2, None) == pp.POSPOP_EPTR


@pytest.mark.parametrize("item_rows", (1, 2, 3, 127))
def test_regroup_short_path(gpu, orc, tune_override, item_rows):
    """w = 8 work items of at most 3 rows through the per-lane bit regroup
    (tune entry `short 1`), bit-exact; other widths keep the transpose flush."""
    sizes = synth.log_uniform_sizes(3000, 1, 5000, seed=91)
    sizes[::29] = 0
    offs = synth.csr_offsets(sizes)
    host = synth.random_bytes(int(offs[-1]), seed=92)
    base = torch.empty(host.size + 32, dtype=torch.uint8, device=gpu)[3:3 + host.size]
    base.copy_(torch.from_numpy(host))
    offs_d = torch.from_numpy(offs.view(np.int64)).to(gpu)
    tune_override(f"batch 512 1 16 1 1 {item_rows} 1\nshort 1\n")
    assert "short 1" in pp.pospopcnt_tune_describe()
    for w in (8, 16):
        c = torch.zeros((len(sizes), w), dtype=torch.int64, device=gpu)
        pp.pospopcnt_batch(w, c, base, offs_d)
        assert np.array_equal(counts_np(c), orc.batch(w, host, offs)), (w, item_rows)
    # one-hot bytes: each array's class histogram
    oh = synth.one_hot_bytes(int(offs[-1]), 93)
    base.copy_(torch.from_numpy(oh))
    c = torch.zeros((len(sizes), 8), dtype=torch.int64, device=gpu)
    pp.pospopcnt_batch(8, c, base, offs_d)
    got = counts_np(c)
    assert np.array_equal(got, orc.batch(8, oh, offs))
    assert np.array_equal(got.sum(axis=1), sizes.astype(np.uint64))


def test_w256_every_tune_shape(gpu, orc, tune_override):
    """w = 256 (a word spans two granules) through the two-parity batch kernel,
    for every block shape and item size the tune table may choose."""
    sizes = synth.log_uniform_sizes(300, 1, 200000, seed=55)
    sizes[::23] = 0
    offs = synth.csr_offsets(sizes)
    host = synth.random_bytes(int(offs[-1]), seed=56)
    base = torch.empty(host.size + 32, dtype=torch.uint8, device=gpu)[3:3 + host.size]
    base.copy_(torch.from_numpy(host))
    offs_d = torch.from_numpy(offs.view(np.int64)).to(gpu)
    exp = orc.batch(256, host, offs)
    for bs, minb in ((256, 2), (512, 1), (128, 4)):
        for depth in (16, 32):
            for hint in (0, 1):
                for item_rows in (1, 31, 127):
                    tune_override(f"batch {bs} {minb} {depth} {hint} 1 {item_rows} 1\n")
                    c = torch.zeros((len(sizes), 256), dtype=torch.int64, device=gpu)
                    pp.pospopcnt_batch(256, c, base, offs_d)
                    assert np.array_equal(counts_np(c), exp), (bs, depth, hint, item_rows)
