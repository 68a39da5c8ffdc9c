"""Programmatic dependent launch (tune entry `pdl 1`) keeps stream order.

With the entry set, every counting and planning kernel is launched so that
it may be scheduled while the previous kernel on the stream still runs; each
kernel waits for its predecessor before touching memory.  These tests put a
producer kernel (the input generator, launched plainly) directly before the
counting kernels on one stream, chain the library's own kernels (the batch
call is four kernels), and check every result against the CPU oracle, with
the entry on and off.
"""
import numpy as np
import pytest
import torch

from paper_2412_16370_gb300 import binding as pp
from paper_2412_16370_gb300 import synth, synth_device

from _gpu import WORD_W, counts_np

pytestmark = pytest.mark.gpu


@pytest.fixture
def tune_with(gpu, tmp_path):
    saved = tmp_path / "saved_tune.txt"
    saved.write_text(pp.pospopcnt_tune_describe())
    base = "\n".join(l for l in saved.read_text().splitlines() if not l.startswith("pdl"))

    def install(pdl):
        f = tmp_path / "tune.txt"
        f.write_text(base + f"\npdl {pdl}\n")
        pp.pospopcnt_tune_load(str(f))
        assert f"pdl {pdl}" in pp.pospopcnt_tune_describe()

    yield install
    pp.pospopcnt_tune_load(str(saved))


@pytest.mark.parametrize("pdl", (0, 1))
def test_producer_then_counts_on_one_stream(gpu, orc, tune_with, pdl):
    tune_with(pdl)
    s = torch.cuda.Stream()
    n_big, n_small = (16 << 20) + 5, 777
    buf = torch.empty(n_big + 64, dtype=torch.uint8, device=gpu)
    outs = []
    with torch.cuda.stream(s):
        for k in range(6):
            w = WORD_W[k % 4]
            # the generator overwrites the buffer right before each count
            synth_device.random_(buf, 300 + k, stream=s)
            c = torch.zeros(w, dtype=torch.int64, device=gpu)
            pp.pospopcnt_async(w, c, buf[3:3 + n_big], n_big, s)
            pp.pospopcnt_async(w, c, buf[3:3 + n_big], n_big, s)
            cs = torch.zeros(w, dtype=torch.int64, device=gpu)
            pp.pospopcnt_async(w, cs, buf[9:9 + n_small], n_small, s)
            outs.append((k, w, c, cs))
    s.synchronize()
    for k, w, c, cs in outs:
        host = synth.random_bytes(n_big + 64, seed=300 + k)
        assert np.array_equal(counts_np(c), 2 * orc.bytes(w, host[3:3 + n_big])), (pdl, k)
        assert np.array_equal(counts_np(cs), orc.bytes(w, host[9:9 + n_small])), (pdl, k)


@pytest.mark.parametrize("pdl", (0, 1))
def test_batch_gather_masked_chains(gpu, orc, tune_with, pdl):
    tune_with(pdl)
    s = torch.cuda.Stream()
    sizes = synth.log_uniform_sizes(2000, 1, 100000, seed=41)
    sizes[::17] = 0
    offs = synth.csr_offsets(sizes)
    total = int(offs[-1])
    buf = torch.empty(total + 64, dtype=torch.uint8, device=gpu)
    offs_d = torch.from_numpy(offs.view(np.int64)).to(gpu)
    starts = offs[:-1].astype(np.int64) + 1
    lens = sizes.astype(np.int64)
    ptrs_d = torch.from_numpy(buf.data_ptr() + starts).to(gpu)
    lens_d = torch.from_numpy(lens).to(gpu)
    n_words = total // 4
    sel = torch.empty((n_words + 7) // 8 + 8, dtype=torch.uint8, device=gpu)
    res = []
    with torch.cuda.stream(s):
        for k in range(3):
            synth_device.random_(buf, 500 + k, stream=s)
            synth_device.random_(sel, 600 + k, stream=s)
            cb = torch.zeros((len(sizes), 8), dtype=torch.int64, device=gpu)
            pp.pospopcnt_batch(8, cb, buf, offs_d, len(sizes), s)
            cg = torch.zeros(16, dtype=torch.int64, device=gpu)
            pp.pospopcnt_gather(16, cg, ptrs_d, lens_d, len(sizes), s)
            cm = torch.zeros(32, dtype=torch.int64, device=gpu)
            pp.pospopcnt_masked(32, cm, buf, n_words, sel, s)
            res.append((k, cb, cg, cm))
    s.synchronize()
    assert pp.pospopcnt_batch_status(s) == pp.POSPOP_OK
    for k, cb, cg, cm in res:
        host = synth.random_bytes(total + 64, seed=500 + k)
        selh = synth.random_bytes(sel.numel(), seed=600 + k)
        assert np.array_equal(counts_np(cb), orc.batch(8, host[:total], offs)), (pdl, k)
        regions = [host[a:a + b] for a, b in zip(starts, lens)]
        assert np.array_equal(counts_np(cg), orc.gather(16, regions)), (pdl, k)
        assert np.array_equal(counts_np(cm), orc.masked(32, host[:4 * n_words], n_words, selh)), (pdl, k)


def test_graph_capture_with_pdl(gpu, orc, tune_with):
    tune_with(1)
    sizes = synth.log_uniform_sizes(500, 1, 200000, seed=8)
    offs = synth.csr_offsets(sizes)
    host = synth.random_bytes(int(offs[-1]), seed=9)
    base = torch.from_numpy(host).to(gpu)
    offs_d = torch.from_numpy(offs.view(np.int64)).to(gpu)
    s = torch.cuda.Stream()
    c = torch.zeros((len(sizes), 16), dtype=torch.int64, device=gpu)
    g = pp.pospopcnt_batch_graph_create(16, c, base, offs_d, stream=s)
    try:
        s.synchronize()
        c.zero_()
        torch.cuda.synchronize()
        for _ in range(4):
            pp.pospopcnt_graph_launch(g, s)
        s.synchronize()
        assert np.array_equal(counts_np(c), 4 * orc.batch(16, host, offs))
    finally:
        pp.pospopcnt_graph_destroy(g)
