"""Guard words around the counters: no entry point writes outside its
counter array (the sanitizer substitute, since compute-sanitizer is not
available).  Each call's counters sit between two guard regions filled with
a sentinel; after the call the guards are intact and the counts match the
oracle."""
import numpy as np
import pytest
import torch

from paper_2412_16370_gb300 import binding as pp
from paper_2412_16370_gb300 import synth

from _gpu import counts_np

pytestmark = pytest.mark.gpu

SENTINEL = 0x5A5A5A5A5A5A5A5A
GUARD = 512   # 64-bit words on each side


def _guarded(n, gpu):
    buf = torch.full((GUARD + n + GUARD,), SENTINEL, dtype=torch.int64, device=gpu)
    inner = buf[GUARD:GUARD + n]
    inner.zero_()
    return buf, inner


def _guards_ok(buf, n):
    h = buf.cpu().numpy().view(np.uint64)
    return bool((h[:GUARD] == SENTINEL).all() and (h[GUARD + n:] == SENTINEL).all())


@pytest.mark.parametrize("w", (1, 8, 16, 64, 128, 256))
def test_single_array_and_host_forms(gpu, orc, w):
    host = synth.random_bytes((9 << 20) + 13, seed=71)
    data = torch.from_numpy(host).to(gpu)
    exp = orc.bytes(w, host[3:])
    buf, c = _guarded(w, gpu)
    pp.pospopcnt_async(w, c, data[3:])
    torch.cuda.synchronize()
    assert _guards_ok(buf, w) and np.array_equal(counts_np(c), exp)
    hbuf = np.full(GUARD + w + GUARD, SENTINEL, dtype=np.uint64)
    hbuf[GUARD:GUARD + w] = 0
    pp.pospopcnt_host(w, hbuf[GUARD:GUARD + w], host[3:])
    assert (hbuf[:GUARD] == SENTINEL).all() and (hbuf[GUARD + w:] == SENTINEL).all()
    assert np.array_equal(hbuf[GUARD:GUARD + w], exp)


@pytest.mark.parametrize("w", (8, 32, 256))
def test_batch_gather_masked_forms(gpu, orc, w):
    sizes = synth.log_uniform_sizes(1000, 1, 300000, seed=72)
    sizes[::11] = 0
    offs = synth.csr_offsets(sizes)
    host = synth.random_bytes(int(offs[-1]) + 64, seed=73)
    base = torch.from_numpy(host).to(gpu)
    m = len(sizes)
    buf, c = _guarded(m * w, gpu)
    pp.pospopcnt_batch(w, c, base, torch.from_numpy(offs.view(np.int64)).to(gpu), m)
    torch.cuda.synchronize()
    assert _guards_ok(buf, m * w)
    assert np.array_equal(counts_np(c).reshape(m, w), orc.batch(w, host[:int(offs[-1])], offs))
    starts = offs[:-1].astype(np.int64) + 1
    ptrs = torch.from_numpy(base.data_ptr() + starts).to(gpu)
    lens = torch.from_numpy(sizes.astype(np.int64)).to(gpu)
    buf, c = _guarded(w, gpu)
    pp.pospopcnt_gather(w, c, ptrs, lens, m)
    torch.cuda.synchronize()
    assert _guards_ok(buf, w)
    regions = [host[a:a + b] for a, b in zip(starts, sizes)]
    assert np.array_equal(counts_np(c), orc.gather(w, regions))
    if w <= 64:
        W = w // 8
        n = (48 << 20) // W + 7       # two 16-row chunks per warp of every staged shape
        words_h = synth.random_bytes(n * W, seed=74)
        sel_h = synth.random_bytes(4 * ((n + 31) // 32), seed=75)
        words = torch.from_numpy(words_h).to(gpu)
        sel = torch.from_numpy(sel_h).to(gpu)
        for nn in (n, 1000):          # staged and register forms
            buf, c = _guarded(w, gpu)
            pp.pospopcnt_masked(w, c, words, nn, sel)
            torch.cuda.synchronize()
            assert _guards_ok(buf, w)
            assert np.array_equal(counts_np(c), orc.masked(w, words_h[:nn * W], nn, sel_h)), nn
