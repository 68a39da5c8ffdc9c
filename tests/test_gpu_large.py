"""Large arrays at full size (1 GiB and 8 GiB) vs the CPU oracle, bit-exact.

The large-array sweep: w = 8, 16, 32, 64 over arrays of Bernoulli(p) bits,
p in {0.01, 0.5, 0.99}, plus an all-ones array, made on the device by the
generator twin and counted with the same library call the benchmark times.
The oracle counts the host copy of each array (word-aligned chunks, all host
cores).  All-ones arrays are also checked against the closed form, and
counted repeatedly into the same counters until every counter passes 2**32.
"""
import numpy as np
import pytest
import torch

from paper_2412_16370_gb300 import binding as pp
from paper_2412_16370_gb300 import synth, synth_device

from _gpu import WORD_W, counts_np, gpu_count, oracle_device_bytes

pytestmark = pytest.mark.gpu

GIB = 1 << 30


@pytest.fixture(scope="module")
def big(gpu):
    t = torch.empty(8 * GIB, dtype=torch.uint8, device=gpu)
    yield t
    del t
    torch.cuda.empty_cache()


@pytest.mark.parametrize("size", (GIB, 8 * GIB), ids=("1GiB", "8GiB"))
@pytest.mark.parametrize("p", (0.01, 0.5, 0.99))
def test_bernoulli(gpu, orc, big, size, p):
    seed = 1000 + int(p * 100)
    data = big[:size]
    synth_device.bernoulli_(data, p, seed)
    # the device bytes are the recipe's bytes (sampled windows)
    for s0 in (0, size // 3 + 5, size - 1000):
        win = data[s0:s0 + 1000].cpu().numpy()
        assert np.array_equal(win, synth.bernoulli_bytes(win.size, p, seed, start=s0))
    got = {w: gpu_count(w, data) for w in WORD_W}
    exp = oracle_device_bytes(orc, WORD_W, data)
    for w in WORD_W:
        assert np.array_equal(got[w], exp[w]), (size, p, w)


@pytest.mark.parametrize("size", (GIB, 8 * GIB), ids=("1GiB", "8GiB"))
def test_all_ones_closed_form_and_overflow(gpu, orc, big, size):
    data = big[:size]
    synth_device.fill_(data, 0xFF)
    for w in WORD_W:
        per = size * 8 // w
        assert np.array_equal(gpu_count(w, data), np.full(w, per, dtype=np.uint64))
        # add-into: repeat until every counter exceeds 2**32
        reps = (1 << 32) // per + 1
        c = torch.zeros(w, dtype=torch.int64, device=gpu)
        for _ in range(reps):
            pp.pospopcnt_async(w, c, data)
        torch.cuda.synchronize()
        got = counts_np(c)
        assert np.array_equal(got, np.full(w, reps * per, dtype=np.uint64))
        assert int(got.min()) > (1 << 32)
    if size == GIB:
        exp = oracle_device_bytes(orc, WORD_W, data)
        for w in WORD_W:
            assert np.array_equal(exp[w], np.full(w, size * 8 // w, dtype=np.uint64))


def test_unaligned_large(gpu, orc, big):
    """1 GiB minus a few bytes, starting 13 bytes past a 16-byte boundary."""
    synth_device.random_(big[:GIB + 64], 555)
    data = big[13:13 + GIB - 29]
    got = {w: gpu_count(w, data) for w in WORD_W}
    exp = oracle_device_bytes(orc, WORD_W, data)
    for w in WORD_W:
        assert np.array_equal(got[w], exp[w]), w
