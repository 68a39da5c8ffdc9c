"""Several independent counts in one launch (pospopcnt_multi) vs the oracle.

Each count is the byte-length count of its own span, width and counters;
the group is planned on the host and counted in one launch per 256 counts.
Checked bit for bit against the CPU oracle: mixed widths 1..64, sizes from
empty to several MiB, unaligned starts, more than 256 counts (several
launches), counters that alias (counts into one counter array add up), the
add-into semantics, and argument errors (nothing is counted).
"""
import numpy as np
import pytest
import torch

from paper_2412_16370_gb300 import binding as pp
from paper_2412_16370_gb300 import synth, synth_device

from _gpu import counts_np, oracle_device_bytes

pytestmark = pytest.mark.gpu

WIDTHS = (1, 2, 4, 8, 16, 32, 64)


@pytest.fixture(scope="module")
def pool(gpu):
    n = 64 << 20
    t = torch.empty(n + 64, dtype=torch.uint8, device=gpu)
    synth_device.random_(t, 777)
    torch.cuda.synchronize()
    return t, t.cpu().numpy()


@pytest.mark.parametrize("n,hi", [(1, 1 << 20), (37, 3 << 20), (300, 200000), (700, 5000)])
def test_mixed_group_matches_oracle(gpu, orc, pool, n, hi):
    dev, host = pool
    rng = np.random.default_rng(n)
    sizes = synth.log_uniform_sizes(n, 1, hi, seed=n + 1)
    sizes[::17] = 0
    starts = rng.integers(0, dev.numel() - 64 - hi, n)
    w = np.array(WIDTHS)[rng.integers(0, len(WIDTHS), n)]
    c = torch.zeros((n, 64), dtype=torch.int64, device=gpu)
    c[:, :] = 5                                  # counts are added into
    pp.pospopcnt_multi(w.tolist(), [c[i] for i in range(n)],
                       [dev.data_ptr() + int(s) for s in starts], sizes.tolist())
    got = counts_np(c)
    for i in range(n):
        seg = host[int(starts[i]):int(starts[i]) + int(sizes[i])]
        exp = orc.bytes(int(w[i]), seg) + np.uint64(5)
        assert np.array_equal(got[i, :w[i]], exp), (i, int(w[i]), int(sizes[i]))
        assert (got[i, w[i]:] == 5).all()


def test_aliased_counters_add_up(gpu, orc, pool):
    """Pieces of one array counted into one counter array: the whole's count
    (pieces start on 64-byte boundaries from the start, so on word boundaries)."""
    dev, host = pool
    start, total = 11, (5 << 20) + 333
    cuts = [0, 64, 4096, 1 << 20, (3 << 20) + 128, total]
    for w in (8, 64):
        c = torch.zeros(w, dtype=torch.int64, device=gpu)
        pp.pospopcnt_multi([w] * (len(cuts) - 1), [c] * (len(cuts) - 1),
                           [dev.data_ptr() + start + a for a in cuts[:-1]],
                           [b - a for a, b in zip(cuts[:-1], cuts[1:])])
        assert np.array_equal(counts_np(c), orc.bytes(w, host[start:start + total])), w


def test_large_group_in_whole_waves(gpu, orc, pool):
    dev, host = pool
    n = 4
    span = 16 << 20
    w = [8, 16, 32, 64]
    c = torch.zeros((n, 64), dtype=torch.int64, device=gpu)
    pp.pospopcnt_multi(w, [c[i] for i in range(n)],
                       [dev.data_ptr() + 3 + i * span for i in range(n)], [span] * n)
    got = counts_np(c)
    for i in range(n):
        seg = host[3 + i * span:3 + (i + 1) * span]
        assert np.array_equal(got[i, :w[i]], orc.bytes(w[i], seg)), i


def test_large_counts_grid_stride(gpu, orc):
    """A group of large counts (the grid-stride form: four 512 MiB counts,
    unaligned starts, widths 8..64) with two tiny counts and an empty one in
    it: every count equals the oracle's."""
    span = 512 << 20
    buf = torch.empty(4 * span + 4096, dtype=torch.uint8, device=gpu)
    synth_device.random_(buf, 779)
    w = [8, 16, 32, 64, 16, 8, 32]
    starts = [3 + i * span for i in range(4)] + [4 * span + 5, 4 * span + 100, 0]
    sizes = [span] * 4 + [1, 777, 0]
    c = torch.zeros((7, 64), dtype=torch.int64, device=gpu)
    pp.pospopcnt_multi(w, [c[i] for i in range(7)], [buf.data_ptr() + a for a in starts], sizes)
    got = counts_np(c)
    for i in range(7):
        exp = (oracle_device_bytes(orc, (w[i],), buf[starts[i]:starts[i] + sizes[i]])[w[i]]
               if sizes[i] else np.zeros(w[i], dtype=np.uint64))
        assert np.array_equal(got[i, :w[i]], exp), i


def test_group_larger_than_l2(gpu, orc):
    """Four 96 MiB counts (384 MiB, well past the 129 MB L2) in one launch,
    unaligned starts, widths 8..64: each equals the oracle's count."""
    span = 96 << 20
    buf = torch.empty(4 * span + 64, dtype=torch.uint8, device=gpu)
    synth_device.random_(buf, 778)
    w = [8, 16, 32, 64]
    c = torch.zeros((4, 64), dtype=torch.int64, device=gpu)
    pp.pospopcnt_multi(w, [c[i] for i in range(4)],
                       [buf.data_ptr() + 7 + i * span for i in range(4)], [span] * 4)
    got = counts_np(c)
    exp = {i: oracle_device_bytes(orc, (w[i],), buf[7 + i * span:7 + (i + 1) * span])[w[i]]
           for i in range(4)}
    for i in range(4):
        assert np.array_equal(got[i, :w[i]], exp[i]), i


def test_errors_count_nothing(gpu, orc, pool):
    dev, host_pool = pool
    L = pp.lib()
    c = torch.zeros((2, 64), dtype=torch.int64, device=gpu)
    host = np.zeros(16, dtype=np.uint8)
    import ctypes

    def call(ws, cs, ps, ns):
        n = len(ws)
        W = (ctypes.c_int * n)(*ws)
        C = (ctypes.c_uint64 * n)(*cs)
        P = (ctypes.c_uint64 * n)(*ps)
        N = (ctypes.c_size_t * n)(*ns)
        return L.pospopcnt_multi(n, W, C, P, N, None)

    good = (c[0].data_ptr(), dev.data_ptr(), 1000)
    assert call([8, 12], [good[0], c[1].data_ptr()], [good[1], good[1]], [1000, 10]) == pp.POSPOP_EINVAL
    assert call([8, 8], [good[0], c[1].data_ptr()], [good[1], host.ctypes.data], [1000, 10]) == pp.POSPOP_EPTR
    assert call([8, 8], [good[0], 0], [good[1], good[1]], [1000, 10]) == pp.POSPOP_EINVAL
    assert call([8, 8], [good[0], 0], [good[1], 0], [1000, 0]) == pp.POSPOP_OK   # empty: skipped
    assert L.pospopcnt_multi(0, None, None, None, None, None) == pp.POSPOP_OK
    torch.cuda.synchronize()
    got = counts_np(c)
    assert got[1].sum() == 0
    # only the call without errors counted (its first count; the second is empty)
    assert np.array_equal(got[0, :8], orc.bytes(8, host_pool[:1000]))
    assert got[0, 8:].sum() == 0
