"""Bounded device-side waits run out and are reported, on healthy copies.

The staged kernels (the bulk-copy roofline read and the staged selected
count) wait on an mbarrier phase for each stage's bulk copy.  That wait is
bounded by the tune entry `wait <cycles>`; when it runs out the warp writes
POSPOP_ETIMEDOUT to the stream's status word, waits (with the fixed bound)
for its own copies still in flight and leaves.  With `wait 0` every first
wait gives up before it tries, so the exit is taken on healthy copies that
do land: nothing here waits on a copy that never arrives.  The tests check
that the stream then synchronises (the kernels finished), that the status
reads POSPOP_ETIMEDOUT once and is cleared, and that the same calls under
the default limit give exact results again.
"""
import numpy as np
import pytest
import torch

from paper_2412_16370_gb300 import binding as pp
from paper_2412_16370_gb300 import synth, synth_device

from _gpu import counts_np

pytestmark = pytest.mark.gpu

RING_SHAPES = (1, 2, 3)   # staged k: 8 warps x 3 stages, 12 x 2, 16 x 1


@pytest.fixture
def tune_lines(gpu, tmp_path):
    saved = tmp_path / "saved_tune.txt"
    saved.write_text(pp.pospopcnt_tune_describe())
    base = [l for l in saved.read_text().splitlines()
            if not l.startswith(("roofline", "staged", "wait"))]

    def install(*extra):
        f = tmp_path / "tune.txt"
        f.write_text("\n".join(base + list(extra)) + "\n")
        pp.pospopcnt_tune_load(str(f))
        return pp.pospopcnt_tune_describe()

    yield install
    pp.pospopcnt_tune_load(str(saved))


def _interior_sum(host: np.ndarray, start: int, n: int) -> int:
    a = (start + 15) & ~15
    e = (start + n) & ~15
    return int(host[a:e].view("<u4").astype(np.uint64).sum()) if e > a else 0


def test_wait_entry_round_trips(gpu, tune_lines):
    desc = tune_lines("wait 0")
    assert "\nwait 0\n" in desc
    desc = tune_lines("wait 12345")
    assert "\nwait 12345\n" in desc
    desc = tune_lines()
    assert "\nwait " not in desc      # the default (2^31) is not written out


@pytest.mark.parametrize("nbytes", (4 << 20, (64 << 20) + 8192 * 3 + 48))
def test_roofline_bulk_wait_expires_and_recovers(gpu, tune_lines, nbytes):
    buf = torch.empty(nbytes + 16, dtype=torch.uint8, device=gpu)
    synth_device.random_(buf, 81)
    host = buf.cpu().numpy()
    data = buf[5:5 + nbytes]
    s = torch.cuda.Stream()
    for bs in (256, 128):                      # 8 and 4 warps per block, 3 stages each
        tune_lines(f"roofline {bs} 2 2", "wait 0")
        out = torch.zeros(1, dtype=torch.int64, device=gpu)
        pp.pospopcnt_roofline_read(data, out, nbytes, s)
        s.synchronize()                        # the kernel finished
        assert pp.pospopcnt_batch_status(s) == pp.POSPOP_ETIMEDOUT, bs
        assert pp.pospopcnt_batch_status(s) == pp.POSPOP_OK      # cleared once read
        tune_lines(f"roofline {bs} 2 2")       # default limit
        out.zero_()
        pp.pospopcnt_roofline_read(data, out, nbytes, s)
        assert pp.pospopcnt_batch_status(s) == pp.POSPOP_OK
        assert int(out.cpu().numpy().view(np.uint64)[0]) == _interior_sum(host, 5, nbytes), bs


@pytest.mark.parametrize("w", (8, 32))
def test_staged_select_wait_expires_and_recovers(gpu, orc, tune_lines, w):
    W = w // 8
    n = (48 << 20) // W + 3          # enough 16-row chunks for every ring shape
    words_h = synth.random_bytes(n * W, seed=90 + w)
    sel_h = synth.random_bytes(4 * ((n + 31) // 32), seed=91 + w)
    words = torch.from_numpy(words_h).to(gpu)
    sel = torch.from_numpy(sel_h).to(gpu)
    exp = orc.masked(w, words_h, n, sel_h)
    s = torch.cuda.Stream()
    for k in RING_SHAPES:
        tune_lines(f"staged {k}", "wait 0")
        c = torch.zeros(w, dtype=torch.int64, device=gpu)
        pp.pospopcnt_masked(w, c, words, n, sel, s)
        s.synchronize()
        assert pp.pospopcnt_batch_status(s) == pp.POSPOP_ETIMEDOUT, k
        tune_lines(f"staged {k}")
        c.zero_()
        pp.pospopcnt_masked(w, c, words, n, sel, s)
        assert pp.pospopcnt_batch_status(s) == pp.POSPOP_OK, k
        assert np.array_equal(counts_np(c), exp), k


def test_small_limit_is_either_exact_or_reported(gpu, orc, tune_lines):
    """A limit of a few hundred cycles: some waits may expire and some not;
    every call finishes, and a call whose status is OK is exact."""
    w, W = 16, 2
    n = (48 << 20) // W
    words_h = synth.random_bytes(n * W, seed=95)
    sel_h = synth.random_bytes(4 * ((n + 31) // 32), seed=96)
    words = torch.from_numpy(words_h).to(gpu)
    sel = torch.from_numpy(sel_h).to(gpu)
    exp = orc.masked(w, words_h, n, sel_h)
    s = torch.cuda.Stream()
    tune_lines("staged 1", "wait 300")
    for _ in range(3):
        c = torch.zeros(w, dtype=torch.int64, device=gpu)
        pp.pospopcnt_masked(w, c, words, n, sel, s)
        st = pp.pospopcnt_batch_status(s)
        assert st in (pp.POSPOP_OK, pp.POSPOP_ETIMEDOUT)
        if st == pp.POSPOP_OK:
            assert np.array_equal(counts_np(c), exp)
