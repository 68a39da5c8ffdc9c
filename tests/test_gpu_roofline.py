"""The roofline read kernels (pospopcnt_roofline_read) on the GPU.

Both forms (direct 16-byte loads; cp.async.bulk staging through shared
memory with mbarrier completion) must add exactly the sum of the 32-bit
little-endian words of the 16-byte-aligned interior of the input to *sum,
for every launch variant, ragged sizes and unaligned starts.
"""
import numpy as np
import pytest
import torch

from paper_2412_16370_gb300 import binding as pp
from paper_2412_16370_gb300 import synth, synth_device

pytestmark = pytest.mark.gpu

VARIANTS = [(256, 0), (256, 1), (512, 0), (512, 1), (1024, 0), (1024, 1), (256, 2), (128, 2)]


@pytest.fixture
def tune_roof(gpu, tmp_path):
    saved = tmp_path / "saved_tune.txt"
    saved.write_text(pp.pospopcnt_tune_describe())
    keep = [l for l in saved.read_text().splitlines() if not l.startswith("roofline")]

    def install(bs, hint, cps):
        f = tmp_path / "tune.txt"
        f.write_text("\n".join(keep) + f"\nroofline {bs} {hint} {cps}\n")
        pp.pospopcnt_tune_load(str(f))

    yield install
    pp.pospopcnt_tune_load(str(saved))


def _interior_sum(host: np.ndarray, start: int, n: int) -> int:
    a = (start + 15) & ~15
    e = (start + n) & ~15
    if e <= a:
        return 0
    return int(host[a:e].view("<u4").astype(np.uint64).sum())


def test_every_variant_exact(gpu, tune_roof):
    total = (48 << 20) + 4096
    buf = torch.empty(total, dtype=torch.uint8, device=gpu)
    synth_device.random_(buf, 71)
    host = buf.cpu().numpy()
    cases = [(0, 0), (0, 15), (3, 16), (5, 40), (0, 8192), (16, 8192 * 3 + 48), (7, 1 << 20),
             (0, (1 << 20) + 8192 * 5 + 16 * 7), (9, (48 << 20) - 77)]
    s = torch.cuda.Stream()
    for bs, hint in VARIANTS:
        for cps in (1, 3):
            tune_roof(bs, hint, cps)
            for start, n in cases:
                out = torch.zeros(1, dtype=torch.int64, device=gpu)
                pp.pospopcnt_roofline_read(buf[start:start + n] if n else buf[start:start], out, n, s)
                assert pp.pospopcnt_batch_status(s) == pp.POSPOP_OK
                got = int(out.cpu().numpy().view(np.uint64)[0])
                assert got == _interior_sum(host, start, n), (bs, hint, cps, start, n)


def test_bulk_form_large_and_adds_into(gpu, tune_roof):
    n = 1 << 30
    buf = torch.empty(n, dtype=torch.uint8, device=gpu)
    synth_device.fill_(buf, 0x01)
    tune_roof(256, 2, 1)
    out = torch.full((1,), 5, dtype=torch.int64, device=gpu)
    for _ in range(3):
        pp.pospopcnt_roofline_read(buf, out, n)
    torch.cuda.synchronize()
    assert pp.pospopcnt_batch_status() == pp.POSPOP_OK
    assert int(out.item()) == 5 + 3 * (n // 4) * 0x01010101
    # same bytes, direct form
    tune_roof(256, 1, 18)
    out2 = torch.zeros(1, dtype=torch.int64, device=gpu)
    pp.pospopcnt_roofline_read(buf, out2, n)
    torch.cuda.synchronize()
    assert int(out2.item()) == (n // 4) * 0x01010101


def test_bulk_form_random_bytes(gpu, tune_roof):
    n = (256 << 20) + 8192 + 32
    buf = torch.empty(n + 16, dtype=torch.uint8, device=gpu)
    synth_device.random_(buf, 72)
    host = synth.random_bytes(n + 16, seed=72)
    for bs in (256, 128):
        tune_roof(bs, 2, 2)
        out = torch.zeros(1, dtype=torch.int64, device=gpu)
        pp.pospopcnt_roofline_read(buf[3:3 + n], out, n)
        torch.cuda.synchronize()
        assert int(out.cpu().numpy().view(np.uint64)[0]) == _interior_sum(host, 3, n), bs
