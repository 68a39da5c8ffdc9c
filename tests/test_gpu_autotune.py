"""The autotuner (pospopcnt_autotune) on the GPU.

It times the launch candidates of the single-array kernel per width group
and size class, of the batched kernel per width group (launch shape on a mix
of batches, work-item rows per array size class), of the serving kernel per
serving size class and of the roofline read kernels, installs the fastest
and writes the table.  The written table must load back entry for entry, and
counts made with it (single array, batch, served requests) must still equal
the oracle's.
"""
import re

import numpy as np
import pytest
import torch

from paper_2412_16370_gb300 import binding as pp
from paper_2412_16370_gb300 import synth

from _gpu import WORD_W, counts_np

pytestmark = pytest.mark.gpu


def _entries(text):
    return [l for l in text.splitlines() if l and not l.startswith("#")]


def test_autotune_writes_a_loadable_table_and_counts_stay_exact(gpu, orc, tmp_path):
    saved = tmp_path / "saved.txt"
    saved.write_text(pp.pospopcnt_tune_describe())
    out = tmp_path / "tuned.txt"
    try:
        pp.pospopcnt_autotune(64 << 20, str(out))
        text = out.read_text()
        assert "autotuned" in text
        for kind in ("batch", "roofline", "pdl", "staged"):
            assert kind in text, kind
        for cls in range(5):   # each size class, for every width or per width
            assert re.search(rf"^stream (\d+ )?{cls} ", text, re.M), cls
        for k in range(4):     # each serving size class
            assert re.search(rf"^serve {k} \d+ \d+ \d+ \d+$", text, re.M), k
        assert "autotuned" in pp.pospopcnt_tune_describe()
        pp.pospopcnt_tune_load(str(out))          # the written table parses
        # ... and loads back entry for entry
        assert _entries(pp.pospopcnt_tune_describe()) == _entries(text)
        # counts under the tuned table: a single array and a ragged batch
        host = synth.random_bytes((3 << 20) + 11, seed=91)
        data = torch.from_numpy(host).to(gpu)[5:]
        for w in WORD_W:
            c = torch.zeros(w, dtype=torch.int64, device=gpu)
            pp.pospopcnt_async(w, c, data)
            torch.cuda.synchronize()
            assert np.array_equal(counts_np(c), orc.bytes(w, host[5:])), w
        sizes = synth.log_uniform_sizes(500, 1, 100000, seed=92)
        offs = synth.csr_offsets(sizes)
        bh = synth.random_bytes(int(offs[-1]), seed=93)
        base = torch.from_numpy(bh).to(gpu)
        cb = torch.zeros((len(sizes), 16), dtype=torch.int64, device=gpu)
        pp.pospopcnt_batch(16, cb, base, torch.from_numpy(offs.view(np.int64)).to(gpu))
        assert np.array_equal(counts_np(cb), orc.batch(16, bh, offs))
        # served requests of every serving class small enough for the buffer
        srv = pp.pospop_server_create(1 << 30, 64, 2)
        try:
            res = np.zeros((4, 64), dtype=np.uint64)
            for k, nb in enumerate((1000, 3 << 20)):
                pp.pospop_server_submit(srv, 32, data.data_ptr(), nb, res[k])
            assert pp.pospop_server_drain(srv, 10000) == pp.POSPOP_OK
        finally:
            pp.pospop_server_destroy(srv)
        for k, nb in enumerate((1000, 3 << 20)):
            assert np.array_equal(res[k, :32], orc.bytes(32, host[5:5 + nb])), nb
    finally:
        pp.pospopcnt_tune_load(str(saved))


def test_per_width_entries_load_plan_and_count(gpu, orc, tmp_path):
    """A table whose entries differ by width group: each width plans with its
    own entry, the table writes back in the per-width form, and counts stay
    exact; malformed per-width lines are refused."""
    saved = tmp_path / "saved.txt"
    saved.write_text(pp.pospopcnt_tune_describe())
    keep = [l for l in saved.read_text().splitlines()
            if not l.startswith(("stream", "batch"))]
    shapes = {8: (256, 2, 16, 0), 16: (512, 1, 32, 1), 32: (128, 4, 16, 1), 64: (512, 1, 16, 0)}
    lines = keep + ["stream 2 512 1 16 1 1 8"]   # every width, then per-width overrides
    for w, (bs, minb, d, h) in shapes.items():
        lines.append(f"stream {w} 2 {bs} {minb} {d} {h} 1 8")
        lines.append(f"batch {w} {bs} {minb} {d} {h} 1 {63 + w} 1")
    f = tmp_path / "perw.txt"
    f.write_text("\n".join(lines) + "\n")
    try:
        pp.pospopcnt_tune_load(str(f))
        text = pp.pospopcnt_tune_describe()
        for w, (bs, minb, d, h) in shapes.items():
            assert f"stream {w} 2 {bs} {minb} {d} {h} 1 8" in text, w
            assert f"batch {w} {bs} {minb} {d} {h} 1 {63 + w} 1" in text, w
        host = synth.random_bytes((2 << 20) + 5, seed=94)   # size class 2
        data = torch.from_numpy(host).to(gpu)
        sizes = synth.log_uniform_sizes(300, 1, 100000, seed=95)
        offs = synth.csr_offsets(sizes)
        bh = synth.random_bytes(int(offs[-1]), seed=96)
        base = torch.from_numpy(bh).to(gpu)
        offs_d = torch.from_numpy(offs.view(np.int64)).to(gpu)
        for w in (1, 4, 8, 16, 32, 64, 128, 256):
            g = min(max(w, 8), 64)
            bs, _, d, h = shapes[g]
            plan = pp.pospopcnt_plan(w, len(host) - 1)
            assert (plan["block"], plan["depth"], plan["hint"]) == (bs, d, h), w
            c = torch.zeros(w, dtype=torch.int64, device=gpu)
            pp.pospopcnt_async(w, c, data[1:])
            cb = torch.zeros((len(sizes), w), dtype=torch.int64, device=gpu)
            pp.pospopcnt_batch(w, cb, base, offs_d)
            torch.cuda.synchronize()
            assert np.array_equal(counts_np(c), orc.bytes(w, host[1:])), w
            assert np.array_equal(counts_np(cb), orc.batch(w, bh, offs)), w
        for bad in ("stream 24 2 512 1 16 1 1 8", "stream 8 2 512 1 16 1 1",
                    "batch 8 512 1 16 1 1 127 1 5", "batch 128 512 1 16 1 1 127 1",
                    "stream 8 2 512 1 16 1 1 x"):
            fb = tmp_path / "bad.txt"
            fb.write_text("\n".join(keep + [bad]) + "\n")
            with pytest.raises(pp.PospopError):
                pp.pospopcnt_tune_load(str(fb))
    finally:
        pp.pospopcnt_tune_load(str(saved))
