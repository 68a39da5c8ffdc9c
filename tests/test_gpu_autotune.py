"""The autotuner (pospopcnt_autotune) on the GPU.

It times the launch candidates of the single-array kernel per size class,
of the batched kernel on a ragged batch and of the roofline read kernels,
installs the fastest and writes the table.  The written table must load
back, and counts made with it must still equal the oracle's.
"""
import numpy as np
import pytest
import torch

from paper_2412_16370_gb300 import binding as pp
from paper_2412_16370_gb300 import synth

from _gpu import WORD_W, counts_np

pytestmark = pytest.mark.gpu


def test_autotune_writes_a_loadable_table_and_counts_stay_exact(gpu, orc, tmp_path):
    saved = tmp_path / "saved.txt"
    saved.write_text(pp.pospopcnt_tune_describe())
    out = tmp_path / "tuned.txt"
    try:
        pp.pospopcnt_autotune(64 << 20, str(out))
        text = out.read_text()
        assert "autotuned" in text
        for kind in ("stream 0", "stream 4", "batch", "roofline", "pdl", "staged"):
            assert kind in text, kind
        assert "autotuned" in pp.pospopcnt_tune_describe()
        pp.pospopcnt_tune_load(str(out))          # the written table parses
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
    finally:
        pp.pospopcnt_tune_load(str(saved))
