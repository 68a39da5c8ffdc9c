"""Shard-and-sum with the CUDA path on one GPU.

Counts are additive under concatenation of whole words (Section 4, step 1
and its footnote), so one array split by shard.shard_range into 2..8 shards
(boundaries 64 bytes apart from the start, so every shard starts on a word
boundary for every w <= 64 and keeps the whole's 16-byte phase) and counted
shard by shard with the single-array entry point must sum to the oracle's
count of the whole array.  This is the per-rank work of a multi-GPU count;
the all-reduce of the w counters is covered by the gloo test on the CPU.
"""
import numpy as np
import pytest
import torch

from paper_2412_16370_gb300 import binding as pp
from paper_2412_16370_gb300 import shard, synth_device

from _gpu import WORD_W, counts_np, oracle_device_bytes

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("nbytes,offset", [((96 << 20) + 77, 13), ((1 << 20) + 1, 0),
                                           (4097, 5), (63, 1)])
def test_shards_sum_to_the_whole(gpu, orc, nbytes, offset):
    buf = torch.empty(nbytes + offset + 16, dtype=torch.uint8, device=gpu)
    synth_device.random_(buf, 4242 + offset)
    data = buf[offset:offset + nbytes]
    exp = oracle_device_bytes(orc, WORD_W + (1,), data)
    for world in range(2, 9):
        for w in WORD_W + (1,):
            per_rank = []
            for rank in range(world):
                lo, hi = shard.shard_range(nbytes, rank, world)
                c = torch.zeros(w, dtype=torch.int64, device=gpu)
                if hi > lo:
                    pp.pospopcnt_async(w, c, data[lo:hi], hi - lo)
                per_rank.append(c)
            torch.cuda.synchronize()
            total = np.sum([counts_np(c) for c in per_rank], axis=0, dtype=np.uint64)
            assert np.array_equal(total, exp[w]), (world, w)
