"""Shard-and-sum across ranks, on CPU with the gloo backend (world size 2 and 3).

Each rank counts its shard (with the CPU oracle: this checks the sharding
arithmetic, not the kernels), the counters are summed with an all-reduce,
and the total must equal the count of the whole input.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2412_16370_gb300 import shard, synth


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, nbytes, offset, result_q):
    import oracle
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        data = synth.random_bytes(nbytes + offset, seed=77)[offset:]
        lo, hi = shard.shard_range(nbytes, rank, world)
        orc = oracle.load()
        out = {}
        for w in (1, 8, 16, 32, 64):
            c = torch.from_numpy(orc.bytes(w, data[lo:hi]).view(np.int64).copy())
            shard.sum_counts(c)
            out[w] = c.numpy().view(np.uint64).copy()
        result_q.put((rank, out))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,nbytes,offset", [(2, 1_000_003, 5), (3, 4097, 0), (2, 63, 1)])
def test_shard_and_sum(world, nbytes, offset):
    import oracle
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, nbytes, offset, q))
             for r in range(world)]
    for p in procs:
        p.start()
    results = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    data = synth.random_bytes(nbytes + offset, seed=77)[offset:]
    orc = oracle.load()
    for _, out in results:
        for w, got in out.items():
            assert np.array_equal(got, orc.bytes(w, data)), w


def test_shard_ranges_cover_and_align():
    for n in (0, 1, 63, 64, 65, 10 ** 6 + 7):
        for world in (1, 2, 3, 8):
            rs = shard.all_ranks_ranges(n, world)
            assert rs[0][0] == 0 and rs[-1][1] == n
            for (a, b), (c, _) in zip(rs, rs[1:]):
                assert b == c and a <= b
            for a, _ in rs:
                assert a % 64 == 0 or a == n
