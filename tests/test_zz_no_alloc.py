"""pospopcnt_batch_noalloc: the batched count for callers that cannot allocate.

Some callers cannot call cudaMalloc (graph capture that rejects allocation,
services with a fixed memory footprint, programs whose device memory belongs
to another allocator).  The no-allocation entry point keeps its work plan in
a fixed array of the library's device image.  These tests call it through the
C ABI and check it against the CPU oracle and against pospopcnt_batch bit for
bit, on two calls in a row (the array keeps the previous call's contents,
which must not leak into the next result); record it into a CUDA graph in the
capture mode that rejects allocation anywhere in the process; check that
decreasing offsets leave the counters untouched, that counters in pinned host
memory work as they do for pospopcnt_batch, and its size limit.  This file is
collected last.
"""
import numpy as np
import pytest
import torch

from paper_2412_16370_gb300 import binding as pp
from paper_2412_16370_gb300 import synth, synth_device

from _gpu import counts_np, oracle_batch_parallel

pytestmark = pytest.mark.gpu

MAX_ARRAYS = 65535


def _batch(dev, m, seed, hi=300000):
    sizes = synth.log_uniform_sizes(m, 1, hi, seed=seed)
    sizes[::41] = 0
    offs = synth.csr_offsets(sizes)
    buf = torch.empty(int(offs[-1]) + 64, dtype=torch.uint8, device=dev)
    synth_device.random_(buf, 500 + seed)
    base = buf[3:3 + int(offs[-1])]
    return base, torch.from_numpy(offs.view(np.int64)).to(dev)


def test_noalloc_matches_oracle_and_batch_on_two_calls_in_a_row(gpu, orc):
    L = pp.lib()
    for m, seed in ((5000, 1), (777, 2)):
        base, offs = _batch(gpu, m, seed)
        host = base.cpu().numpy()
        offs_h = offs.cpu().numpy().view(np.uint64)
        for w in (1, 8, 16, 32, 64):
            exp = oracle_batch_parallel(orc, w, host, offs_h)
            ref = torch.zeros((m, w), dtype=torch.int64, device=gpu)
            pp.pospopcnt_batch(w, ref, base, offs, m)
            assert pp.pospopcnt_batch_status() == pp.POSPOP_OK
            assert np.array_equal(counts_np(ref), exp), (m, w)
            for _ in range(2):
                got = torch.zeros((m, w), dtype=torch.int64, device=gpu)
                s = torch.cuda.current_stream().cuda_stream
                rc = L.pospopcnt_batch_noalloc(w, got.data_ptr(), base.data_ptr(), offs.data_ptr(),
                                               m, s)
                assert rc == pp.POSPOP_OK
                torch.cuda.synchronize()
                assert np.array_equal(counts_np(got), exp), (m, w)
                assert torch.equal(got, ref), (m, w)


def test_noalloc_recorded_in_a_graph_that_rejects_allocation(gpu, orc):
    """Captured in global mode (no thread may allocate while it records),
    replayed twice: counts equal two pospopcnt_batch calls and the oracle."""
    m, w = 3000, 16
    base, offs = _batch(gpu, m, 4)
    exp = oracle_batch_parallel(orc, w, base.cpu().numpy(), offs.cpu().numpy().view(np.uint64))
    c = torch.zeros((m, w), dtype=torch.int64, device=gpu)
    pp.pospopcnt_batch_noalloc(w, c, base, offs, m)      # warm-up call outside the capture
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s, capture_error_mode="global"):
        rc = pp.lib().pospopcnt_batch_noalloc(w, c.data_ptr(), base.data_ptr(), offs.data_ptr(),
                                              m, s.cuda_stream)
    assert rc == pp.POSPOP_OK
    c.zero_()
    torch.cuda.synchronize()
    g.replay()
    g.replay()
    torch.cuda.synchronize()
    ref = torch.zeros((m, w), dtype=torch.int64, device=gpu)
    for _ in range(2):
        pp.pospopcnt_batch(w, ref, base, offs, m)
    torch.cuda.synchronize()
    assert torch.equal(c, ref)
    assert np.array_equal(counts_np(c), 2 * exp)


def test_noalloc_decreasing_offsets_change_nothing(gpu):
    offs = torch.tensor([0, 10, 30, 20, 40], dtype=torch.int64, device=gpu)
    base = torch.ones(64, dtype=torch.uint8, device=gpu)
    c = torch.full((4, 8), 7, dtype=torch.int64, device=gpu)
    pp.pospopcnt_batch_noalloc(8, c, base, offs, 4)
    torch.cuda.synchronize()
    assert (c == 7).all()
    offs[3] = 30      # the next good call counts (the rejected plan does not linger)
    pp.pospopcnt_batch_noalloc(8, c, base, offs, 4)
    torch.cuda.synchronize()
    assert c.sum().item() == 4 * 8 * 7 + 40


def test_noalloc_counters_in_pinned_host_memory(gpu):
    """Counters in pinned host memory, which the kernels reach through its
    device address, exactly as pospopcnt_batch does."""
    m, w = 500, 32
    base, offs = _batch(gpu, m, 5, hi=20000)
    ref = torch.zeros((m, w), dtype=torch.int64, device=gpu)
    pp.pospopcnt_batch(w, ref, base, offs, m)
    got = torch.zeros((m, w), dtype=torch.int64, pin_memory=True)
    pp.pospopcnt_batch_noalloc(w, got, base, offs, m)
    torch.cuda.synchronize()
    assert torch.equal(got, ref.cpu())


def test_noalloc_allocates_nothing_and_respects_its_limit(gpu):
    L = pp.lib()
    m = MAX_ARRAYS
    base, offs = _batch(gpu, m, 3, hi=4096)
    c = torch.zeros((m, 8), dtype=torch.int64, device=gpu)
    pp.pospopcnt_batch_noalloc(8, c, base, offs, m)     # first call: symbol lookup
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    ref = torch.zeros((m, 8), dtype=torch.int64, device=gpu)
    got = torch.zeros((m, 8), dtype=torch.int64, device=gpu)
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    pp.pospopcnt_batch_noalloc(8, got, base, offs, m)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free1        # no device memory taken
    pp.pospopcnt_batch(8, ref, base, offs, m)
    torch.cuda.synchronize()
    assert torch.equal(got, ref)
    assert free0 >= free1
    s = torch.cuda.current_stream().cuda_stream
    big = torch.zeros(MAX_ARRAYS + 2, dtype=torch.int64, device=gpu)
    assert L.pospopcnt_batch_noalloc(8, got.data_ptr(), base.data_ptr(), big.data_ptr(),
                                     MAX_ARRAYS + 1, s) == pp.POSPOP_ERANGE
    assert L.pospopcnt_batch_noalloc(12, got.data_ptr(), base.data_ptr(), offs.data_ptr(),
                                     10, s) == pp.POSPOP_EINVAL
    assert L.pospopcnt_batch_noalloc(8, got.data_ptr(), base.data_ptr(), offs.data_ptr(),
                                     0, s) == pp.POSPOP_OK
