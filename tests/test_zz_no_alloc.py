"""pospopcnt_batch_noalloc: the batched count for callers that cannot allocate.

Some callers cannot call cudaMalloc (graph capture that rejects allocation,
services with a fixed memory footprint, programs whose device memory belongs
to another allocator).  The no-allocation entry point keeps its work plan in
a fixed array of the library's device image.  These tests call it through the
C ABI and check it against pospopcnt_batch bit for bit, on two calls in a row
(the array keeps the previous call's contents, which must not leak into the
next result), and check its size limit.  This file is collected last.
"""
import numpy as np
import pytest
import torch

from paper_2412_16370_gb300 import binding as pp
from paper_2412_16370_gb300 import synth, synth_device

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


def test_noalloc_matches_batch_on_two_calls_in_a_row(gpu):
    L = pp.lib()
    for m, seed in ((5000, 1), (777, 2)):
        base, offs = _batch(gpu, m, seed)
        for w in (8, 16, 32, 64):
            ref = torch.zeros((m, w), dtype=torch.int64, device=gpu)
            pp.pospopcnt_batch(w, ref, base, offs, m)
            assert pp.pospopcnt_batch_status() == pp.POSPOP_OK
            for _ in range(2):
                got = torch.zeros((m, w), dtype=torch.int64, device=gpu)
                s = torch.cuda.current_stream().cuda_stream
                rc = L.pospopcnt_batch_noalloc(w, got.data_ptr(), base.data_ptr(), offs.data_ptr(),
                                               m, s)
                assert rc == pp.POSPOP_OK
                torch.cuda.synchronize()
                assert torch.equal(got, ref), (m, w)


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
