"""Runtime entry points on the GPU: workspace reservation for capture into a
caller's CUDA graph, and shutdown / set-up again."""
import numpy as np
import pytest
import torch

from paper_2412_16370_gb300 import binding as pp
from paper_2412_16370_gb300 import synth

from _gpu import counts_np

pytestmark = pytest.mark.gpu


def _batch_case(gpu, m, seed):
    sizes = synth.log_uniform_sizes(m, 1, 50000, seed=seed)
    offs = synth.csr_offsets(sizes)
    host = synth.random_bytes(int(offs[-1]), seed=seed + 1)
    base = torch.from_numpy(host).to(gpu)
    offs_d = torch.from_numpy(offs.view(np.int64)).to(gpu)
    return host, offs, base, offs_d


def test_reserve_then_capture_in_a_caller_graph(gpu, orc):
    m = 3000
    host, offs, base, offs_d = _batch_case(gpu, m, 61)
    exp = orc.batch(32, host, offs)
    s = torch.cuda.Stream()
    c = torch.zeros((m, 32), dtype=torch.int64, device=gpu)
    pp.pospopcnt_reserve(m, s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s, capture_error_mode="thread_local"):
        pp.pospopcnt_batch(32, c, base, offs_d, m, s)
    torch.cuda.synchronize()
    c.zero_()
    torch.cuda.synchronize()
    g.replay()
    g.replay()
    torch.cuda.synchronize()
    assert np.array_equal(counts_np(c), 2 * exp)
    # a capture that would need a larger workspace is refused, not allocated
    s2 = torch.cuda.Stream()
    rc = []
    dummy = torch.zeros(1, device=gpu)
    g2 = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g2, stream=s2, capture_error_mode="thread_local"):
        dummy.add_(1)
        rc.append(pp.lib().pospopcnt_batch(32, c.data_ptr(), base.data_ptr(), offs_d.data_ptr(),
                                           m, s2.cuda_stream))
    assert rc == [pp.POSPOP_ENOMEM]


def test_shutdown_and_set_up_again(gpu, orc):
    host = synth.random_bytes(1 << 20, seed=62)
    data = torch.from_numpy(host).to(gpu)
    exp = orc.bytes(16, host)
    for _ in range(2):
        c = torch.zeros(16, dtype=torch.int64, device=gpu)
        pp.pospopcnt_async(16, c, data)
        torch.cuda.synchronize()
        assert np.array_equal(counts_np(c), exp)
        pp.shutdown()
    pp.init(0)
    pp.init(0)   # idempotent
    c = torch.zeros(16, dtype=torch.int64, device=gpu)
    pp.pospopcnt_async(16, c, data)
    torch.cuda.synchronize()
    assert np.array_equal(counts_np(c), exp)
