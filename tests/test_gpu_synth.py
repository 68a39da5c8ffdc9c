"""The device input generator writes exactly the numpy recipe's bytes."""
import numpy as np
import pytest
import torch

from paper_2412_16370_gb300 import synth, synth_device

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("start,n,pad", [(0, 1, 0), (3, 17, 5), (0, 4096, 0), (12345, 100003, 7),
                                         (1 << 33, 70001, 1)])
def test_generator_twin(gpu, start, n, pad):
    buf = torch.zeros(n + pad + 32, dtype=torch.uint8, device=gpu)
    d = buf[pad:pad + n]
    synth_device.random_(d, 99, start=start)
    assert np.array_equal(d.cpu().numpy(), synth.random_bytes(n, 99, start=start))
    for p in (0.01, 0.99, 0.3):
        synth_device.bernoulli_(d, p, 7, start=start)
        assert np.array_equal(d.cpu().numpy(), synth.bernoulli_bytes(n, p, 7, start=start)), p
    synth_device.one_hot_(d, 5, start=start)
    assert np.array_equal(d.cpu().numpy(), synth.one_hot_bytes(n, 5, start=start))
    synth_device.fill_(d, 0xA5)
    assert (d == 0xA5).all()
    # bytes outside the window are untouched
    assert not buf[:pad].any() and not buf[pad + n:].any()
