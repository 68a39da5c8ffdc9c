"""The seeded input recipe, checked on the host (no GPU): the generator is
SplitMix64 as published, and each workload generator has the distribution
the benchmark configurations state (Zipf(1.1) one-hot classes, log-uniform
sizes with median 2 KiB and mean about 275 KB on [1 B, 4 MiB], the short
sweep's 280 lengths, Bernoulli(p) bit densities, Poisson arrivals)."""
import math

import numpy as np
import pytest

from paper_2412_16370_gb300 import synth


def test_splitmix64_matches_the_published_sequence():
    # SplitMix64 (Steele, Lea and Flood, 2014) from state 0: its first three
    # outputs, as listed with the reference implementation
    got = synth.splitmix64(0, np.arange(3, dtype=np.uint64))
    assert [int(x) for x in got] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_random_bytes_are_little_endian_outputs_and_windows_agree():
    b = synth.random_bytes(24, seed=5)
    words = synth.splitmix64(5, np.arange(3, dtype=np.uint64))
    assert bytes(b) == words.astype("<u8").tobytes()
    whole = synth.random_bytes(1000, seed=9)
    for start in (0, 1, 7, 8, 13, 500):
        assert np.array_equal(synth.random_bytes(100, seed=9, start=start), whole[start:start + 100])


def test_zipf_classes():
    p = synth.zipf_probabilities()
    stated = [.398, .186, .119, .087, .068, .055, .047, .040]
    assert np.allclose(p, stated, atol=1.5e-3)
    assert abs(sum(p) - 1.0) < 1e-12
    t = synth.zipf_thresholds()
    assert t == sorted(t) and len(t) == 7 and t[-1] < 2 ** 32
    n = 1 << 20
    cats = synth.one_hot_categories(n, seed=4)
    freq = np.bincount(cats, minlength=8) / n
    sigma = np.sqrt(np.asarray(p) * (1 - np.asarray(p)) / n)
    assert (np.abs(freq - p) < 6 * sigma).all()
    bytes_ = synth.one_hot_bytes(4096, seed=4)
    assert all(bin(int(x)).count("1") == 1 and int(x) < 256 for x in bytes_)


def test_log_uniform_sizes_of_the_ragged_batch():
    s = synth.log_uniform_sizes(200000, 1, 4 << 20, seed=3)
    assert s.min() >= 1 and s.max() <= 4 << 20
    assert 1900 <= np.median(s) <= 2200                 # sqrt(4 MiB) = 2048
    mean = (4 << 20) / math.log((4 << 20) + 1)   # log-uniform on [1, 4 MiB + 1): (b - a) / ln(b / a)
    assert abs(s.mean() / mean - 1) < 0.03
    offs = synth.csr_offsets(s)
    assert offs[0] == 0 and offs[-1] == s.sum() and (np.diff(offs.astype(np.int64)) == s).all()


def test_short_sweep_lengths():
    lens = synth.short_sweep_lengths()
    assert len(lens) == 280
    assert lens[:256] == list(range(1, 257))
    assert {511, 512, 513, 65535, 65536, 65537} <= set(lens)


@pytest.mark.parametrize("p", (0.01, 0.99))
def test_bernoulli_densities(p):
    n = 1 << 20
    b = synth.bernoulli_bytes(n, p, seed=6)
    ones = int(np.unpackbits(b).sum())
    bits = 8 * n
    assert abs(ones - bits * p) < 6 * math.sqrt(bits * p * (1 - p))
    assert synth.bernoulli_threshold(0.0) == 0 and synth.bernoulli_threshold(1.0) == 2 ** 32


def test_poisson_request_stream():
    n = 200000
    rate = 1e5
    r = synth.poisson_requests(n, rate, seed=8, lo=64, hi=256 << 20, pool_bytes=8 << 30)
    gaps = np.diff(np.concatenate([[0.0], r["arrival_s"]]))
    assert (gaps >= 0).all()
    assert abs(gaps.mean() * rate - 1) < 6 / math.sqrt(n)
    assert abs(gaps.std() * rate - 1) < 0.02            # exponential: sd = mean
    freq = np.bincount(r["w"], minlength=65)[[8, 16, 32, 64]] / n
    assert (np.abs(freq - 0.25) < 6 * math.sqrt(0.25 * 0.75 / n)).all()
    assert r["nbytes"].min() >= 64 and r["nbytes"].max() <= 256 << 20
    assert ((r["offset"] >= 0) & (r["offset"] + r["nbytes"] <= 8 << 30)).all()
