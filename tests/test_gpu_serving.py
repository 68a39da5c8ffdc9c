"""The continuous-batching serving loop (pospop_server_*) on the GPU.

Requests of mixed width and size over a device-resident pool must give the
same counts in the mix as alone (and as the CPU oracle), admission must keep
the in-flight input bytes within the budget and the admitted requests within
the slot cap, later arrivals must be launched while earlier batches are still
running, the tune table's per-class serving entries must take effect, and
every wait must end with a status.  The general tests run under each
schedule (size classes, dispatch by remaining bytes, and the same per size
class of the bytes left).
"""
import numpy as np
import pytest
import torch

from paper_2412_16370_gb300 import binding as pp
from paper_2412_16370_gb300 import synth, synth_device

pytestmark = pytest.mark.gpu

MIB = 1 << 20


@pytest.fixture(scope="module")
def pool(gpu):
    n = 256 * MIB
    t = torch.empty(n + 64, dtype=torch.uint8, device=gpu)
    synth_device.random_(t, 2024)
    torch.cuda.synchronize()
    return t


@pytest.fixture
def serve_tune(gpu, tmp_path):
    saved = tmp_path / "saved_tune.txt"
    saved.write_text(pp.pospopcnt_tune_describe())
    keep = [l for l in saved.read_text().splitlines() if not l.startswith(("serve ", "serve_light"))]

    def install(*lines):
        f = tmp_path / "tune.txt"
        f.write_text("\n".join(keep + list(lines)) + "\n")
        pp.pospopcnt_tune_load(str(f))

    yield install
    pp.pospopcnt_tune_load(str(saved))


@pytest.fixture(params=(0, 1, 2, 3), ids=("classes", "remaining", "remaining_by_class",
                                           "resident"))
def mode(serve_tune, request):
    """Run a test under each schedule: size classes (`serve_mode 0`),
    dispatch by remaining bytes (`serve_mode 1`), the same per size class of
    the bytes left (`serve_mode 2`) and the resident grid fed through a
    device-side queue (`serve_mode 3`)."""
    serve_tune(f"serve_mode {request.param}")
    return request.param


def _requests(n, seed, lo, hi, pool_bytes):
    r = synth.poisson_requests(n, 1.0, seed, lo, hi, pool_bytes=pool_bytes)
    return r["w"].astype(np.int32), r["nbytes"].astype(np.uint64), r["offset"].astype(np.uint64)


def _solo(pool, w, nbytes, offs):
    out = torch.zeros((len(w), 64), dtype=torch.int64, device=pool.device)
    base = pool.data_ptr()
    for k in range(len(w)):
        pp.pospopcnt_async(int(w[k]), out[k], base + int(offs[k]), int(nbytes[k]))
    torch.cuda.synchronize()
    return out.cpu().numpy().view(np.uint64)


def test_mix_equals_solo_and_oracle(gpu, orc, pool, mode):
    n = 3000
    w, nbytes, offs = _requests(n, 11, 1, 8 * MIB, 256 * MIB)
    nbytes[::97] = 0   # some empty requests
    srv = pp.pospop_server_create(1 << 30, 512, 4)
    try:
        results = np.zeros((n, 64), dtype=np.uint64)
        arrival = (np.arange(n) * 2000).astype(np.int64)   # one request every 2 us
        ptrs = pool.data_ptr() + offs
        recs = pp.pospop_server_run_trace(srv, arrival, w, ptrs, nbytes, results)
        assert (recs["status"] == 0).all()
        assert np.array_equal(recs["nbytes"], nbytes)
        st = pp.pospop_server_stats(srv)
        assert st["submitted"] == st["finished"] == n and st["inflight"] == 0
    finally:
        pp.pospop_server_destroy(srv)
    solo = _solo(pool, w, nbytes, offs)
    for k in range(n):
        assert np.array_equal(results[k, :w[k]], solo[k, :w[k]]), k
    host = pool.cpu().numpy()
    for k in range(0, n, 37):
        seg = host[int(offs[k]):int(offs[k]) + int(nbytes[k])]
        assert np.array_equal(results[k, :w[k]], orc.bytes(int(w[k]), seg)), k


def _max_overlap(recs, start_key, weight=None):
    """Largest sum of weights over requests whose [start, done) intervals overlap."""
    ev = []
    for k, r in enumerate(recs):
        wt = 1 if weight is None else int(weight[k])
        ev.append((int(r[start_key]), wt))
        ev.append((int(r["t_done_ns"]), -wt))
    ev.sort(key=lambda x: (x[0], x[1]))
    cur = best = 0
    for _, d in ev:
        cur += d
        best = max(best, cur)
    return best


def test_budget_and_slots_respected(gpu, pool, mode):
    n = 400
    w, nbytes, offs = _requests(n, 12, 1 * MIB, 4 * MIB, 256 * MIB)
    budget = 6 * MIB
    srv = pp.pospop_server_create(budget, 3, 4)
    try:
        results = np.zeros((n, 64), dtype=np.uint64)
        recs = pp.pospop_server_run_trace(srv, np.zeros(n, dtype=np.int64), w,
                                          pool.data_ptr() + offs, nbytes, results)
    finally:
        pp.pospop_server_destroy(srv)
    assert (recs["status"] == 0).all()
    assert _max_overlap(recs, "t_admit_ns", nbytes) <= budget
    assert _max_overlap(recs, "t_admit_ns") <= 3
    solo = _solo(pool, w, nbytes, offs)
    for k in range(n):
        assert np.array_equal(results[k, :w[k]], solo[k, :w[k]]), k


def test_later_arrivals_overlap_running_batches(gpu, pool, mode):
    """Continuous batching: requests are launched while earlier launches run."""
    n = 64
    w = np.full(n, 16, dtype=np.int32)
    nbytes = np.full(n, 128 * MIB, dtype=np.uint64)
    offs = (np.arange(n) % 2 * 64).astype(np.uint64)
    arrival = (np.arange(n) * 5000).astype(np.int64)     # every 5 us; each takes ~20 us
    srv = pp.pospop_server_create(64 << 30, 4096, 4)
    try:
        results = np.zeros((n, 64), dtype=np.uint64)
        recs = pp.pospop_server_run_trace(srv, arrival, w, pool.data_ptr() + offs, nbytes, results)
    finally:
        pp.pospop_server_destroy(srv)
    assert (recs["status"] == 0).all()
    launches = sorted(set(int(x) for x in recs["t_launch_ns"]))
    assert len(launches) > 1
    # some batch was launched before an earlier batch had finished
    first_done = {}
    for r in recs:
        first_done.setdefault(int(r["t_launch_ns"]), int(r["t_done_ns"]))
    overlapped = any(launches[i + 1] < first_done[launches[i]] for i in range(len(launches) - 1))
    assert overlapped
    exp = _solo(pool, w[:2], nbytes[:2], offs[:2])
    for k in range(n):
        assert np.array_equal(results[k, :16], exp[k % 2, :16])


def test_strided_items_mix_equals_oracle(gpu, orc, pool, serve_tune):
    """Tune entry `serve_strided 1` (a work item takes every K-th row of its
    request) at light and full load: every result equals the oracle's."""
    n = 400
    w, nbytes, offs = _requests(n, 21, 1, 24 * MIB, 256 * MIB)
    nbytes[::41] = 0
    host = pool.cpu().numpy()
    for light in ("serve_light 0", "serve_light 68719476736"):
        serve_tune("serve_mode 0", "serve_strided 1", light)
        srv = pp.pospop_server_create(1 << 30, 512, 4)
        try:
            results = np.zeros((n, 64), dtype=np.uint64)
            recs = pp.pospop_server_run_trace(srv, (np.arange(n) * 3000).astype(np.int64), w,
                                              pool.data_ptr() + offs, nbytes, results)
        finally:
            pp.pospop_server_destroy(srv)
        assert (recs["status"] == 0).all()
        for k in range(n):
            seg = host[int(offs[k]):int(offs[k]) + int(nbytes[k])]
            assert np.array_equal(results[k, :w[k]], orc.bytes(int(w[k]), seg)), (light, k)


def test_promoted_batches_equal_solo(gpu, pool, serve_tune):
    """Tune entry `serve_promote 1` (requests that waited over 1 us may run on
    the next smaller class's stream) with `serve_order 1`: a loaded trace of
    mixed sizes still gives every request its single-array count."""
    serve_tune("serve_mode 0", "serve_promote 1", "serve_order 1", "serve 3 0 511 2 1", "serve 2 127 511 2 4")
    n = 300
    w, nbytes, offs = _requests(n, 23, 4096, 96 * MIB, 150 * MIB)
    srv = pp.pospop_server_create(8 << 30, 1024, 2)
    try:
        results = np.zeros((n, 64), dtype=np.uint64)
        recs = pp.pospop_server_run_trace(srv, (np.arange(n) * 2000).astype(np.int64), w,
                                          pool.data_ptr() + offs, nbytes, results)
    finally:
        pp.pospop_server_destroy(srv)
    assert (recs["status"] == 0).all()
    solo = _solo(pool, w, nbytes, offs)
    for k in range(n):
        assert np.array_equal(results[k, :w[k]], solo[k, :w[k]]), k


@pytest.mark.parametrize("srf_mode", (1, 2, 3))
@pytest.mark.parametrize("launch_bytes", (8 * MIB, 256 * MIB))
def test_dispatch_by_remaining_bytes(gpu, orc, pool, serve_tune, launch_bytes, srf_mode):
    """serve_mode 1 and 2: requests dispatched smallest-remaining first in
    launches of at most `launch_bytes` (with 8 MiB a request of up to 24 MiB
    is counted over several launches, its counters adding up in its slot,
    and with mode 2 its later launches move to smaller classes' streams as
    its bytes left shrink): every result equals the oracle's, empty requests
    included, and the budget and slot cap hold."""
    serve_tune(f"serve_mode {srf_mode}", f"serve_srf {launch_bytes} 4 255")
    n = 500
    w, nbytes, offs = _requests(n, 25, 1, 24 * MIB, 256 * MIB)
    nbytes[::53] = 0
    budget = 64 * MIB
    srv = pp.pospop_server_create(budget, 16, 4)
    try:
        results = np.zeros((n, 64), dtype=np.uint64)
        recs = pp.pospop_server_run_trace(srv, (np.arange(n) * 1500).astype(np.int64), w,
                                          pool.data_ptr() + offs, nbytes, results)
        st = pp.pospop_server_stats(srv)
        assert st["submitted"] == st["finished"] == n and st["inflight"] == 0
    finally:
        pp.pospop_server_destroy(srv)
    assert (recs["status"] == 0).all()
    assert _max_overlap(recs, "t_admit_ns", nbytes) <= budget
    assert _max_overlap(recs, "t_admit_ns") <= 16
    host = pool.cpu().numpy()
    for k in range(n):
        seg = host[int(offs[k]):int(offs[k]) + int(nbytes[k])]
        assert np.array_equal(results[k, :w[k]], orc.bytes(int(w[k]), seg)), (launch_bytes, srf_mode, k)


def test_aged_requests_take_half_a_launch(gpu, orc, pool, serve_tune):
    """serve_mode 1 with `serve_srf_age 1`: at almost every launch the
    longest-waiting request takes up to half of it ahead of the smallest
    remaining ones (its items then split across launches out of the queue's
    order): every result still equals the oracle's."""
    serve_tune("serve_mode 1", f"serve_srf {8 * MIB} 4 255", "serve_srf_age 1")
    n = 400
    w, nbytes, offs = _requests(n, 27, 1, 24 * MIB, 256 * MIB)
    nbytes[::47] = 0
    srv = pp.pospop_server_create(96 * MIB, 64, 4)
    try:
        results = np.zeros((n, 64), dtype=np.uint64)
        recs = pp.pospop_server_run_trace(srv, (np.arange(n) * 1000).astype(np.int64), w,
                                          pool.data_ptr() + offs, nbytes, results)
    finally:
        pp.pospop_server_destroy(srv)
    assert (recs["status"] == 0).all()
    host = pool.cpu().numpy()
    for k in range(n):
        seg = host[int(offs[k]):int(offs[k]) + int(nbytes[k])]
        assert np.array_equal(results[k, :w[k]], orc.bytes(int(w[k]), seg)), k


@pytest.mark.parametrize("srf_mode", (1, 2, 3))
def test_dispatch_by_remaining_bytes_host_input(gpu, orc, serve_tune, srf_mode):
    """serve_mode 1 and 2 on a pooled server: host input staged in the pool,
    counted over several launches, equal to the oracle; the pool is released."""
    serve_tune(f"serve_mode {srf_mode}", f"serve_srf {4 * MIB} 2 127")
    data = [synth.random_bytes(int(s), seed=600 + k)
            for k, s in enumerate((5 * MIB + 3, 17, 0, 9 * MIB, 1 * MIB))]
    srv = pp.pospop_server_create_pooled(12 * MIB, 8, 2)
    res = np.zeros((len(data), 64), dtype=np.uint64)
    try:
        for k, d in enumerate(data):
            pp.pospop_server_submit_host(srv, (8, 16, 32, 64, 8)[k], d, d.size, res[k])
        assert pp.pospop_server_drain(srv, 30000) == pp.POSPOP_OK
        assert pp.pospop_server_pool_stats(srv)[1] == 0
    finally:
        pp.pospop_server_destroy(srv)
    for k, d in enumerate(data):
        w = (8, 16, 32, 64, 8)[k]
        assert np.array_equal(res[k, :w], orc.bytes(w, d)), k


def test_resident_grid_stops_when_idle_and_restarts(gpu, orc, pool, serve_tune):
    """serve_mode 3: the resident grid is told to leave after the idle time
    (200 us here) and launched again for the next requests; every result of
    both rounds equals the oracle's."""
    import time
    serve_tune("serve_mode 3", "serve_resident 200 200000")
    host = pool.cpu().numpy()
    srv = pp.pospop_server_create(1 << 30, 64, 2)
    try:
        for rnd in range(2):
            n0 = pp.pospopcnt_launch_count()
            w, nbytes, offs = _requests(40, 31 + rnd, 1, 4 * MIB, 256 * MIB)
            res = np.zeros((40, 64), dtype=np.uint64)
            for k in range(40):
                pp.pospop_server_submit(srv, int(w[k]), pool.data_ptr() + int(offs[k]),
                                        int(nbytes[k]), res[k])
            assert pp.pospop_server_drain(srv, 10000) == pp.POSPOP_OK
            recs = pp.pospop_server_poll(srv, 64, timeout_ms=100)
            assert len(recs) == 40 and all(r.status == 0 for r in recs)
            assert pp.pospopcnt_launch_count() > n0        # a grid was launched this round
            for k in range(40):
                seg = host[int(offs[k]):int(offs[k]) + int(nbytes[k])]
                assert np.array_equal(res[k, :w[k]], orc.bytes(int(w[k]), seg)), (rnd, k)
            time.sleep(0.02)                               # the grid leaves meanwhile
    finally:
        pp.pospop_server_destroy(srv)


def test_resident_grid_wait_runs_out(gpu, orc, pool, serve_tune):
    """serve_mode 3 with a 1 us limit on the grid's wait for a new run: the
    grid keeps leaving on its own (its bounded wait runs out), the server
    fails exactly the requests whose items were published but not counted
    (POSPOP_ETIMEDOUT), every other request completes with the oracle's
    counts, and with the normal limit the next requests all complete."""
    serve_tune("serve_mode 3", "serve_resident 1000000 1")
    host = pool.cpu().numpy()
    n = 300
    w, nbytes, offs = _requests(n, 41, 1, 2 * MIB, 256 * MIB)
    srv = pp.pospop_server_create(1 << 30, 256, 2)
    try:
        results = np.zeros((n, 64), dtype=np.uint64)
        recs = pp.pospop_server_run_trace(srv, (np.arange(n) * 20000).astype(np.int64), w,
                                          pool.data_ptr() + offs, nbytes, results)
        st = recs["status"]
        assert set(np.unique(st).tolist()) <= {pp.POSPOP_OK, pp.POSPOP_ETIMEDOUT}
        for k in np.nonzero(st == pp.POSPOP_OK)[0]:
            seg = host[int(offs[k]):int(offs[k]) + int(nbytes[k])]
            assert np.array_equal(results[k, :w[k]], orc.bytes(int(w[k]), seg)), k
        serve_tune("serve_mode 3", "serve_resident 2000 200000")
        w2, nb2, off2 = _requests(100, 42, 1, 2 * MIB, 256 * MIB)
        res2 = np.zeros((100, 64), dtype=np.uint64)
        recs2 = pp.pospop_server_run_trace(srv, (np.arange(100) * 2000).astype(np.int64), w2,
                                           pool.data_ptr() + off2, nb2, res2)
        assert (recs2["status"] == 0).all()
        for k in range(100):
            seg = host[int(off2[k]):int(off2[k]) + int(nb2[k])]
            assert np.array_equal(res2[k, :w2[k]], orc.bytes(int(w2[k]), seg)), k
    finally:
        pp.pospop_server_destroy(srv)


def test_lone_large_request(gpu, orc, pool, mode):
    """One 128 MiB request on an idle server (its work items are spread over
    every SM): the result equals the oracle's count."""
    srv = pp.pospop_server_create(1 << 30, 16, 2)
    try:
        res = np.zeros(64, dtype=np.uint64)
        p0 = pool.data_ptr() + 13
        pp.pospop_server_submit(srv, 16, p0, 128 * MIB, res)
        assert pp.pospop_server_drain(srv, 10000) == pp.POSPOP_OK
        recs = pp.pospop_server_poll(srv, timeout_ms=100)
        assert len(recs) == 1 and recs[0].status == 0
    finally:
        pp.pospop_server_destroy(srv)
    seg = pool[13:13 + 128 * MIB].cpu().numpy()
    assert np.array_equal(res[:16], orc.bytes(16, seg))


def test_class_streams_and_cap_entries(gpu, pool, serve_tune):
    """`serve 3 0 127 1 1`: requests from 128 MiB run one batch at a time, one
    request a batch; `serve 0 8 127 64 2`: small requests at most two a batch."""
    serve_tune("serve_mode 0", "serve 3 0 127 1 1", "serve 0 8 127 64 2")
    nb, ns = 12, 40
    w = np.concatenate([np.full(nb, 32), np.full(ns, 8)]).astype(np.int32)
    nbytes = np.concatenate([np.full(nb, 128 * MIB), np.full(ns, 4096)]).astype(np.uint64)
    offs = np.concatenate([np.arange(nb) % 3 * 32 * MIB, np.arange(ns) * 4099]).astype(np.uint64)
    arrival = np.zeros(nb + ns, dtype=np.int64)
    srv = pp.pospop_server_create(64 << 30, 4096, 8)
    try:
        results = np.zeros((nb + ns, 64), dtype=np.uint64)
        recs = pp.pospop_server_run_trace(srv, arrival, w, pool.data_ptr() + offs, nbytes, results)
    finally:
        pp.pospop_server_destroy(srv)
    assert (recs["status"] == 0).all()
    big = recs[:nb]
    order = np.argsort(big["t_launch_ns"])
    launches = big["t_launch_ns"][order].astype(np.int64)
    dones = big["t_done_ns"][order].astype(np.int64)
    assert len(set(launches.tolist())) == nb                 # one request per batch
    assert (launches[1:] >= dones[:-1]).all()                # one batch at a time
    small = recs[nb:]
    _, per_launch = np.unique(small["t_launch_ns"], return_counts=True)
    assert per_launch.max() <= 2
    solo = _solo(pool, w, nbytes, offs)
    for k in range(nb + ns):
        assert np.array_equal(results[k, :w[k]], solo[k, :w[k]]), k


def test_host_input_admitted_by_pool_space(gpu, orc, mode):
    """A pooled server stages host input into its device pool: with a budget
    (the pool) far smaller than the sum of the requests, admission waits for
    pool space, the pool's high-water mark stays within the budget, and every
    result equals the oracle's count.  Pinned and pageable sources mixed."""
    budget = 48 * MIB
    n = 60
    sizes = synth.log_uniform_sizes(n, 1 * MIB, 16 * MIB, seed=31)
    sizes[::11] = 0
    sizes[5::13] = 4099
    widths = np.array([8, 16, 32, 64, 1, 4], dtype=np.int32)[np.arange(n) % 6]
    bufs = []
    for k in range(n):
        data = synth.random_bytes(int(sizes[k]) + 3, seed=400 + k)[3:]
        if k % 2:
            t = torch.empty(data.size, dtype=torch.uint8, pin_memory=True)
            t.numpy()[:] = data
            bufs.append((t, data))
        else:
            bufs.append((data, data))
    assert int(sizes.sum()) > 4 * budget
    srv = pp.pospop_server_create_pooled(budget, 4096, 4)
    results = np.zeros((n, 64), dtype=np.uint64)
    try:
        ids = [pp.pospop_server_submit_host(srv, int(widths[k]), bufs[k][0], int(sizes[k]),
                                            results[k]) for k in range(n)]
        assert pp.pospop_server_drain(srv, 60000) == pp.POSPOP_OK
        recs = []
        while len(recs) < n:
            got = pp.pospop_server_poll(srv, n, 1000)
            assert got
            recs += got
        pool_bytes, used, hwm = pp.pospop_server_pool_stats(srv)
    finally:
        pp.pospop_server_destroy(srv)
    assert pool_bytes == budget and used == 0 and 0 < hwm <= budget
    by_id = {r.id: r for r in recs}
    rec = [by_id[i] for i in ids]
    assert all(r.status == 0 for r in rec)
    # admission waited for space: admitted bytes in flight never exceed the budget,
    # and some request was admitted only after another had finished
    ev = sorted([(r.t_admit_ns, int(r.nbytes)) for r in rec] + [(r.t_done_ns, -int(r.nbytes)) for r in rec],
                key=lambda x: (x[0], x[1]))
    cur = peak = 0
    for _, d in ev:
        cur += d
        peak = max(peak, cur)
    assert peak <= budget
    assert max(r.t_admit_ns for r in rec) > min(r.t_done_ns for r in rec)
    for k in range(n):
        w = int(widths[k])
        assert np.array_equal(results[k, :w], orc.bytes(w, bufs[k][1])), k


def test_pooled_server_errors_and_device_requests(gpu, orc, pool):
    srv = pp.pospop_server_create(1 * MIB, 4, 1)
    try:
        host = np.zeros(64, dtype=np.uint8)
        rc = pp.lib().pospop_server_submit_host(srv, 8, host.ctypes.data, 64, None, None)
        assert rc == pp.POSPOP_EINVAL                   # not a pooled server
        assert pp.pospop_server_pool_stats(srv) == (0, 0, 0)
    finally:
        pp.pospop_server_destroy(srv)
    srv = pp.pospop_server_create_pooled(4 * MIB, 64, 2)
    try:
        L = pp.lib()
        host = np.zeros(64, dtype=np.uint8)
        assert L.pospop_server_submit_host(srv, 8, pool.data_ptr(), 64, None,
                                           None) == pp.POSPOP_EPTR
        assert L.pospop_server_submit_host(srv, 8, host.ctypes.data, 5 * MIB, None,
                                           None) == pp.POSPOP_ERANGE
        # device-pointer requests still work on a pooled server, beside host ones
        r_dev = np.zeros(64, dtype=np.uint64)
        r_host = np.zeros(64, dtype=np.uint64)
        data = synth.random_bytes(3 * MIB + 5, seed=71)
        pp.pospop_server_submit(srv, 32, pool.data_ptr() + 7, 3 * MIB, r_dev)
        pp.pospop_server_submit_host(srv, 16, data, data.size, r_host)
        assert pp.pospop_server_drain(srv, 10000) == pp.POSPOP_OK
        assert pp.pospop_server_pool_stats(srv)[1] == 0
    finally:
        pp.pospop_server_destroy(srv)
    assert np.array_equal(r_dev[:32], orc.bytes(32, pool[7:7 + 3 * MIB].cpu().numpy()))
    assert np.array_equal(r_host[:16], orc.bytes(16, data))


def test_errors_and_bounded_waits(gpu, pool, mode):
    srv = pp.pospop_server_create(1 * MIB, 4, 1)
    try:
        L = pp.lib()
        import ctypes
        rid = ctypes.c_uint64()
        res = np.zeros(64, dtype=np.uint64)
        assert L.pospop_server_submit(srv, 16, pool.data_ptr(), 2 * MIB, res.ctypes.data,
                                      ctypes.byref(rid)) == pp.POSPOP_ERANGE
        assert L.pospop_server_submit(srv, 12, pool.data_ptr(), 16, res.ctypes.data,
                                      ctypes.byref(rid)) == pp.POSPOP_EINVAL
        host = np.zeros(64, dtype=np.uint8)
        assert L.pospop_server_submit(srv, 8, host.ctypes.data, 64, res.ctypes.data,
                                      ctypes.byref(rid)) == pp.POSPOP_EPTR
        # nothing submitted: a poll times out, a drain returns at once
        assert pp.pospop_server_poll(srv, timeout_ms=50) == []
        assert pp.pospop_server_drain(srv, 1000) == pp.POSPOP_OK
        # an empty request completes with zero counts
        res[:] = 7
        pp.pospop_server_submit(srv, 8, None, 0, res)
        assert pp.pospop_server_drain(srv, 5000) == pp.POSPOP_OK
        recs = pp.pospop_server_poll(srv, timeout_ms=100)
        assert len(recs) == 1 and recs[0].status == 0
        assert not res[:8].any() and (res[8:] == 7).all()
    finally:
        pp.pospop_server_destroy(srv)


def test_small_requests_overtake_large_ones(gpu, pool, mode):
    """Small requests that arrive while large ones run finish long before
    them: on a higher-priority stream (size classes), or at the next launch
    (dispatch by remaining bytes)."""
    lo_prio, hi_prio = torch.cuda.Stream.priority_range()
    if mode == 0 and lo_prio == hi_prio:
        pytest.skip("device has a single stream priority level")
    nb, ns = 64, 64        # 8 GiB of large requests (about 1.1 ms), small ones at 0.2..0.52 ms
    w = np.concatenate([np.full(nb, 16), np.full(ns, 8)]).astype(np.int32)
    nbytes = np.concatenate([np.full(nb, 128 * MIB), np.full(ns, 16384)]).astype(np.uint64)
    offs = np.concatenate([np.arange(nb) % 2 * 64 * MIB,
                           (np.arange(ns) * 16411) % (128 * MIB)]).astype(np.uint64)
    arrival = np.concatenate([np.zeros(nb), 200_000 + np.arange(ns) * 5000]).astype(np.int64)
    srv = pp.pospop_server_create(64 << 30, 4096, 4)
    try:
        results = np.zeros((nb + ns, 64), dtype=np.uint64)
        recs = pp.pospop_server_run_trace(srv, arrival, w, pool.data_ptr() + offs, nbytes, results)
    finally:
        pp.pospop_server_destroy(srv)
    assert (recs["status"] == 0).all()
    solo = _solo(pool, w, nbytes, offs)
    for k in range(nb + ns):
        assert np.array_equal(results[k, :w[k]], solo[k, :w[k]]), k
    t0 = int(recs["t_submit_ns"].min())
    big_done = int(recs["t_done_ns"][:nb].max())
    small_done = recs["t_done_ns"][nb:].astype(np.int64)
    small_lat = small_done - recs["t_submit_ns"][nb:].astype(np.int64)
    assert small_done.max() < big_done
    assert np.median(small_lat) < 0.25 * (big_done - t0)


def test_every_width_in_one_mix(gpu, orc, pool, mode):
    """Requests of widths 1, 2, 4, 8, 16, 32 and 64 in the same batches."""
    n = 700
    widths = np.array([1, 2, 4, 8, 16, 32, 64], dtype=np.int32)
    w = widths[np.arange(n) % len(widths)]
    rng = np.random.default_rng(17)
    nbytes = synth.log_uniform_sizes(n, 1, 2 * MIB, seed=18).astype(np.uint64)
    offs = rng.integers(0, 64 * MIB, n).astype(np.uint64)
    srv = pp.pospop_server_create(1 << 30, 256, 2)
    try:
        results = np.zeros((n, 64), dtype=np.uint64)
        recs = pp.pospop_server_run_trace(srv, (np.arange(n) * 3000).astype(np.int64), w,
                                          pool.data_ptr() + offs, nbytes, results)
    finally:
        pp.pospop_server_destroy(srv)
    assert (recs["status"] == 0).all()
    host = pool.cpu().numpy()
    for k in range(n):
        seg = host[int(offs[k]):int(offs[k]) + int(nbytes[k])]
        assert np.array_equal(results[k, :w[k]], orc.bytes(int(w[k]), seg)), (k, int(w[k]))
