"""GPU tests of the request server (continuous batching, Sec. 3.2.3 job management).

Every served result must be the same as the oracle's and as the same request
run alone (exactly: digests and boundaries are integers / bytes).
"""
import time

import numpy as np
import pytest
import torch

import oracle
from gen import inputs as G

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hg():
    import paper_1202_3669_b300 as hgb
    ctx = hgb.Context(0)
    yield ctx
    ctx.close()


def mixed_requests(count, seed, median=48 * 1024, hi=6 << 20):
    """70 % chunking + MD5, 30 % 64 KiB-block SHA-1 with root; log-normal sizes."""
    import paper_1202_3669_b300 as hgb
    sizes = G.lognormal_sizes(count, seed, median=median, sigma=1.8, hi=hi)
    g = G.rng(seed + 1)
    reqs = []
    for i, sz in enumerate(sizes):
        data = G.uniform_bytes(int(sz), seed * 1000 + i)
        if g.random() < 0.7:
            reqs.append((data, hgb.HG_REQ_CDC, hgb.MD5, 0, False))
        else:
            reqs.append((data, hgb.HG_REQ_BLOCKS, hgb.SHA1, 65536, True))
    return reqs


def expected(req):
    import paper_1202_3669_b300 as hgb
    data, kind, algo, block, root = req
    if kind == hgb.HG_REQ_CDC:
        ends = oracle.cdc(data, nthreads=8)
        return ends, oracle.hash_chunks(algo, data, ends), None
    dg, rt = oracle.hash_blocks(algo, data, block)
    return None, dg, rt


def check_result(req, res):
    import paper_1202_3669_b300 as hgb
    ends, dg, rt = expected(req)
    assert res["status"] == 0
    if req[1] == hgb.HG_REQ_CDC:
        assert np.array_equal(res["ends"].astype(np.uint64), ends)
    assert np.array_equal(res["digests"], dg)
    if rt is not None:
        assert res["root"] == rt


def test_mix_equals_alone_and_oracle(hg):
    import paper_1202_3669_b300 as hgb
    reqs = mixed_requests(80, seed=5)
    srv = hgb.Server(hg, device_budget=2 << 30, max_wave_bytes=64 << 20, max_wave_requests=32)
    tickets = [srv.submit(*r) for r in reqs]           # all at once: they batch and overlap
    mix = [srv.poll(t) for t in tickets]
    st = srv.stats()
    assert st["completed"] == len(reqs) and st["waves"] >= 2
    alone = []
    for r in reqs:                                      # one at a time: each is its own wave
        alone.append(srv.poll(srv.submit(*r)))
    srv.close()
    for r, a, b in zip(reqs, mix, alone):
        check_result(r, a)
        assert a["count"] == b["count"]
        assert np.array_equal(a["digests"], b["digests"])
        if a["ends"] is not None:
            assert np.array_equal(a["ends"], b["ends"])
        assert a["root"] == b["root"]
        assert a["t_submit_ns"] <= a["t_admit_ns"] <= a["t_done_ns"]


def test_wave_target_splits_waves_and_keeps_results(hg):
    """A small per-wave byte target closes waves early (more, smaller waves); a request
    larger than the target but within max_wave_bytes still runs, in a wave of its own.
    Results are unchanged."""
    import paper_1202_3669_b300 as hgb
    reqs = mixed_requests(40, seed=11)
    reqs.append((G.uniform_bytes((3 << 20) + 5, 999), hgb.HG_REQ_CDC, hgb.MD5, 0, False))
    total = sum(r[0].size for r in reqs)
    target = 1 << 20
    srv = hgb.Server(hg, device_budget=2 << 30, max_wave_bytes=64 << 20, wave_target_bytes=target)
    assert srv.cfg.wave_target_bytes == target
    tickets = [srv.submit(*r) for r in reqs]
    res = [srv.poll(t) for t in tickets]
    st = srv.stats()
    srv.close()
    for r, x in zip(reqs, res):
        check_result(r, x)
    # every wave but those holding one large request carries at most `target` bytes
    assert st["waves"] >= total // (target + (6 << 20))
    assert st["completed"] == len(reqs)


def test_admission_under_small_budget(hg):
    """The arena holds only a few requests at once; everything still completes exactly."""
    import paper_1202_3669_b300 as hgb
    srv = hgb.Server(hg, device_budget=34 << 20, max_wave_bytes=8 << 20, max_wave_requests=8,
                     max_inflight_waves=2)
    reqs = [(G.uniform_bytes(6 << 20, 300 + i), hgb.HG_REQ_CDC, hgb.MD5, 0, False)
            for i in range(12)]
    tickets = [srv.submit(*r) for r in reqs]
    for r, t in zip(reqs, tickets):
        check_result(r, srv.poll(t))
    st = srv.stats()
    assert st["arena_used"] == 0 and st["completed"] == 12
    srv.close()


def test_oversized_request_refused(hg):
    import paper_1202_3669_b300 as hgb
    srv = hgb.Server(hg, device_budget=256 << 20, max_wave_bytes=16 << 20)
    big = np.zeros((16 << 20) + 1, np.uint8)
    with pytest.raises(hgb.HashGPUError) as e:
        srv.submit(big)
    assert e.value.status == hgb._lib.HG_ENOMEM
    srv.close()


def test_cancel_and_nonblocking_poll(hg):
    import paper_1202_3669_b300 as hgb
    srv = hgb.Server(hg, device_budget=200 << 20, max_wave_bytes=32 << 20, max_wave_requests=1,
                     max_inflight_waves=1)
    reqs = [(G.uniform_bytes(24 << 20, 400 + i), hgb.HG_REQ_CDC, hgb.MD5, 0, False)
            for i in range(6)]
    tickets = [srv.submit(*r) for r in reqs]
    rc_last = srv.cancel(tickets[-1])                   # queued behind five 24 MiB requests
    assert rc_last in (0, hgb._lib.HG_EAGAIN)
    first = srv.poll(tickets[0], timeout_us=0)          # may or may not be done yet
    if first is not None:
        check_result(reqs[0], first)
    else:
        check_result(reqs[0], srv.poll(tickets[0]))
    for r, t in zip(reqs[1:-1], tickets[1:-1]):
        check_result(r, srv.poll(t))
    last = srv.poll(tickets[-1])
    if rc_last == 0:
        assert last["status"] == hgb._lib.HG_ECANCELED
    else:
        check_result(reqs[-1], last)
    srv.close()


def test_destroy_with_queued_requests(hg):
    import paper_1202_3669_b300 as hgb
    srv = hgb.Server(hg, device_budget=200 << 20, max_wave_bytes=32 << 20, max_wave_requests=1,
                     max_inflight_waves=1)
    keep = [G.uniform_bytes(20 << 20, 500 + i) for i in range(5)]
    for d in keep:
        srv.submit(d)
    t0 = time.time()
    srv.close()                                         # cancels the queue, drains the GPU
    assert time.time() - t0 < 30


def test_replay_trace(hg):
    import paper_1202_3669_b300 as hgb
    reqs = mixed_requests(200, seed=9, median=16 * 1024, hi=1 << 20)
    srv = hgb.Server(hg, device_budget=1 << 30, max_wave_bytes=64 << 20)
    pinned = [torch.from_numpy(r[0]).pin_memory() for r in reqs]
    rq = [srv.make_request(p, r[1], r[2], r[3], r[4]) for p, r in zip(pinned, reqs)]
    arrivals = (G.poisson_arrivals(2000.0, len(rq), seed=10) * 1e9).astype(np.uint64)
    lat, span = srv.replay(rq, arrivals)
    assert (lat > 0).all() and span >= arrivals[-1]
    assert srv.stats()["completed"] == len(rq)
    srv.close()


def test_pinned_inputs_gathered_by_kernel(hg):
    """Inputs in pinned host memory (slices at odd offsets of one pinned pool, as a
    service would hold them, starting at every residue mod 16) take the gather
    kernel up to 2 MiB (in 256 KiB pieces) and copy calls above; both land exactly."""
    import paper_1202_3669_b300 as hgb
    pool_np = G.uniform_bytes(24 << 20, seed=901)
    pool = torch.from_numpy(pool_np).pin_memory()
    g = np.random.default_rng(902)
    sizes = [1, 2, 3, 4, 5, 63, 64, 65, 4095, 4097, 100_000, 511 << 10, 512 << 10, (512 << 10) + 1,
             (256 << 10) + 17, (2 << 20) - 1, 2 << 20, (2 << 20) + 1, 3 << 20] + g.integers(1, 600_000, 40).tolist()
    srv = hgb.Server(hg, device_budget=1 << 30, max_wave_bytes=32 << 20, max_wave_requests=64)
    reqs = []
    for i, z in enumerate(sizes):
        off = int(g.integers(0, pool_np.size - z - 16))
        off += (i - off) % 16                          # every start residue mod 16 in turn
        view = pool[off:off + z]
        kind = hgb.HG_REQ_CDC if i % 3 else hgb.HG_REQ_BLOCKS
        reqs.append((pool_np[off:off + z], view, kind))
    tickets = []
    for _, view, kind in reqs:
        if kind == hgb.HG_REQ_CDC:
            tickets.append(srv.submit(view, kind, hgb.MD5))
        else:
            tickets.append(srv.submit(view, kind, hgb.SHA1, 4096, True))
    for (data, _, kind), t in zip(reqs, tickets):
        res = srv.poll(t)
        assert res["status"] == 0
        if kind == hgb.HG_REQ_CDC:
            want = oracle.cdc(data, nthreads=8)
            assert np.array_equal(res["ends"].astype(np.uint64), want)
            assert np.array_equal(res["digests"], oracle.hash_chunks(oracle.MD5, data, want))
        else:
            dg, rt = oracle.hash_blocks(oracle.SHA1, data, 4096)
            assert np.array_equal(res["digests"], dg) and res["root"] == rt
    srv.close()
