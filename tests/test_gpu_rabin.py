"""GPU parity of the Rabin fingerprint window (HG_WIN_RABIN) against the CPU oracle.

The window bitmap, candidates, boundaries and chunk digests are integer
results: every comparison is exact. The interior fast path (aligned input,
specialised window lengths) and the byte-load path (edges, unaligned input,
other window lengths) are both covered.
"""

import numpy as np
import pytest
import torch

import oracle
from gen import inputs as G
from tests.gpu_util import bitmap_to_cuts, oracle_digests_parallel, to_device
from tests.pins import check_chunking

pytestmark = pytest.mark.gpu
R = oracle.WIN_RABIN


@pytest.fixture(scope="module")
def hg():
    import paper_1202_3669_b300 as hgb
    ctx = hgb.Context(0)
    yield ctx
    ctx.close()


def P(**kw):
    import paper_1202_3669_b300 as hgb
    kw.setdefault("window", 48)
    return hgb.params(window_hash=hgb.WIN_RABIN, **kw)


SIZES = [0, 1, 47, 48, 49, 100, 8191, 8192, 32768, 32769, 8192 * 7 + 77, 300_001, (1 << 20) + 13]
WINDOWS = [(48, 6, 0x2A), (16, 5, 0x11), (20, 4, 0x3), (24, 5, 0x1F), (32, 6, 0x20), (64, 5, 0),
           (1, 3, 0x5), (7, 4, 0xA), (33, 6, 0x21), (55, 5, 0x1), (48, 13, 0x0F0F)]


@pytest.mark.parametrize("n", SIZES)
@pytest.mark.parametrize("window,mask_bits,magic", WINDOWS)
def test_window_bitmap(hg, n, window, mask_bits, magic):
    data = G.uniform_bytes(n, seed=n * 5 + window)
    want = oracle.window_candidates(data, window, mask_bits, magic, nthreads=8, kind=R)
    for off in (0, 3):
        bm = hg.window_bitmap(to_device(data, off), P(window=window, mask_bits=mask_bits, magic=magic))
        got = bitmap_to_cuts(bm, n)
        assert np.array_equal(got, want), (off, got[:10], want[:10])
    hg.sync()


@pytest.mark.parametrize("n", [0, 5000, 3 << 20, (20 << 20) + 12345])
@pytest.mark.parametrize("algo", [oracle.MD5, oracle.SHA1])
def test_cdc_hash(hg, n, algo):
    data = G.uniform_bytes(n, seed=n + 17)
    ends, cnt, dg = hg.cdc_hash(to_device(data, 0 if n % 2 else 5), algo, P(mask_bits=13, magic=0x0F0F))
    hg.sync()
    k = int(cnt.item())
    cands = oracle.window_candidates(data, 48, 13, 0x0F0F, nthreads=16, kind=R)
    want = oracle.select(cands, data.size, 2048, 65536)
    assert np.array_equal(ends[:k].cpu().numpy().astype(np.uint64), want)
    check_chunking(want.tolist(), cands.tolist(), n, 2048, 65536)
    assert np.array_equal(dg[:k].cpu().numpy(), oracle.hash_chunks(algo, data, want))


def test_cdc_segmented_text_like(hg):
    """Above 64 MiB hg_cdc_hash runs segments with a carried open chunk."""
    data = G.text_like_bytes((70 << 20) + 333, seed=5)
    p = P(window=32, mask_bits=11, magic=0x155, min_chunk=512, max_chunk=16384)
    ends, cnt, dg = hg.cdc_hash(to_device(data), oracle.MD5, p)
    hg.sync()
    k = int(cnt.item())
    want = oracle.cdc(data, 32, 11, 0x155, 512, 16384, nthreads=16, kind=R)
    assert np.array_equal(ends[:k].cpu().numpy().astype(np.uint64), want)
    assert np.array_equal(dg[:k].cpu().numpy(), oracle.hash_chunks(oracle.MD5, data, want))


def test_boundaries_dense_and_static(hg):
    data = G.uniform_bytes((3 << 20) + 7, seed=19)
    p = P(window=24, mask_bits=2, magic=1, min_chunk=64, max_chunk=4096)    # list overflows
    want = oracle.cdc(data, 24, 2, 1, 64, 4096, nthreads=16, kind=R)
    ends, cnt = hg.cdc_boundaries(to_device(data), p)
    hg.sync()
    assert np.array_equal(ends[:int(cnt.item())].cpu().numpy().astype(np.uint64), want)
    import ctypes as C
    from paper_1202_3669_b300 import _lib
    d1 = to_device(data, 1)
    cap = data.size // 64 + 2
    e_st = torch.empty(cap, dtype=torch.int64, device="cuda")
    c_st = torch.zeros(1, dtype=torch.int64, device="cuda")
    rc = _lib.lib.hg_cdc_boundaries_static(d1.data_ptr(), data.size, C.byref(p), e_st.data_ptr(),
                                           cap, c_st.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert rc == 0
    torch.cuda.synchronize()
    assert np.array_equal(e_st[:int(c_st.item())].cpu().numpy().astype(np.uint64), want)


def test_stream_equals_one_shot(hg):
    import paper_1202_3669_b300 as hgb
    data = G.uniform_bytes((9 << 20) + 5, seed=23)
    p = P()
    want = oracle.cdc(data, 48, 13, 0x0F0F, nthreads=16, kind=R)
    st = hgb.CdcStream(hg, hgb.SHA1, p, max_feed=4 << 20)
    d = to_device(data)
    rng = np.random.default_rng(5)
    pos, ends, digs = 0, [], []
    while pos < data.size:
        k = int(min(data.size - pos, rng.integers(1, 4 << 20)))
        e, g = st.feed(d[pos:pos + k])
        ends.append(e); digs.append(g)
        pos += k
    e, g = st.close()
    ends.append(e); digs.append(g)
    got = np.concatenate([x.cpu().numpy().astype(np.uint64) for x in ends])
    assert np.array_equal(got, want)
    dg = np.concatenate([x.cpu().numpy() for x in digs])
    assert np.array_equal(dg, oracle.hash_chunks(oracle.SHA1, data, want))


def test_config_rabin_1gib(hg):
    """1 GiB uniform (seed 4), default Rabin parameters (48-byte window), compared in
    full: the whole candidate list, every chunk end and every chunk digest of one
    hg_cdc_hash call equal the oracle's, computed on all host cores."""
    import os
    n = 1 << 30
    data = G.uniform_bytes(n, seed=4)
    d = to_device(data)
    p = P()
    cands, ccnt = hg.cdc_candidates(d, p, cap=n // 1024)
    ends, cnt, dg = hg.cdc_hash(d, oracle.MD5, p)
    hg.sync()
    got_c = cands[:int(ccnt.item())].cpu().numpy().astype(np.uint64)
    k = int(cnt.item())
    got_e = ends[:k].cpu().numpy().astype(np.uint64)
    got_d = dg[:k].cpu().numpy()
    del d, cands, ends, dg
    want_c = oracle.window_candidates(data, 48, 13, 0x0F0F, nthreads=os.cpu_count() or 1, kind=R)
    assert np.array_equal(got_c, want_c)
    want_e = oracle.select(want_c, n, 2048, 65536)
    assert np.array_equal(got_e, want_e)
    assert np.array_equal(got_d, oracle_digests_parallel(oracle.MD5, data, want_e))


@pytest.mark.parametrize("algo", [oracle.MD5, oracle.SHA1])
@pytest.mark.parametrize("offset", [0, 5])
def test_batch(hg, algo, offset):
    """Batched Rabin chunking (per-file tiles, files at any offset) equals each file alone."""
    import paper_1202_3669_b300 as hgb
    sizes = np.array([0, 1, 47, 48, 49, 100, 2047, 8192, 8193, 70_000, 0, 300_000, (1 << 20) + 77,
                      2_500_000, 65_537] + G.lognormal_sizes(120, seed=41, median=30_000, sigma=1.4,
                                                           hi=3 << 20).tolist(), dtype=np.int64)
    data, off = G.files_from_sizes(sizes, 42)
    p = P()
    b = hgb.Batch(hg, off, p)
    out = b.cdc_hash(to_device(data, offset), algo, graph=bool(offset))
    b.sync()
    for f in range(len(sizes)):
        body = data[off[f]:off[f + 1]]
        want = oracle.cdc(body, 48, 13, 0x0F0F, 2048, 65536, nthreads=8, kind=R)
        ends, dg = b.file_results(f, *out)
        assert np.array_equal(ends, want), (f, sizes[f])
        assert np.array_equal(dg, oracle.hash_chunks(algo, body, want)), f
    b.close()


def test_batch_other_window_dense(hg):
    import paper_1202_3669_b300 as hgb
    sizes = G.lognormal_sizes(40, seed=43, median=60_000, sigma=1.0, hi=1 << 20)
    data, off = G.files_from_sizes(sizes, 44)
    p = P(window=33, mask_bits=3, magic=2, min_chunk=100, max_chunk=1000)
    b = hgb.Batch(hg, off, p)
    out = b.cdc_hash(to_device(data, 1), hgb.MD5)
    b.sync()
    for f in range(len(sizes)):
        body = data[off[f]:off[f + 1]]
        want = oracle.cdc(body, 33, 3, 2, 100, 1000, nthreads=8, kind=R)
        ends, dg = b.file_results(f, *out)
        assert np.array_equal(ends, want), f
        assert np.array_equal(dg, oracle.hash_chunks(oracle.MD5, body, want)), f
    b.close()


def test_server(hg):
    """A server whose chunking requests use the Rabin window: exact per request."""
    import paper_1202_3669_b300 as hgb
    srv = hgb.Server(hg, device_budget=512 << 20, max_wave_bytes=32 << 20, max_wave_requests=16, p=P())
    sizes = G.lognormal_sizes(30, seed=45, median=50_000, sigma=1.6, hi=4 << 20)
    reqs = [(G.uniform_bytes(int(z), 4600 + i), hgb.HG_REQ_CDC, hgb.SHA1 if i % 2 else hgb.MD5, 0, False)
            for i, z in enumerate(sizes)]
    tickets = [srv.submit(*r) for r in reqs]
    for (data, _, algo, _, _), t in zip(reqs, tickets):
        res = srv.poll(t)
        assert res["status"] == 0
        want = oracle.cdc(data, 48, 13, 0x0F0F, 2048, 65536, nthreads=8, kind=R)
        assert np.array_equal(res["ends"].astype(np.uint64), want)
        assert np.array_equal(res["digests"], oracle.hash_chunks(algo, data, want))
    srv.close()
