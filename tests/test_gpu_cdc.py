"""GPU parity of content-based chunking (Sec. 2.1, Sec. 3.2.2, Fig. 3) against the oracle.

Window candidates, compaction and boundary offsets are integer results and
must match exactly; chunk digests byte for byte.
"""
import numpy as np
import pytest
import torch

import oracle
from gen import inputs as G
from tests.gpu_util import bitmap_to_cuts, oracle_digests_parallel, to_device
from tests.pins import check_chunking

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hg():
    import paper_1202_3669_b300 as hgb
    ctx = hgb.Context(0)
    yield ctx
    ctx.close()


def P(**kw):
    import paper_1202_3669_b300 as hgb
    return hgb.params(**kw)


SIZES = [0, 1, 19, 20, 21, 100, 8191, 8192, 8193, 8192 * 3 + 77, 100_000, (1 << 20) + 13]
WINDOWS = [(20, 6, 0x2A), (16, 5, 0x11), (17, 5, 0x3), (1, 3, 0x5), (55, 6, 0x3F), (48, 5, 0),
           (32, 4, 0xA), (24, 5, 0x1F), (33, 6, 0x20), (20, 13, 0x0F0F)]


@pytest.mark.parametrize("n", SIZES)
@pytest.mark.parametrize("window,mask_bits,magic", WINDOWS)
def test_window_bitmap(hg, n, window, mask_bits, magic):
    data = G.uniform_bytes(n, seed=n * 7 + window)
    for off in (0, 3):
        bm = hg.window_bitmap(to_device(data, off), P(window=window, mask_bits=mask_bits, magic=magic))
        got = bitmap_to_cuts(bm, n)
        want = oracle.window_candidates(data, window, mask_bits, magic, nthreads=8)
        assert np.array_equal(got, want), (off, got[:10], want[:10])
    hg.sync()


@pytest.mark.parametrize("n", [0, 50, 8192 * 5 + 3, 300_000, (2 << 20) + 1])
@pytest.mark.parametrize("mask_bits", [3, 8, 13])
def test_candidates(hg, n, mask_bits):
    data = G.uniform_bytes(n, seed=n + mask_bits)
    cands, cnt = hg.cdc_candidates(to_device(data), P(mask_bits=mask_bits, magic=1), cap=n + 8)
    c = int(cnt.item())
    want = oracle.window_candidates(data, 20, mask_bits, 1, nthreads=8)
    assert c == want.size
    assert np.array_equal(cands[:c].cpu().numpy().astype(np.uint64), want)
    hg.sync()


def test_candidates_capacity(hg):
    data = G.uniform_bytes(200_000, seed=3)
    want = oracle.window_candidates(data, 20, 6, 1, nthreads=8)
    cands, cnt = hg.cdc_candidates(to_device(data), P(mask_bits=6, magic=1), cap=10)
    assert int(cnt.item()) == want.size > 10
    assert np.array_equal(cands[:10].cpu().numpy().astype(np.uint64), want[:10])
    hg.sync()


def run_cdc(hg, data, algo=oracle.MD5, offset=0, **kw):
    p = P(**kw)
    d = to_device(data, offset)
    ends, cnt, dg = hg.cdc(d, algo, p)
    c = int(cnt.item())
    hg.sync()
    return ends[:c].cpu().numpy().astype(np.uint64), dg[:c].cpu().numpy()


@pytest.mark.parametrize("n", [0, 1, 2047, 2048, 2049, 65536, 65537, 200_000, (1 << 20) + 5])
@pytest.mark.parametrize("kw", [dict(), dict(mask_bits=9, magic=0x55, min_chunk=700, max_chunk=5000),
                                dict(window=16, mask_bits=8, magic=3, min_chunk=1, max_chunk=300)])
@pytest.mark.parametrize("offset", [0, 5])
def test_cdc_small(hg, n, kw, offset):
    data = G.uniform_bytes(n, seed=n + 99)
    q = dict(window=20, mask_bits=13, magic=0x0F0F, min_chunk=2048, max_chunk=65536)
    q.update(kw)
    ends, dg = run_cdc(hg, data, offset=offset, **q)
    cands = oracle.window_candidates(data, q["window"], q["mask_bits"], q["magic"], nthreads=8)
    want = oracle.select(cands, n, q["min_chunk"], q["max_chunk"])
    assert np.array_equal(ends, want)
    check_chunking(want.tolist(), cands.tolist(), n, q["min_chunk"], q["max_chunk"])
    assert np.array_equal(dg, oracle.hash_chunks(oracle.MD5, data, want))


def test_cdc_dense_candidates_use_bitmap_path(hg):
    """More candidates than the list holds: selection scans the bitmap instead."""
    data = G.uniform_bytes(1 << 20, seed=8)
    ends, dg = run_cdc(hg, data, mask_bits=2, magic=1, min_chunk=64, max_chunk=4096)
    cands = oracle.window_candidates(data, 20, 2, 1, nthreads=8)
    assert cands.size > (1 << 20) // 128 + 4096
    assert np.array_equal(ends, oracle.select(cands, data.size, 64, 4096))
    assert np.array_equal(dg, oracle.hash_chunks(oracle.MD5, data, ends))


def test_cdc_constant_input(hg):
    for v in range(256):
        if oracle.window_candidates(bytes([v]) * 20, 20, 13, 0x0F0F).size == 0:
            break
    data = np.full(1_000_000, v, np.uint8)
    ends, _ = run_cdc(hg, data)
    assert ends.tolist() == list(range(65536, 1_000_000, 65536)) + [1_000_000]


@pytest.mark.parametrize("algo", [oracle.MD5, oracle.SHA1])
def test_hash_chunks_arbitrary(hg, algo):
    import paper_1202_3669_b300 as hgb
    data = G.uniform_bytes(300_000, seed=4)
    g = G.rng(5)
    ends = np.unique(np.concatenate([g.integers(1, 300_000, 300), [300_000, 1, 2, 3, 64, 65, 128]]))
    d = to_device(data, 3)
    e = torch.from_numpy(ends.astype(np.int64)).cuda()
    dg = hg.hash_chunks(d, e, algo)
    hg.sync()
    assert np.array_equal(dg.cpu().numpy(), oracle.hash_chunks(algo, data, ends.astype(np.uint64)))


# Chunk digests read their message through shared-memory rings filled by
# asynchronous copies of 16-byte granules: every start residue mod 16 (the
# shift of the unaligned loop and the extra granule of the first group) with
# lengths at and around the 64-byte block edges, empty chunks included.
STAGED_LENGTHS = [0, 1, 15, 16, 55, 56, 63, 64, 65, 127, 128, 129, 191, 192, 255, 256, 257, 319,
                  320, 321, 1000, 4095, 4096, 4097, 70_000]


@pytest.mark.parametrize("algo", [oracle.MD5, oracle.SHA1])
@pytest.mark.parametrize("offset", [0, 7])
def test_hash_chunks_staged_edges(hg, algo, offset):
    ends, cur = [], 0
    for L in STAGED_LENGTHS:
        for r in range(16):
            pad = (r - (offset + cur)) % 16         # a spacer chunk to reach residue r
            cur += pad
            ends.append(cur)
            cur += L
            ends.append(cur)
    ends = np.array(ends, dtype=np.uint64)
    data = G.uniform_bytes(int(ends[-1]), seed=len(ends))
    d = to_device(data, offset)
    e = torch.from_numpy(ends.astype(np.int64)).cuda()
    dg = hg.hash_chunks(d, e, algo)
    hg.sync()
    assert np.array_equal(dg.cpu().numpy(), oracle.hash_chunks(algo, data, ends))


def test_boundaries_capacity_reports_count(hg):
    data = G.uniform_bytes(1 << 20, seed=12)
    want = oracle.cdc(data, nthreads=8)
    ends, cnt = hg.cdc_boundaries(to_device(data), cap=5)
    assert int(cnt.item()) == want.size > 5
    assert np.array_equal(ends[:5].cpu().numpy().astype(np.uint64), want[:5])
    hg.sync()


@pytest.fixture(scope="module")
def versions():
    base = G.uniform_bytes(64 << 20, seed=2)
    v2, _ = G.edited_version(base, seed=3)
    return base, v2


def test_config_cdc_two_versions(hg, versions):
    """64 MiB base + 1%-edited second version: boundaries, MD5 digests, shared fraction."""
    out = []
    for v in versions:
        ends, dg = run_cdc(hg, v)
        cands = oracle.window_candidates(v, 20, 13, 0x0F0F, nthreads=16)
        want = oracle.select(cands, v.size, 2048, 65536)
        assert np.array_equal(ends, want)
        check_chunking(want.tolist(), cands.tolist(), v.size, 2048, 65536)
        assert np.array_equal(dg, oracle.hash_chunks(oracle.MD5, v, want))
        out.append((ends, dg))
    frac = oracle.shared_fraction(out[0][0], out[0][1], out[1][0], out[1][1])
    assert 0.3 < frac < 0.99


@pytest.mark.parametrize("n", [0, 1, 5000, 3 << 20, (20 << 20) + 12345, (100 << 20) + 7])
@pytest.mark.parametrize("algo", [oracle.MD5, oracle.SHA1])
def test_cdc_hash_pipelined(hg, n, algo):
    """hg_cdc_hash (segmented, digests as chunks are decided) equals the oracle."""
    data = G.uniform_bytes(n, seed=n + 7)
    d = to_device(data, 0 if n % 2 else 5)
    ends, cnt, dg = hg.cdc_hash(d, algo)
    hg.sync()
    k = int(cnt.item())
    want = oracle.cdc(data, nthreads=8)
    assert np.array_equal(ends[:k].cpu().numpy().astype(np.uint64), want)
    assert np.array_equal(dg[:k].cpu().numpy(), oracle.hash_chunks(algo, data, want))


def test_cdc_hash_dense_and_params(hg):
    """Candidate-list overflow (bitmap walk with a limit) and other parameters, segmented."""
    import paper_1202_3669_b300 as hgb
    data = G.uniform_bytes((97 << 20) + 99, seed=77)
    for p in (hgb.params(mask_bits=3, magic=1, min_chunk=256, max_chunk=4096),
              hgb.params(window=17, mask_bits=9, magic=0x55, min_chunk=700, max_chunk=70000)):
        ends, cnt, dg = hg.cdc_hash(to_device(data), hgb.MD5, p)
        hg.sync()
        k = int(cnt.item())
        want = oracle.select(oracle.window_candidates(data, p.window, p.mask_bits, p.magic, nthreads=8),
                             data.size, p.min_chunk, p.max_chunk)
        assert np.array_equal(ends[:k].cpu().numpy().astype(np.uint64), want)
        assert np.array_equal(dg[:k].cpu().numpy(), oracle.hash_chunks(oracle.MD5, data, want))


def test_config_cdc_two_versions_pipelined(hg, versions):
    for v in versions:
        ends, cnt, dg = hg.cdc_hash(to_device(v), oracle.MD5)
        hg.sync()
        k = int(cnt.item())
        want = oracle.cdc(v, nthreads=16)
        assert np.array_equal(ends[:k].cpu().numpy().astype(np.uint64), want)
        assert np.array_equal(dg[:k].cpu().numpy(), oracle.hash_chunks(oracle.MD5, v, want))


@pytest.mark.parametrize("n", [5000, (20 << 20) + 3, (70 << 20) + 11])
def test_cdc_hash_from_host(hg, n):
    """hg_cdc_hash_h2d: the call copies pinned host bytes in pieces while it chunks."""
    data = G.uniform_bytes(n, seed=n + 1)
    host = torch.from_numpy(data).pin_memory()
    dev = torch.empty(n, dtype=torch.uint8, device="cuda")
    ends, cnt, dg = hg.cdc_hash_from_host(host, dev, oracle.SHA1)
    hg.sync()
    k = int(cnt.item())
    want = oracle.cdc(data, nthreads=8)
    assert np.array_equal(ends[:k].cpu().numpy().astype(np.uint64), want)
    assert np.array_equal(dg[:k].cpu().numpy(), oracle.hash_chunks(oracle.SHA1, data, want))
    assert torch.equal(dev.cpu(), host)


@pytest.mark.parametrize("hoff,doff", [(3, 5), (1, 0), (0, 7)])
def test_cdc_hash_from_host_unaligned(hg, hoff, doff):
    """hg_cdc_hash_h2d with the host bytes and the device buffer at odd offsets (the device
    side then takes the byte-load window path throughout)."""
    n = (9 << 20) + 333
    data = G.uniform_bytes(n, seed=n + hoff)
    hbuf = torch.empty(n + 16, dtype=torch.uint8).pin_memory()
    hbuf[hoff:hoff + n] = torch.from_numpy(data)
    host = hbuf[hoff:hoff + n]
    dbuf = torch.empty(n + 16, dtype=torch.uint8, device="cuda")
    dev = dbuf[doff:doff + n]
    ends, cnt, dg = hg.cdc_hash_from_host(host, dev, oracle.MD5)
    hg.sync()
    k = int(cnt.item())
    want = oracle.cdc(data, nthreads=8)
    assert np.array_equal(ends[:k].cpu().numpy().astype(np.uint64), want)
    assert np.array_equal(dg[:k].cpu().numpy(), oracle.hash_chunks(oracle.MD5, data, want))
    assert torch.equal(dev.cpu(), host)


@pytest.mark.parametrize("pieces", [
    [1, 19, 20, 21, 5000, 65536, 65537, 1 << 20],
    [4096] * 300,
    [3 << 20, 7, (5 << 20) + 1],
    [64 << 20],
])
@pytest.mark.parametrize("algo", [oracle.MD5, oracle.SHA1])
def test_stream_feeds_equal_one_shot(hg, pieces, algo):
    """Streaming with carried leftovers (Sec. 3.2.4) equals chunking the whole stream."""
    import paper_1202_3669_b300 as hgb
    total = sum(pieces)
    data = G.uniform_bytes(total, seed=len(pieces) + total % 1000)
    d = to_device(data)
    st = hgb.CdcStream(hg, algo, max_feed=max(pieces))
    ends, dgs, off = [], [], 0
    for k in pieces:
        e, g = st.feed(d[off:off + k])
        ends.append(e.cpu().numpy())
        dgs.append(g.cpu().numpy())
        off += k
    e, g = st.close()
    ends.append(e.cpu().numpy())
    dgs.append(g.cpu().numpy())
    hg.sync()
    got_e = np.concatenate(ends).astype(np.uint64)
    got_d = np.concatenate(dgs)
    want = oracle.cdc(data, nthreads=8)
    assert np.array_equal(got_e, want)
    assert np.array_equal(got_d, oracle.hash_chunks(algo, data, want))


def test_stream_other_params_and_tiny_min(hg):
    import paper_1202_3669_b300 as hgb
    p = hgb.params(window=17, mask_bits=6, magic=0x11, min_chunk=8, max_chunk=3000)
    data = G.uniform_bytes(400_000, seed=5)
    d = to_device(data)
    st = hgb.CdcStream(hg, hgb.MD5, p, max_feed=50_000)
    ends, off = [], 0
    for k in [1, 2, 3, 16, 17, 18, 50_000, 49_999, 30_000] + [25_000] * 10:
        if off >= data.size:
            break
        k = min(k, data.size - off)
        ends.append(st.feed(d[off:off + k])[0].cpu().numpy())
        off += k
    if off < data.size:
        ends.append(st.feed(d[off:])[0].cpu().numpy())
    ends.append(st.close()[0].cpu().numpy())
    got = np.concatenate(ends).astype(np.uint64)
    want = oracle.select(oracle.window_candidates(data, 17, 6, 0x11, nthreads=8), data.size, 8, 3000)
    assert np.array_equal(got, want)


@pytest.mark.parametrize("dist", ["uniform", "text"])
def test_config_cdc_1gib(hg, dist):
    """1 GiB (uniform seed 4 / text-like seed 5) at the bench's sizes, compared in full:
    the whole candidate list (hg_cdc_candidates), every chunk end and every chunk digest
    of one hg_cdc_hash call equal the oracle's, computed on all host cores."""
    import os
    n = 1 << 30
    data = G.uniform_bytes(n, seed=4) if dist == "uniform" else G.text_like_bytes(n, seed=5)
    d = to_device(data)
    cands, ccnt = hg.cdc_candidates(d, cap=n // 1024)
    ends, cnt, dg = hg.cdc_hash(d, oracle.MD5)
    hg.sync()
    nc = int(ccnt.item())
    got_c = cands[:nc].cpu().numpy().astype(np.uint64)
    k = int(cnt.item())
    got_e = ends[:k].cpu().numpy().astype(np.uint64)
    got_d = dg[:k].cpu().numpy()
    del d, cands, ends, dg
    want_c = oracle.window_candidates(data, 20, 13, 0x0F0F, nthreads=os.cpu_count() or 1)
    assert np.array_equal(got_c, want_c)
    want_e = oracle.select(want_c, n, 2048, 65536)
    assert np.array_equal(got_e, want_e)
    assert np.array_equal(got_d, oracle_digests_parallel(oracle.MD5, data, want_e))
    check_chunking(want_e[:5000].tolist(), want_c[want_c <= want_e[4999]].tolist(),
                   int(want_e[4999]), 2048, 65536)


@pytest.mark.parametrize("algo", [oracle.MD5, oracle.SHA1])
def test_cdc_hash_all_chunks_at_max(hg, algo):
    """Constant input: every chunk is cut at max, more of them than lone-lane warps
    (the longest-chunk list stays empty) and, on a short input, fewer (all listed)."""
    for v in range(256):
        if oracle.window_candidates(bytes([v]) * 20, 20, 13, 0x0F0F).size == 0:
            break
    for n in (100 << 20, (3 << 20) + 17):
        data = np.full(n, v, np.uint8)
        ends, cnt, dg = hg.cdc_hash(to_device(data), algo)
        hg.sync()
        k = int(cnt.item())
        want = np.array(list(range(65536, n, 65536)) + [n], np.uint64)
        assert np.array_equal(ends[:k].cpu().numpy().astype(np.uint64), want)
        assert np.array_equal(dg[:k].cpu().numpy(), oracle.hash_chunks(algo, data, want))
