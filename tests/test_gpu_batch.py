"""GPU parity of batched chunking + chunk digests (many files, one pass) against the oracle.

Each file of a batch must be chunked and digested exactly as it is alone
(Sec. 2.1 / Fig. 3 per file); the batch form (Sec. 3.2.3 batching) only
changes how the work is scheduled.
"""
import numpy as np
import pytest
import torch

import oracle
from gen import inputs as G
from tests.gpu_util import oracle_files, to_device

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hg():
    import paper_1202_3669_b300 as hgb
    ctx = hgb.Context(0)
    yield ctx
    ctx.close()


def check_batch(hg, sizes, seed, algo, p=None, graph=False, offset=0):
    import paper_1202_3669_b300 as hgb
    p = p or hgb.default_params()
    sizes = np.asarray(sizes, dtype=np.int64)
    data, off = G.files_from_sizes(sizes, seed)
    b = hgb.Batch(hg, off, p)
    d = to_device(data, offset)
    out = b.cdc_hash(d, algo, graph=graph)
    b.sync()
    ends_h, cnt_h, dg_h = (t.cpu().numpy() for t in out)
    so = np.asarray(b.slot_off, dtype=np.int64)
    got = [(ends_h[so[f]:so[f] + cnt_h[f]].astype(np.uint64), dg_h[so[f]:so[f] + cnt_h[f]])
           for f in range(len(sizes))]
    b.close()
    want = oracle_files(data, off, p, algo)
    for f in range(len(sizes)):
        (ends, dg), (we, wd) = got[f], want[f]
        assert np.array_equal(ends, we), (f, sizes[f], ends[:5], we[:5])
        assert np.array_equal(dg, wd), f
    return out


@pytest.mark.parametrize("algo", [oracle.MD5, oracle.SHA1])
def test_batch_mixed_small(hg, algo):
    sizes = [0, 1, 19, 20, 21, 100, 2047, 2048, 5000, 8192, 8193, 70_000, 0, 3, 300_000,
             (1 << 20) + 77, 2_500_000, 50, 65_536, 65_537]
    check_batch(hg, sizes, seed=101, algo=algo)


def test_batch_lognormal(hg):
    sizes = G.lognormal_sizes(300, seed=11, median=32 * 1024, sigma=1.5, hi=4 << 20)
    check_batch(hg, sizes, seed=12, algo=oracle.SHA1)


def test_batch_graph_and_unaligned(hg):
    sizes = G.lognormal_sizes(64, seed=21, median=20_000, sigma=1.2, hi=2 << 20)
    check_batch(hg, sizes, seed=22, algo=oracle.MD5, graph=True, offset=3)


def test_batch_graph_replay_equals_direct(hg):
    import paper_1202_3669_b300 as hgb
    sizes = G.lognormal_sizes(128, seed=31, median=40_000, sigma=1.3, hi=3 << 20)
    data, off = G.files_from_sizes(sizes, 32)
    b = hgb.Batch(hg, off)
    d = to_device(data)
    o1 = b.cdc_hash(d, hgb.SHA1)
    o2 = b.outputs(hgb.SHA1)
    for _ in range(3):                                   # capture once, replay
        b.cdc_hash(d, hgb.SHA1, out=o2, graph=True)
    b.sync()
    assert torch.equal(o1[1], o2[1])
    for f in range(len(sizes)):
        a, k = int(b.slot_off[f]), int(o1[1][f])
        assert torch.equal(o1[0][a:a + k], o2[0][a:a + k])
        assert torch.equal(o1[2][a:a + k], o2[2][a:a + k])
    b.close()


def test_batch_dense_candidates(hg):
    """More candidates than the list holds: per-file selection scans the bitmap."""
    import paper_1202_3669_b300 as hgb
    p = hgb.params(mask_bits=2, magic=1, min_chunk=64, max_chunk=4096)
    sizes = [70_000, 1_200_000, 5, 300, 90_000]
    check_batch(hg, sizes, seed=41, algo=oracle.MD5, p=p)


def test_batch_other_params(hg):
    import paper_1202_3669_b300 as hgb
    p = hgb.params(window=17, mask_bits=9, magic=0x55, min_chunk=700, max_chunk=5000)
    sizes = G.lognormal_sizes(40, seed=51, median=30_000, sigma=1.0, hi=2 << 20)
    check_batch(hg, sizes, seed=52, algo=oracle.SHA1, p=p)


def test_batch_autotune_keeps_results(hg):
    import paper_1202_3669_b300 as hgb
    sizes = G.lognormal_sizes(200, seed=61, median=64 * 1024, sigma=1.5, hi=8 << 20)
    data, off = G.files_from_sizes(sizes, 62)
    b = hgb.Batch(hg, off)
    d = to_device(data)
    o1 = b.cdc_hash(d, hgb.SHA1)
    best = b.autotune(d, hgb.SHA1)
    assert best.hash_threads in (32, 64, 128) and best.window_ctas_per_sm >= 0
    o2 = b.cdc_hash(d, hgb.SHA1)
    b.sync()
    assert torch.equal(o1[1], o2[1])
    b.close()


def test_config_batch_4096_files(hg):
    """4096 log-normal files (median 64 KiB, sigma 2.4, 512 B..256 MiB, about 3.9 GB) in
    one graph-replayed batch: every file's chunk ends and SHA-1 digests equal the
    oracle's for that file alone."""
    seed, sizes = G.batch_workload_seed()
    out = check_batch(hg, sizes, seed=seed + 1000, algo=oracle.SHA1, graph=True)
    counts = out[1].cpu().numpy()
    assert (counts >= np.ceil(sizes / 65536)).all()
    assert (counts <= sizes // 2048 + 1).all()


def test_autotune_cache_reuses_tuning(hg, tmp_path):
    """The autotuner cache: the first call tunes and appends a line keyed by GPU,
    parameters and batch shape; the second finds it and tunes nothing; another batch
    shape misses."""
    import json

    import paper_1202_3669_b300 as hgb
    sizes = G.lognormal_sizes(150, seed=71, median=48 * 1024, sigma=1.3, hi=4 << 20)
    data, off = G.files_from_sizes(sizes, 72)
    d = to_device(data)
    cache = str(tmp_path / "autotune.jsonl")
    b = hgb.Batch(hg, off)
    t1 = b.autotune(d, hgb.SHA1, cache=cache)
    assert not b.tuned_from_cache
    t2 = b.autotune(d, hgb.SHA1, cache=cache)
    assert b.tuned_from_cache
    assert (t1.window_ctas_per_sm, t1.hash_threads, t1.hash_ctas_per_sm) == \
        (t2.window_ctas_per_sm, t2.hash_threads, t2.hash_ctas_per_sm)
    lines = open(cache).read().splitlines()
    assert len(lines) == 1
    rec = json.loads(lines[0])
    assert rec["key"]["nfile"] == 150 and rec["key"]["algo"] == hgb.SHA1
    assert rec["tuning"]["hash_threads"] == t1.hash_threads
    out = b.cdc_hash(d, hgb.SHA1)                # results with the cached tuning
    b.sync()
    b.close()
    b2 = hgb.Batch(hg, off[:101])                # another shape: a miss, a second line
    b2.autotune(d, hgb.MD5, cache=cache)
    assert not b2.tuned_from_cache and len(open(cache).read().splitlines()) == 2
    b2.close()
    want = oracle_files(data, off, hgb.default_params(), oracle.SHA1)
    so = np.asarray(hgb.Batch(hg, off).slot_off, dtype=np.int64)
    for f in (0, 50, 149):
        k = int(out[1][f].item())
        assert np.array_equal(out[0][so[f]:so[f] + k].cpu().numpy().astype(np.uint64), want[f][0])


@pytest.mark.parametrize("window_ctas", [0, 3, 8])
def test_batch_window_kernel_forms(hg, window_ctas):
    """Both window kernels of a batch (one-warp span CTAs: window_ctas_per_sm = 0;
    persistent CTAs: >= 1) give the oracle's chunks, aligned and unaligned files."""
    import paper_1202_3669_b300 as hgb
    sizes = G.lognormal_sizes(90, seed=81, median=30_000, sigma=1.6, hi=3 << 20)
    data, off = G.files_from_sizes(sizes, 82)
    for offset in (0, 5):
        b = hgb.Batch(hg, off)
        tn = hgb.hg_batch_tuning()
        assert hgb.hg_batch_get_tuning(b.h, tn) == 0
        tn.window_ctas_per_sm = window_ctas
        assert hgb.hg_batch_set_tuning(b.h, tn) == 0
        out = b.cdc_hash(to_device(data, offset), hgb.SHA1)
        b.sync()
        ends_h, cnt_h, dg_h = (x.cpu().numpy() for x in out)
        so = np.asarray(b.slot_off, dtype=np.int64)
        want = oracle_files(data, off, hgb.default_params(), oracle.SHA1)
        for f in range(len(sizes)):
            k = int(cnt_h[f])
            assert np.array_equal(ends_h[so[f]:so[f] + k].astype(np.uint64), want[f][0]), (f, offset)
            assert np.array_equal(dg_h[so[f]:so[f] + k], want[f][1]), (f, offset)
        b.close()
