"""Run-to-run determinism of the device path: the same call on the same bytes gives the
same bytes out, whatever the scheduling.

compute-sanitizer's race checker is not available here, so this is the stand-in for
race detection: the kernels use atomics (tile counts, work counters, block-map slots),
persistent grids and several streams, and a race in any of them that changed a
result would show as two runs that disagree. Each case runs repeatedly, twice with
another context's work on a second stream in flight at the same time, and is also
compared once with the oracle, so that "always the same" is also "right".
"""
import numpy as np
import pytest
import torch

import oracle
from gen import inputs as G
from tests.gpu_util import to_device

pytestmark = pytest.mark.gpu


def _chunk_once(ctx, d, algo, stream):
    ends, cnt, dg = ctx.cdc_hash(d, algo, stream=stream)
    return ends, cnt, dg


@pytest.mark.parametrize("algo", [oracle.MD5, oracle.SHA1])
def test_cdc_hash_repeats_bit_exactly(algo):
    import paper_1202_3669_b300 as hgb
    n = (70 << 20) + 4097                      # two segments and a ragged tail
    data = G.uniform_bytes(n, seed=901)
    other = G.uniform_bytes(64 << 20, seed=902)
    d, d2 = to_device(data, 3), to_device(other)
    a, b = hgb.Context(0), hgb.Context(0)
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    runs, keep = [], []
    for rep in range(4):
        if rep >= 2:                           # a second context's chunking in flight too
            keep.append(b.cdc_hash(d2, oracle.MD5, stream=s2))   # outputs live until the sync
        ends, cnt, dg = _chunk_once(a, d, algo, s1)
        torch.cuda.synchronize()
        k = int(cnt.item())
        runs.append((ends[:k].cpu().clone(), dg[:k].cpu().clone()))
    a.sync(), b.sync()
    for e, g in runs[1:]:
        assert torch.equal(e, runs[0][0]) and torch.equal(g, runs[0][1])
    want = oracle.cdc(data, nthreads=8)
    assert np.array_equal(runs[0][0].numpy().astype(np.uint64), want)
    a.close(), b.close()


def test_window_bitmap_and_candidates_repeat():
    import paper_1202_3669_b300 as hgb
    ctx = hgb.Context(0)
    data = G.uniform_bytes((9 << 20) + 333, seed=903)
    d = to_device(data, 1)
    p = hgb.default_params()
    bms, cands = [], []
    for _ in range(3):
        bm = ctx.window_bitmap(d, p)
        c, cnt = ctx.cdc_candidates(d, p)
        torch.cuda.synchronize()
        bms.append(bm.cpu().clone())
        cands.append(c[:int(cnt.item())].cpu().clone())
    ctx.sync()
    for x, y in zip(bms[1:], cands[1:]):
        assert torch.equal(x, bms[0]) and torch.equal(y, cands[0])
    ctx.close()


@pytest.mark.parametrize("algo", [oracle.MD5, oracle.SHA1])
def test_batch_repeats_bit_exactly(algo):
    import paper_1202_3669_b300 as hgb
    sizes = G.lognormal_sizes(200, seed=904)
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    data = G.uniform_bytes(int(off[-1]), seed=905)
    ctx = hgb.Context(0)
    bt = hgb.Batch(ctx, off)
    d = to_device(data)
    outs = []
    for rep in range(3):
        ends, counts, dg = bt.cdc_hash(d, algo, graph=(rep > 0))
        bt.sync()
        outs.append((ends.cpu().clone(), counts.cpu().clone(), dg.cpu().clone()))
    for e, c, g in outs[1:]:
        assert torch.equal(c, outs[0][1])
        for f in range(len(sizes)):
            k = int(c[f])
            a, b = bt.file_results(f, e, c, g), bt.file_results(f, *outs[0])
            assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1]) and k == len(a[0])
    bt.close()
    ctx.close()


def test_hash_blocks_repeat():
    import paper_1202_3669_b300 as hgb
    ctx = hgb.Context(0)
    data = G.uniform_bytes((48 << 20) + 100, seed=906)
    d = to_device(data)
    for algo in (oracle.MD5, oracle.SHA1):
        first = None
        for _ in range(3):
            dg, root = ctx.hash_blocks(d, 4096, algo)
            torch.cuda.synchronize()
            cur = (dg.cpu().clone(), root.cpu().clone())
            if first is None:
                first = cur
            assert torch.equal(cur[0], first[0]) and torch.equal(cur[1], first[1])
    ctx.sync()
    ctx.close()
