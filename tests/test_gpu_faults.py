"""Failure paths that a test can drive without faulting the GPU (the failure is made
on the host): a bounded device-side wait that runs out reports HG_ETIMEDOUT through
the context's error word and leaves the context usable; a context budget smaller
than a call's scratch gives HG_ENOMEM before anything is enqueued."""
import ctypes as C

import numpy as np
import pytest
import torch

from gen import inputs as G

pytestmark = pytest.mark.gpu


def test_blockmap_publish_wait_times_out_and_context_recovers():
    import paper_1202_3669_b300 as hgb
    from paper_1202_3669_b300 import _lib
    ctx = hgb.Context(0)
    m = hgb.BlockMap(ctx, hgb.MD5, capacity=4096)
    dg = np.frombuffer(bytes(range(1, 17)) + bytes(range(101, 117)), dtype=np.uint8).reshape(2, 16).copy()
    d = torch.from_numpy(dg).cuda()
    s = torch.cuda.current_stream().cuda_stream
    # a claim of digest 0's slot that was never published, made from the host
    assert _lib.lib.hg_blockmap_inject_claim(m.h, dg[0].ctypes.data, s) == 0
    assert _lib.lib.hg_blockmap_inject_claim(m.h, dg[0].ctypes.data, s) == _lib.HG_EINVAL
    assert _lib.lib.hg_blockmap_set_wait_limit(m.h, 2000) == 0
    m.insert(d)                                  # digest 0 waits on the claim and gives up
    rc = _lib.lib.hg_sync(ctx.h, s)
    assert rc == _lib.HG_ETIMEDOUT
    assert _lib.lib.hg_sync(ctx.h, s) == 0       # the error word was cleared
    # the context and the map keep working
    m.clear()
    assert _lib.lib.hg_blockmap_set_wait_limit(m.h, 0) == 0
    m.insert(d)
    m.insert(d)
    hits, res = m.lookup(d)
    ctx.sync()
    assert int(m.count().item()) == 2 and int(res[0].item()) == 2 and hits.cpu().tolist() == [1, 1]
    m.close()
    ctx.close()


def test_context_budget_gives_enomem():
    import paper_1202_3669_b300 as hgb
    from paper_1202_3669_b300 import _lib
    ctx = hgb.Context(0, budget=1 << 20)         # 1 MiB of scratch
    data = torch.from_numpy(G.uniform_bytes(8 << 20, seed=9)).cuda()
    with pytest.raises(hgb.HashGPUError) as e:
        ctx.cdc_hash(data, hgb.MD5)
    assert e.value.status == _lib.HG_ENOMEM
    with pytest.raises(hgb.HashGPUError) as e:
        ctx.reserve(64 << 20)
    assert e.value.status == _lib.HG_ENOMEM
    # a small input still fits and is chunked
    small = data[:100_000]
    ends, cnt, dg = ctx.cdc_hash(small, hgb.MD5)
    ctx.sync()
    assert int(ends[int(cnt.item()) - 1].item()) == 100_000
    assert _lib.lib.hg_scratch_bytes(ctx.h) <= 1 << 20
    ctx.close()
