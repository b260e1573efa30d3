"""Pinned host buffer pool (hg_alloc_pinned / hg_free_pinned): reuse without a new
host allocation, the host budget, and chunking straight from a pool buffer
(Sec. 3.1 one-copy transfers and buffer reuse; Sec. 3.2.3 memory management)."""
import os

import numpy as np
import pytest
import torch

import oracle
from gen import inputs as G

pytestmark = pytest.mark.gpu


def test_freed_buffer_is_reused():
    import paper_1202_3669_b300 as hgb
    ctx = hgb.Context(0)
    a = ctx.alloc_pinned(3 << 20)
    pa = a.ptr
    assert a.tensor.numel() == 3 << 20 and a.ptr % 4096 == 0
    a.free()
    st = ctx.pinned_stats()
    assert st["host_allocs"] == 1 and st["in_use_bytes"] == 0 and st["held_bytes"] == 3 << 20
    b = ctx.alloc_pinned((3 << 20) - 1000)           # same class: the same buffer comes back
    assert b.ptr == pa
    st = ctx.pinned_stats()
    assert st["host_allocs"] == 1 and st["reuses"] == 1 and st["in_use_bytes"] == 3 << 20
    c = ctx.alloc_pinned(100)                        # another class: a new allocation
    assert c.ptr != pa and ctx.pinned_stats()["host_allocs"] == 2
    b.free()
    c.free()
    ctx.trim_pinned()
    st = ctx.pinned_stats()
    assert st["held_bytes"] == 0 and st["buffers"] == 0
    ctx.close()


def test_host_budget():
    import paper_1202_3669_b300 as hgb
    ctx = hgb.Context(0)
    ctx.set_pinned_budget(8 << 20)
    a = ctx.alloc_pinned(5 << 20)
    with pytest.raises(hgb.HashGPUError):
        ctx.alloc_pinned(5 << 20)                    # 10 MiB would exceed 8 MiB
    b = ctx.alloc_pinned(2 << 20)                    # 7 MiB fits
    a.free()
    d = ctx.alloc_pinned(2 << 20)                    # 9 MiB would not fit: the free 5 MiB goes
    st = ctx.pinned_stats()
    assert st["held_bytes"] == 4 << 20 and st["in_use_bytes"] == 4 << 20 and st["buffers"] == 2
    from paper_1202_3669_b300 import _lib
    pb = b.ptr
    b.free()
    d.free()
    assert _lib.lib.hg_free_pinned(ctx.h, pb) == _lib.HG_EINVAL      # already given back
    assert _lib.lib.hg_free_pinned(ctx.h, pb + 64) == _lib.HG_EINVAL  # not a pool buffer
    ctx.close()


def test_cdc_hash_from_pool_buffer_equals_oracle():
    import paper_1202_3669_b300 as hgb
    ctx = hgb.Context(0)
    n = (9 << 20) + 123
    data = G.uniform_bytes(n, seed=303)
    buf = ctx.alloc_pinned(n)
    buf.numpy()[:] = data
    d_in = torch.empty(n, dtype=torch.uint8, device="cuda")
    ends, cnt, dg = ctx.cdc_hash_from_host(buf.tensor, d_in, hgb.MD5)
    ctx.sync()
    k = int(cnt.item())
    want = oracle.cdc(data, nthreads=os.cpu_count() or 1)
    assert np.array_equal(ends[:k].cpu().numpy().astype(np.uint64), want)
    assert np.array_equal(dg[:k].cpu().numpy(), oracle.hash_chunks(oracle.MD5, data, want))
    buf.free()
    assert ctx.pinned_stats()["host_allocs"] == 1
    ctx.close()
