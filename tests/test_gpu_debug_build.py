"""The bounds-checking debug build (libhashgpu_debug.so, compiled with HG_DEBUG): on
valid inputs it reports no failed check and gives the same results as the release
library, through the same C calls (chunking with digests, one and several segments,
fixed blocks with the hash-of-hashes, a batch)."""
import ctypes as C
import os

import numpy as np
import pytest
import torch

from gen import inputs as G

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dbg():
    from paper_1202_3669_b300 import _lib
    path = os.path.join(os.path.dirname(_lib.LIB_PATH), "libhashgpu_debug.so")
    L = _lib.load(path)
    h = C.c_void_p()
    assert L.hg_init(C.byref(h), 0, 0) == 0
    yield L, h.value
    L.hg_destroy(h.value)


def test_debug_cdc_hash_equals_release(dbg):
    import paper_1202_3669_b300 as hgb
    L, h = dbg
    ctx = hgb.Context(0)
    p = hgb.default_params()
    s = torch.cuda.current_stream().cuda_stream
    for n, seed in ((0, 1), (5000, 2), ((3 << 20) + 11, 3), ((100 << 20) + 77, 4)):
        data = torch.from_numpy(G.uniform_bytes(n, seed)).cuda() if n else torch.empty(16, dtype=torch.uint8, device="cuda")
        cap = n // p.min_chunk + 2
        e = torch.empty(cap, dtype=torch.int64, device="cuda")
        k = torch.zeros(1, dtype=torch.int64, device="cuda")
        d = torch.empty((cap, 20), dtype=torch.uint8, device="cuda")
        for algo in (hgb.MD5, hgb.SHA1):
            assert L.hg_cdc_hash(h, algo, data.data_ptr(), n, C.byref(p), e.data_ptr(), cap,
                                 k.data_ptr(), d.data_ptr(), s) == 0
            assert L.hg_sync(h, s) == 0                   # no failed bounds check
            ends, cnt, dg = ctx.cdc_hash(data[:n], algo)
            ctx.sync()
            c = int(cnt.item())
            dl = 16 if algo == hgb.MD5 else 20
            assert int(k.item()) == c
            assert torch.equal(e[:c], ends[:c])
            assert torch.equal(d.view(-1)[:c * dl], dg[:c].reshape(-1))
    ctx.close()


def test_debug_blocks_and_batch_equal_release(dbg):
    import paper_1202_3669_b300 as hgb
    L, h = dbg
    ctx = hgb.Context(0)
    s = torch.cuda.current_stream().cuda_stream
    data = torch.from_numpy(G.uniform_bytes((8 << 20) + 5, 7)).cuda()
    for algo, dl in ((hgb.MD5, 16), (hgb.SHA1, 20)):
        nblk = (data.numel() + 4095) // 4096
        out = torch.empty((nblk, dl), dtype=torch.uint8, device="cuda")
        rt = torch.empty(dl, dtype=torch.uint8, device="cuda")
        assert L.hg_hash_blocks(h, algo, data.data_ptr(), data.numel(), 4096, out.data_ptr(),
                                rt.data_ptr(), s) == 0
        assert L.hg_sync(h, s) == 0
        o2, r2 = ctx.hash_blocks(data, 4096, algo)
        ctx.sync()
        assert torch.equal(out, o2) and torch.equal(rt, r2)
    sizes = G.lognormal_sizes(120, seed=8, median=40_000, sigma=1.4, hi=4 << 20)
    body, off = G.files_from_sizes(sizes, 9)
    d = torch.from_numpy(body).cuda()
    offs = np.asarray(off, dtype=np.uint64)
    p = hgb.default_params()
    bh = C.c_void_p()
    assert L.hg_batch_create(h, offs.ctypes.data, len(sizes), C.byref(p), C.byref(bh)) == 0
    slots = int(L.hg_batch_slots(bh, None))
    ends = torch.empty(slots, dtype=torch.int64, device="cuda")
    cnts = torch.empty(len(sizes), dtype=torch.int64, device="cuda")
    dg = torch.empty((slots, 20), dtype=torch.uint8, device="cuda")
    assert L.hg_batch_cdc_hash(bh, hgb.SHA1, d.data_ptr(), ends.data_ptr(), cnts.data_ptr(),
                               dg.data_ptr(), s) == 0
    assert L.hg_batch_sync(bh, s) == 0
    b = hgb.Batch(ctx, off)
    e2, c2, g2 = b.cdc_hash(d, hgb.SHA1)
    b.sync()
    assert torch.equal(cnts, c2)
    so = b.slot_off
    for f in range(len(sizes)):
        a, k = int(so[f]), int(c2[f].item())
        assert torch.equal(ends[a:a + k], e2[a:a + k]) and torch.equal(dg[a:a + k], g2[a:a + k])
    L.hg_batch_destroy(bh)
    b.close()
    ctx.close()
