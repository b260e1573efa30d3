"""GPU parity of the device block map (similarity detection by digests) against the oracle.

Membership and byte counts are exact integer results.
"""
import numpy as np
import pytest
import torch

import oracle
from gen import inputs as G
from tests.gpu_util import to_device

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hg():
    import paper_1202_3669_b300 as hgb
    ctx = hgb.Context(0)
    yield ctx
    ctx.close()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("algo", [oracle.MD5, oracle.SHA1])
def test_two_versions_shared_bytes(hg, algo):
    """Chunk digests of a 32 MiB base and its 1%-edited version: the map of the base's
    digests finds exactly the oracle's shared chunks of the second version."""
    import paper_1202_3669_b300 as hgb
    base = G.uniform_bytes(32 << 20, seed=2)
    v2, _ = G.edited_version(base, seed=3)
    outs = []
    for v in (base, v2):
        ends, cnt, dg = hg.cdc_hash(to_device(v), algo)
        hg.sync()
        k = int(cnt.item())
        outs.append((ends[:k], cnt, dg[:k]))
    m = hgb.BlockMap(hg, algo, capacity=20_000)
    m.insert(outs[0][2], count=outs[0][1])
    hits, res = m.lookup(outs[1][2], ends=outs[1][0], count=outs[1][1])
    cnt = m.count()
    hg.sync()
    d1, d2 = outs[0][2].cpu().numpy(), outs[1][2].cpu().numpy()
    e2 = outs[1][0].cpu().numpy()
    assert np.array_equal(hits.cpu().numpy().astype(bool), oracle.blockmap_hits(d1, d2))
    assert tuple(res.cpu().tolist()) == oracle.shared_bytes(d1, e2, d2)
    assert int(cnt.item()) == len({bytes(r) for r in d1})
    frac = res[1].item() / v2.size
    assert frac == pytest.approx(oracle.shared_fraction(outs[0][0].cpu().numpy(), d1, e2, d2))
    m.close()


@pytest.mark.parametrize("dl", [16, 20])
def test_near_collisions_and_duplicates(hg, dl):
    """Digests that share the tag bytes, the home-slot bytes, or all but the last
    byte; all-zero leading bytes; many repeats: membership stays exact."""
    import paper_1202_3669_b300 as hgb
    algo = oracle.MD5 if dl == 16 else oracle.SHA1
    g = np.random.default_rng(9)
    base = g.integers(0, 256, (64, dl), dtype=np.uint8)
    rows = [base]
    same_tag = base.copy(); same_tag[:, 8:] = g.integers(0, 256, (64, dl - 8), dtype=np.uint8)
    same_home = base.copy(); same_home[:, :8] = g.integers(0, 256, (64, 8), dtype=np.uint8)
    last_byte = base.copy(); last_byte[:, dl - 1] ^= 0x5A
    zero_tag = base.copy(); zero_tag[:, :8] = 0
    one_tag = zero_tag.copy(); one_tag[:, 0] = 1
    known = np.concatenate([base, same_tag[:32], same_home[:32], zero_tag[:1]] + [base[:8]] * 20)
    queries = np.concatenate([base, same_tag, same_home, last_byte, zero_tag[:2], one_tag[:2]])
    m = hgb.BlockMap(hg, algo, capacity=1000)
    m.insert(dev(known))
    hits, res = m.lookup(dev(queries))
    cnt = m.count()
    hg.sync()
    want = oracle.blockmap_hits(known, queries)
    assert np.array_equal(hits.cpu().numpy().astype(bool), want)
    assert int(res[0].item()) == int(want.sum())
    assert int(cnt.item()) == len({bytes(r) for r in known})
    m.clear()
    hits, res = m.lookup(dev(queries))
    cnt = m.count()
    hg.sync()
    assert not hits.cpu().numpy().any() and int(cnt.item()) == 0
    m.close()


def test_large_random(hg):
    """2^22 random MD5-sized digests stored, 2^22 queries of which half are stored."""
    import paper_1202_3669_b300 as hgb
    g = np.random.default_rng(10)
    known = g.integers(0, 256, (1 << 22, 16), dtype=np.uint8)
    fresh = g.integers(0, 256, (1 << 21, 16), dtype=np.uint8)
    pick = g.integers(0, known.shape[0], 1 << 21)
    queries = np.concatenate([known[pick], fresh])
    sizes = g.integers(1, 70000, queries.shape[0])
    ends = np.cumsum(sizes).astype(np.int64)
    m = hgb.BlockMap(hg, hgb.MD5, capacity=1 << 22)
    m.insert(dev(known))
    hits, res = m.lookup(dev(queries), ends=dev(ends))
    hg.sync()
    h = hits.cpu().numpy().astype(bool)
    assert h[: 1 << 21].all() and not h[1 << 21:].any()
    assert int(res[0].item()) == 1 << 21
    assert int(res[1].item()) == int(sizes[: 1 << 21].sum())
    m.close()


def test_count_from_device_and_capacity_error(hg):
    import paper_1202_3669_b300 as hgb
    g = np.random.default_rng(11)
    known = g.integers(0, 256, (3000, 16), dtype=np.uint8)
    m = hgb.BlockMap(hg, hgb.MD5, capacity=2000)          # 4096 slots
    dcount = torch.tensor([1500], dtype=torch.int64, device="cuda")
    m.insert(dev(known), count=dcount)                    # only the first 1500
    hits, res = m.lookup(dev(known))
    cnt = m.count()
    hg.sync()
    assert int(cnt.item()) == 1500
    assert hits.cpu().numpy()[:1500].all() and not hits.cpu().numpy()[1500:].any()
    m.close()
    small = hgb.BlockMap(hg, hgb.MD5, capacity=10)        # 1024 slots
    small.insert(dev(g.integers(0, 256, (2000, 16), dtype=np.uint8)))
    with pytest.raises(hgb.HashGPUError):
        hg.sync()
    small.close()
    hg.sync()                                             # the error word was cleared


def test_bad_arguments(hg):
    import paper_1202_3669_b300 as hgb
    from paper_1202_3669_b300 import _lib
    with pytest.raises(hgb.HashGPUError):
        hgb.BlockMap(hg, 7, capacity=10)
    with pytest.raises(hgb.HashGPUError):
        hgb.BlockMap(hg, hgb.MD5, capacity=0)
    m = hgb.BlockMap(hg, hgb.MD5, capacity=10)
    buf = torch.zeros(64, dtype=torch.uint8, device="cuda")
    assert _lib.hg_blockmap_insert(m.h, buf.data_ptr() + 1, 2, None, None) != 0   # misaligned
    assert _lib.hg_blockmap_lookup(m.h, buf.data_ptr(), None, 2, None, None, None, None) != 0
    m.close()
    hg.sync()
