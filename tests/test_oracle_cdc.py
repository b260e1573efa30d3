"""Pins of the oracle's content-based chunking (Sec. 2.1, Sec. 3.2.2, Sec. 4.3).

Window hashes are checked by brute force with hashlib.md5 of every window;
selection against hand-worked fixtures and a declarative rule checker; the
whole chunker against invariants of content-defined chunking.
"""
import hashlib
import json
import os

import numpy as np
import pytest

import oracle
from gen import inputs as G
from tests.pins import brute_window_cuts, check_chunking

HERE = os.path.dirname(os.path.abspath(__file__))


def test_window_hash_is_first_md5_word():
    w = G.uniform_bytes(20, seed=1).tobytes()
    assert oracle.window_hash(w) == int.from_bytes(hashlib.md5(w).digest()[:4], "little")


@pytest.mark.parametrize("window,mask_bits,magic", [(20, 4, 0x5), (20, 6, 0x2A), (16, 3, 0x1),
                                                    (1, 2, 0x3), (55, 4, 0xF), (7, 32, 0)])
@pytest.mark.parametrize("n", [0, 1, 19, 20, 21, 1000, 4096])
def test_window_candidates_brute_force(window, mask_bits, magic, n):
    data = G.uniform_bytes(n, seed=n * 31 + window).tobytes()
    got = oracle.window_candidates(data, window, mask_bits, magic)
    assert got.tolist() == brute_window_cuts(data, window, mask_bits, magic)


def test_window_candidates_threads_agree():
    data = G.uniform_bytes(200_000, seed=5).tobytes()
    a = oracle.window_candidates(data, 20, 8, 0x0F, nthreads=1)
    b = oracle.window_candidates(data, 20, 8, 0x0F, nthreads=7)
    assert a.tolist() == b.tolist() and a.size > 100


def planted_window(seed=0, window=20, mask_bits=13, magic=0x0F0F):
    """A window whose MD5 low bits equal magic, found by search with hashlib."""
    g = G.rng(seed)
    mask = (1 << mask_bits) - 1
    while True:
        w = g.integers(0, 256, size=window, dtype=np.uint8).tobytes()
        if int.from_bytes(hashlib.md5(w).digest()[:4], "little") & mask == magic:
            return w


def test_planted_candidates_found():
    w = planted_window(seed=11)
    base = G.uniform_bytes(10_000, seed=12)
    for pos in (0, 1, 4321, 10_000 - 20):
        buf = G.plant_bytes(base, pos, w).tobytes()
        got = oracle.window_candidates(buf, 20, 13, 0x0F0F).tolist()
        assert pos + 20 in got
        assert got == brute_window_cuts(buf, 20, 13, 0x0F0F)


def test_select_golden():
    with open(os.path.join(HERE, "golden", "select_cases.json")) as f:
        cases = json.load(f)["cases"]
    for c in cases:
        got = oracle.select(np.array(c["cands"], np.uint64), c["n"], c["min"], c["max"]).tolist()
        assert got == c["ends"], c["steps"]
        check_chunking(got, c["cands"], c["n"], c["min"], c["max"])


@pytest.mark.parametrize("seed", range(40))
def test_select_rule_random(seed):
    g = G.rng(1000 + seed)
    n = int(g.integers(0, 3000))
    mn = int(g.integers(1, 60))
    mx = int(g.integers(mn, 200))
    k = int(g.integers(0, max(1, n // 5) + 1))
    cands = np.unique(g.integers(1, n + 1, size=k)) if n else np.zeros(0, np.int64)
    ends = oracle.select(cands.astype(np.uint64), n, mn, mx)
    check_chunking(ends.tolist(), cands.tolist(), n, mn, mx)


def test_cdc_invariants_uniform():
    data = G.uniform_bytes(4 << 20, seed=2)
    cands = oracle.window_candidates(data, 20, 13, 0x0F0F, nthreads=8)
    ends = oracle.select(cands, data.size, 2048, 65536)
    check_chunking(ends.tolist(), cands.tolist(), data.size, 2048, 65536)
    sizes = np.diff(np.concatenate([[0], ends.astype(np.int64)]))
    assert sizes.sum() == data.size
    # candidate density 2^-13 per offset: ~512 in 4 MiB
    assert 350 < cands.size < 700
    assert 2048 + 4000 < sizes.mean() < 2048 + 14000


def test_constant_input_only_forced_cuts():
    # a constant stream has one window value; pick bytes that are not candidates
    for v in range(256):
        if oracle.window_candidates(bytes([v]) * 20, 20, 13, 0x0F0F).size == 0:
            break
    data = bytes([v]) * 300_000
    ends = oracle.cdc(data).tolist()
    assert ends == list(range(65536, 300_000, 65536)) + [300_000]


def test_shift_invariance():
    """Prepending bytes moves the later boundaries by the same amount."""
    data = G.uniform_bytes(2 << 20, seed=21)
    pre = G.uniform_bytes(777, seed=22)
    e1 = oracle.cdc(data, nthreads=8).astype(np.int64)
    e2 = oracle.cdc(np.concatenate([pre, data]), nthreads=8).astype(np.int64) - 777
    tail1 = set(e1[e1 > 200_000].tolist())
    tail2 = set(e2[e2 > 200_000].tolist())
    assert tail1 == tail2


def test_edit_locality():
    """A single overwrite changes only boundaries near it."""
    data = G.uniform_bytes(2 << 20, seed=31)
    ed = data.copy()
    ed[1_000_000:1_000_100] ^= 0x5A
    e1 = set(oracle.cdc(data, nthreads=8).tolist())
    e2 = set(oracle.cdc(ed, nthreads=8).tolist())
    diff = sorted(e1 ^ e2)
    assert all(900_000 < d < 1_300_000 for d in diff), diff
    # an edit that plants a candidate window does move a boundary
    w = bytes(G.uniform_bytes(20, seed=0))
    for seed in range(100000):
        w = G.uniform_bytes(20, seed=seed).tobytes()
        if oracle.window_candidates(w, 20, 13, 0x0F0F).size:
            break
    ed2 = G.plant_bytes(data, 1_000_000, w)
    e3 = set(oracle.cdc(ed2, nthreads=8).tolist())
    diff = sorted(e1 ^ e3)
    assert diff and all(900_000 < d < 1_300_000 for d in diff), diff
