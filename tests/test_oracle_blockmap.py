"""Pins of the similarity-detection oracle (digest membership and shared bytes)."""
import numpy as np

import oracle


def D(*tags, n=16):
    """Digests made of repeated tag bytes, one row per tag."""
    return np.array([[t] * n for t in tags], dtype=np.uint8)


def test_hand_worked_case():
    # v1 chunks carry digests A, B; v2 chunks [0,5) B, [5,15) C, [15,30) A
    known = D(0xA, 0xB)
    hits = oracle.blockmap_hits(known, D(0xB, 0xC, 0xA))
    assert hits.tolist() == [True, False, True]
    assert oracle.shared_bytes(known, [5, 15, 30], D(0xB, 0xC, 0xA)) == (2, 5 + 15)
    assert oracle.shared_fraction([10, 20], known, [5, 15, 30], D(0xB, 0xC, 0xA)) == 20 / 30


def test_full_digest_compared_not_a_prefix():
    a = np.zeros((1, 20), np.uint8)
    b = a.copy()
    b[0, 19] = 1                          # same first 19 bytes
    assert oracle.blockmap_hits(a, b).tolist() == [False]
    assert oracle.blockmap_hits(a, a).tolist() == [True]


def test_duplicates_and_empty_sets():
    known = D(1, 1, 2)
    assert oracle.blockmap_hits(known, D(1, 1, 3, 2)).tolist() == [True, True, False, True]
    assert oracle.blockmap_hits(np.zeros((0, 16), np.uint8), D(1)).tolist() == [False]
    assert oracle.blockmap_hits(known, np.zeros((0, 16), np.uint8)).size == 0
    assert oracle.shared_bytes(known, [], np.zeros((0, 16), np.uint8)) == (0, 0)


def test_identical_and_disjoint_versions():
    g = np.random.default_rng(4)
    dg = g.integers(0, 256, (500, 16), dtype=np.uint8)
    ends = np.cumsum(g.integers(1, 5000, 500))
    assert oracle.shared_bytes(dg, ends, dg) == (500, int(ends[-1]))
    other = g.integers(0, 256, (300, 16), dtype=np.uint8)
    assert oracle.shared_bytes(dg, ends[:300], other) == (0, 0)
    # the known set's order does not matter
    assert oracle.blockmap_hits(dg[::-1], dg[:50]).all()
