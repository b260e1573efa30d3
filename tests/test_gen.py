"""The seeded input recipes are deterministic and have the stated shape."""
import numpy as np

from gen import inputs as G


def test_uniform_deterministic():
    assert np.array_equal(G.uniform_bytes(1000, 5), G.uniform_bytes(1000, 5))
    assert not np.array_equal(G.uniform_bytes(1000, 5), G.uniform_bytes(1000, 6))


def test_text_like_lines():
    t = G.text_like_bytes(8000, seed=5)
    lines = t.reshape(-1, 80)
    assert (lines[:, 79] == ord("\n")).all()
    assert (lines[:, :79] >= 32).all() and (lines[:, :79] < 127).all()
    # Zipf skew: the most common symbol is far more common than the median one
    cnt = np.bincount(lines[:, :79].ravel(), minlength=256)
    c = np.sort(cnt[cnt > 0])[::-1]
    assert c[0] > 8 * c[len(c) // 2]


def test_edited_version_touches_one_percent():
    base = G.uniform_bytes(1 << 20, seed=2)
    v2, log = G.edited_version(base, seed=3)
    touched = sum(e.length for e in log)
    assert touched >= int(np.ceil(0.01 * base.size))
    assert touched - max(e.length for e in log) < int(np.ceil(0.01 * base.size))
    assert all(1 <= e.length <= 512 for e in log)
    assert {e.op for e in log} == {"insert", "delete", "overwrite"}
    ins = sum(e.length for e in log if e.op == "insert")
    dele = sum(e.length for e in log if e.op == "delete")
    assert v2.size == base.size + ins - dele
    v2b, _ = G.edited_version(base, seed=3)
    assert np.array_equal(v2, v2b)


def test_lognormal_batch():
    seed, sizes = G.batch_workload_seed()
    assert seed >= 6 and sizes.size == 4096
    assert abs(int(sizes.sum()) - 4 * G.GiB) <= 0.1 * 4 * G.GiB
    assert sizes.min() >= 512 and sizes.max() <= 256 * G.MiB
    assert 40_000 < np.median(sizes) < 100_000
