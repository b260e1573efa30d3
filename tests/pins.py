"""Independent checks the oracle is pinned to (no oracle code in here).

hashlib (OpenSSL) stands for the RFC 1321 / FIPS 180-4 digests, and the
selection checker states the chunking rule declaratively: it verifies the
properties that, taken together, admit exactly one chunking of a stream.
"""
from __future__ import annotations

import hashlib

import numpy as np


def ref_digest(algo: int, data: bytes) -> bytes:
    return (hashlib.md5 if algo == 0 else hashlib.sha1)(data).digest()


def brute_window_cuts(data: bytes, window: int, mask_bits: int, magic: int) -> list[int]:
    """Cut position p+1 of every window ending at p whose MD5 low bits match."""
    mask = (1 << mask_bits) - 1 if mask_bits < 32 else 0xFFFFFFFF
    out = []
    for p in range(window - 1, len(data)):
        h = int.from_bytes(hashlib.md5(data[p - window + 1:p + 1]).digest()[:4], "little")
        if h & mask == magic:
            out.append(p + 1)
    return out


def brute_window_cuts_with(data: bytes, window: int, mask_bits: int, magic: int, fp) -> list[int]:
    """Cut position p+1 of every window ending at p whose hash fp(window bytes) low bits match."""
    mask = (1 << mask_bits) - 1 if mask_bits < 32 else 0xFFFFFFFF
    return [p + 1 for p in range(window - 1, len(data))
            if fp(data[p - window + 1:p + 1]) & mask == magic]


def check_chunking(ends, cands, n: int, mn: int, mx: int) -> None:
    """Assert that `ends` is the one chunking the min/max greedy rule admits.

    Each chunk [s, e) must be one of:
      (a) e is a candidate, min <= e - s <= max, and no candidate lies in
          [s + min, e)  -- the first qualifying candidate was taken;
      (b) e = s + max < n and no candidate lies in [s + min, s + max];
      (c) e = n, n - s <= max and no candidate lies in [s + min, n).
    These leave one choice of e for every s, so they fix the whole list.
    """
    ends = [int(x) for x in ends]
    cs = np.asarray(sorted(int(c) for c in cands), dtype=np.int64)
    cset = set(int(c) for c in cs)

    def any_in(lo, hi):            # candidate in [lo, hi)
        i = np.searchsorted(cs, lo, side="left")
        return i < cs.size and cs[i] < hi

    if n == 0:
        assert ends == [], ends
        return
    assert ends and ends[-1] == n, (ends[-3:], n)
    s = 0
    for e in ends:
        assert e > s, (s, e)
        assert e - s <= mx, (s, e)
        if e in cset and e - s >= mn and not any_in(s + mn, e):
            pass                                           # (a)
        elif e == s + mx and e < n and not any_in(s + mn, s + mx + 1):
            pass                                           # (b)
        elif e == n and not any_in(s + mn, n):
            pass                                           # (c)
        else:
            raise AssertionError(f"chunk [{s}, {e}) breaks the rule (n={n}, min={mn}, max={mx})")
        s = e
