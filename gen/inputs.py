"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the bench.

This module only draws bytes, sizes and arrival times. It holds none of the
hashing or chunking arithmetic, so the CPU oracle and the CUDA path can both
consume its output without sharing any of the method's code.

Every generator uses numpy's PCG64 bit generator with an explicit integer seed,
so a (function, arguments, seed) triple names one byte string on every machine.

The workloads mirror the ones the paper evaluates with (Sec. 4): large single
buffers for direct hashing and sliding-window hashing (Sec. 4.1), successive
versions of the same file for similarity detection (Sec. 4.3, the checkpoint
workload of Fig. 11), and streams of many files of uneven size submitted as
jobs (Sec. 3.2.3). The paper's own datasets are not available, so seeded
stand-ins with the recipe below replace them.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

MiB = 1 << 20
GiB = 1 << 30


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def uniform_bytes(n: int, seed: int) -> np.ndarray:
    """n i.i.d. uniform bytes (uint8 array)."""
    if n == 0:
        return np.zeros(0, dtype=np.uint8)
    return rng(seed).integers(0, 256, size=n, dtype=np.uint8)


def text_like_bytes(n: int, seed: int, line: int = 80, zipf_s: float = 1.1) -> np.ndarray:
    """Text-like stream: lines of `line-1` symbols then '\\n'.

    Symbols are i.i.d. from a finite Zipf(s) law over the 95 printable ASCII
    characters (rank k has probability proportional to k^-s); rank k maps to a
    character through a seeded permutation. A symbol is drawn by inverting the
    law's CDF at a uniform 16-bit level (probabilities quantised to 2^-16, so
    a GiB takes seconds). The stream is cut to n bytes.
    """
    g = rng(seed)
    chars = np.arange(32, 127, dtype=np.uint8)          # 95 printable
    perm = g.permutation(chars)                          # rank -> char
    w = np.arange(1, 96, dtype=np.float64) ** (-zipf_s)
    cdf = np.cumsum(w / w.sum())
    cdf[-1] = 1.0
    levels = (np.arange(1 << 16, dtype=np.float64) + 0.5) / (1 << 16)
    table = perm[np.searchsorted(cdf, levels, side="right").clip(0, 94)]   # 16-bit level -> char
    nlines = (n + line - 1) // line
    out = np.empty(nlines * line, dtype=np.uint8)
    view = out.reshape(nlines, line)
    step = max(1, (64 * MiB) // line)
    for r0 in range(0, nlines, step):
        r1 = min(nlines, r0 + step)
        u = g.integers(0, 1 << 16, size=(r1 - r0, line - 1), dtype=np.uint16)
        view[r0:r1, : line - 1] = table[u]
    view[:, line - 1] = ord("\n")
    return out[:n].copy()


@dataclass
class Edit:
    op: str      # "insert" | "delete" | "overwrite"
    pos: int     # position in the version being edited
    length: int


def edited_version(base: np.ndarray, seed: int, frac: float = 0.01,
                   max_run: int = 512) -> tuple[np.ndarray, list[Edit]]:
    """Second version of `base` made by seeded edits.

    Edits are drawn until at least ceil(frac * len(base)) bytes have been
    touched. Each edit picks its type uniformly from insert/delete/overwrite,
    its run length uniformly in 1..max_run and its position uniformly over the
    current length; inserted and overwritten bytes are uniform random. The
    edits are applied one after another to a piece table, so positions always
    refer to the current version.
    """
    g = rng(seed)
    target = int(math.ceil(frac * len(base)))
    bufs = [base]
    # piece = (buffer id, start, length)
    pieces: list[tuple[int, int, int]] = [(0, 0, len(base))] if len(base) else []
    length = len(base)
    touched = 0
    log: list[Edit] = []

    def split_at(pos: int) -> int:
        """Split so that a piece starts at `pos`; return that piece index."""
        acc = 0
        for i, (b, s, l) in enumerate(pieces):
            if pos == acc:
                return i
            if pos < acc + l:
                k = pos - acc
                pieces[i:i + 1] = [(b, s, k), (b, s + k, l - k)]
                return i + 1
            acc += l
        return len(pieces)

    while touched < target:
        op = ("insert", "delete", "overwrite")[int(g.integers(0, 3))]
        run = int(g.integers(1, max_run + 1))
        if op == "insert":
            pos = int(g.integers(0, length + 1))
            data = g.integers(0, 256, size=run, dtype=np.uint8)
            bufs.append(data)
            i = split_at(pos)
            pieces.insert(i, (len(bufs) - 1, 0, run))
            length += run
            touched += run
        else:
            if length == 0:
                continue
            pos = int(g.integers(0, length))
            run = min(run, length - pos)
            i = split_at(pos)
            j = split_at(pos + run)
            del pieces[i:j]
            if op == "overwrite":
                data = g.integers(0, 256, size=run, dtype=np.uint8)
                bufs.append(data)
                pieces.insert(i, (len(bufs) - 1, 0, run))
            else:
                length -= run
            touched += run
        log.append(Edit(op, pos, run))
    out = np.concatenate([bufs[b][s:s + l] for b, s, l in pieces]) if pieces else np.zeros(0, np.uint8)
    assert len(out) == length
    return out, log


def lognormal_sizes(count: int, seed: int, median: int = 64 * 1024, sigma: float = 2.4,
                    lo: int = 512, hi: int = 256 * MiB) -> np.ndarray:
    """File sizes: log-normal with the given median and sigma, clipped to [lo, hi]."""
    g = rng(seed)
    s = np.exp(np.log(median) + sigma * g.standard_normal(count))
    return np.clip(np.rint(s), lo, hi).astype(np.int64)


def batch_workload_seed(count: int = 4096, target: int = 4 * GiB, tol: float = 0.10,
                        first_seed: int = 6, **kw) -> tuple[int, np.ndarray]:
    """First seed >= first_seed whose realised total size is within target*(1 +- tol)."""
    seed = first_seed
    while True:
        sizes = lognormal_sizes(count, seed, **kw)
        if abs(int(sizes.sum()) - target) <= tol * target:
            return seed, sizes
        seed += 1


def files_from_sizes(sizes: np.ndarray, seed: int) -> tuple[np.ndarray, np.ndarray]:
    """Concatenated uniform-random file bodies and their offsets (len(sizes)+1, int64)."""
    off = np.zeros(len(sizes) + 1, dtype=np.int64)
    np.cumsum(sizes, out=off[1:])
    return uniform_bytes(int(off[-1]), seed), off


def poisson_arrivals(rate_per_s: float, count: int, seed: int) -> np.ndarray:
    """Arrival times (seconds from 0) of a Poisson process."""
    g = rng(seed)
    return np.cumsum(g.exponential(1.0 / rate_per_s, size=count))


def plant_bytes(buf: np.ndarray, pos: int, pattern: bytes) -> np.ndarray:
    """Copy of buf with `pattern` written at `pos` (used to force known windows)."""
    out = buf.copy()
    out[pos:pos + len(pattern)] = np.frombuffer(pattern, dtype=np.uint8)
    return out
