"""Helpers for the GPU parity tests (placing seeded bytes on the device)."""
import numpy as np
import torch


def to_device(data: np.ndarray, offset: int = 0) -> torch.Tensor:
    """uint8 CUDA tensor holding `data`, starting `offset` bytes past a 256-byte boundary."""
    buf = torch.empty(data.size + offset + 16, dtype=torch.uint8, device="cuda")
    view = buf[offset:offset + data.size]
    if data.size:
        view.copy_(torch.from_numpy(np.ascontiguousarray(data)))
    return view


def bitmap_to_cuts(words: torch.Tensor, n: int) -> np.ndarray:
    """Set bits p of a bitmap -> cut positions p + 1."""
    w = words.cpu().numpy().view(np.uint32)
    bits = np.unpackbits(w.view(np.uint8), bitorder="little")[:n]
    return (np.flatnonzero(bits) + 1).astype(np.uint64)


def _ncpu() -> int:
    import os
    return os.cpu_count() or 1


def oracle_digests_parallel(algo, data: np.ndarray, ends: np.ndarray, nthreads: int = 0) -> np.ndarray:
    """oracle.hash_chunks over all chunks, with the chunk list cut into ranges that
    threads digest independently (the oracle's C call releases the GIL)."""
    import concurrent.futures as cf

    import oracle
    nthreads = nthreads or _ncpu()
    ends = np.asarray(ends, dtype=np.uint64)
    k = ends.size
    if k == 0:
        return np.zeros((0, oracle.DIGEST_LEN[algo]), np.uint8)
    cuts = np.linspace(0, k, min(k, 4 * nthreads) + 1).astype(np.int64)

    def part(j):
        i0, i1 = int(cuts[j]), int(cuts[j + 1])
        if i1 <= i0:
            return np.zeros((0, oracle.DIGEST_LEN[algo]), np.uint8)
        s = int(ends[i0 - 1]) if i0 else 0
        return oracle.hash_chunks(algo, data[s:int(ends[i1 - 1])], ends[i0:i1] - np.uint64(s))

    with cf.ThreadPoolExecutor(nthreads) as ex:
        return np.concatenate(list(ex.map(part, range(cuts.size - 1))))


def oracle_files(data: np.ndarray, off, p, algo, nthreads: int = 0):
    """Per-file oracle chunk ends and digests of files stored back to back (file f is
    data[off[f]:off[f+1]]), each chunked on its own. Small files go to a thread pool
    one file per thread; large files use all threads inside the oracle."""
    import concurrent.futures as cf

    import oracle
    nthreads = nthreads or _ncpu()
    nfile = len(off) - 1
    big = 8 << 20

    def one(f, nt):
        body = data[int(off[f]):int(off[f + 1])]
        cands = oracle.window_candidates(body, p.window, p.mask_bits, p.magic, nthreads=nt,
                                         kind=p.window_hash)
        e = oracle.select(cands, body.size, p.min_chunk, p.max_chunk)
        dg = (oracle_digests_parallel(algo, body, e, nt) if nt > 1
              else oracle.hash_chunks(algo, body, e))
        return e, dg

    res = [None] * nfile
    sizes = np.diff(np.asarray(off, dtype=np.int64))
    small = [f for f in range(nfile) if sizes[f] < big]
    with cf.ThreadPoolExecutor(nthreads) as ex:
        for f, r in zip(small, ex.map(lambda f: one(f, 1), small)):
            res[f] = r
    for f in range(nfile):
        if sizes[f] >= big:
            res[f] = one(f, nthreads)
    return res
