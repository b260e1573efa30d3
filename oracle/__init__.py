"""HashGPU CPU oracle -- test infrastructure only.

A plain, slow C99 restatement of the hashing hot path (md5.c, sha1.c,
direct.c, cdc.c) behind a ctypes wrapper. Only the test-suite, the smoke check
and the benchmark's CPU-baseline leg load it; the product never does. It
shares no code with the CUDA library.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from .build import LIB, build

MD5, SHA1 = 0, 1
DIGEST_LEN = {MD5: 16, SHA1: 20}

_lib = None


def lib(path: str | None = None) -> C.CDLL:
    global _lib
    if path is not None:
        return _bind(C.CDLL(path))
    if _lib is None:
        _lib = _bind(C.CDLL(build()))
    return _lib


def _bind(L: C.CDLL) -> C.CDLL:
    u8p, u64p = C.c_void_p, C.c_void_p
    L.hgo_md5.argtypes = [u8p, C.c_uint64, u8p]
    L.hgo_sha1.argtypes = [u8p, C.c_uint64, u8p]
    L.hgo_digest.argtypes = [C.c_int, u8p, C.c_uint64, u8p]
    L.hgo_digest.restype = C.c_int
    L.hgo_hash_blocks.argtypes = [C.c_int, u8p, C.c_uint64, C.c_uint64, u8p, u8p]
    L.hgo_hash_blocks.restype = C.c_int64
    L.hgo_hash_blocks_pmd.argtypes = [C.c_int, u8p, C.c_uint64, C.c_uint64, C.c_uint64, u8p]
    L.hgo_hash_blocks_pmd.restype = C.c_int64
    L.hgo_window_hash.argtypes = [u8p, C.c_uint32]
    L.hgo_window_hash.restype = C.c_uint32
    L.hgo_window_candidates.argtypes = [u8p, C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint32,
                                        u64p, C.c_uint64, C.c_int]
    L.hgo_window_candidates.restype = C.c_uint64
    L.hgo_rabin_fingerprint.argtypes = [u8p, C.c_uint64]
    L.hgo_rabin_fingerprint.restype = C.c_uint32
    L.hgo_window_candidates_kind.argtypes = [u8p, C.c_uint64, C.c_int, C.c_uint32, C.c_uint32,
                                             C.c_uint32, u64p, C.c_uint64, C.c_int]
    L.hgo_window_candidates_kind.restype = C.c_uint64
    L.hgo_select.argtypes = [u64p, C.c_uint64, C.c_uint64, C.c_uint64, C.c_uint64, u64p, C.c_uint64]
    L.hgo_select.restype = C.c_uint64
    L.hgo_hash_chunks.argtypes = [C.c_int, u8p, u64p, C.c_uint64, u8p]
    L.hgo_hash_chunks.restype = C.c_int
    return L


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data if a.size else 0


def _u8(data) -> np.ndarray:
    if isinstance(data, (bytes, bytearray, memoryview)):
        return np.frombuffer(bytes(data), dtype=np.uint8)
    return np.ascontiguousarray(data, dtype=np.uint8)


def digest(algo: int, data, L=None) -> bytes:
    L = L or lib()
    a = _u8(data)
    out = np.zeros(DIGEST_LEN[algo], np.uint8)
    assert L.hgo_digest(algo, _ptr(a), a.size, _ptr(out)) == 0
    return out.tobytes()


def md5(data, L=None) -> bytes:
    return digest(MD5, data, L)


def sha1(data, L=None) -> bytes:
    return digest(SHA1, data, L)


def hash_blocks(algo: int, data, block: int, root: bool = True, L=None):
    """(digests uint8[nblk, dlen], root bytes or None)."""
    L = L or lib()
    a = _u8(data)
    dl = DIGEST_LEN[algo]
    nblk = (a.size + block - 1) // block
    dg = np.zeros((nblk, dl), np.uint8)
    rt = np.zeros(dl, np.uint8)
    got = L.hgo_hash_blocks(algo, _ptr(a), a.size, block, _ptr(dg), rt.ctypes.data if root else None)
    assert got == nblk
    return dg, (rt.tobytes() if root else None)


def hash_blocks_pmd(algo: int, data, block: int, segment: int, L=None):
    """Two-level block identifiers, uint8[nblk, dlen]."""
    L = L or lib()
    a = _u8(data)
    dl = DIGEST_LEN[algo]
    nblk = (a.size + block - 1) // block
    ids = np.zeros((max(nblk, 1), dl), np.uint8)
    got = L.hgo_hash_blocks_pmd(algo, _ptr(a), a.size, block, segment, _ptr(ids))
    assert got == nblk
    return ids[:nblk]


def window_hash(win, L=None) -> int:
    L = L or lib()
    a = _u8(win)
    return int(L.hgo_window_hash(_ptr(a), a.size))


WIN_MD5, WIN_RABIN = 0, 1
RABIN_POLY = 0x9E3779BB


def rabin_fingerprint(msg, L=None) -> int:
    L = L or lib()
    a = _u8(msg)
    return int(L.hgo_rabin_fingerprint(_ptr(a), a.size))


def window_candidates(data, window: int = 20, mask_bits: int = 13, magic: int = 0x0F0F,
                      nthreads: int = 1, L=None, kind: int = WIN_MD5) -> np.ndarray:
    """Sorted candidate cut positions (uint64); kind picks the MD5 or the Rabin window."""
    L = L or lib()
    a = _u8(data)
    if kind == WIN_MD5:
        cnt = L.hgo_window_candidates(_ptr(a), a.size, window, mask_bits, magic, None, 0, nthreads)
    else:
        cnt = L.hgo_window_candidates_kind(_ptr(a), a.size, kind, window, mask_bits, magic, None,
                                           0, nthreads)
    assert cnt != 2 ** 64 - 1, kind
    out = np.zeros(cnt, np.uint64)
    if cnt:
        if kind == WIN_MD5:
            got = L.hgo_window_candidates(_ptr(a), a.size, window, mask_bits, magic,
                                          _ptr(out), cnt, nthreads)
        else:
            got = L.hgo_window_candidates_kind(_ptr(a), a.size, kind, window, mask_bits, magic,
                                               _ptr(out), cnt, nthreads)
        assert got == cnt
    return out


def select(cands, n: int, min_chunk: int, max_chunk: int, L=None) -> np.ndarray:
    """Chunk end offsets (uint64), the last equal to n."""
    L = L or lib()
    c = np.ascontiguousarray(cands, dtype=np.uint64)
    cap = n // max(1, min_chunk) + 2
    out = np.zeros(cap, np.uint64)
    cnt = L.hgo_select(_ptr(c), c.size, n, min_chunk, max_chunk, _ptr(out), cap)
    assert cnt <= cap
    return out[:cnt].copy()


def hash_chunks(algo: int, data, ends, L=None) -> np.ndarray:
    L = L or lib()
    a = _u8(data)
    e = np.ascontiguousarray(ends, dtype=np.uint64)
    out = np.zeros((e.size, DIGEST_LEN[algo]), np.uint8)
    assert L.hgo_hash_chunks(algo, _ptr(a), _ptr(e), e.size, _ptr(out)) == 0
    return out


def cdc(data, window: int = 20, mask_bits: int = 13, magic: int = 0x0F0F,
        min_chunk: int = 2048, max_chunk: int = 65536, nthreads: int = 1, L=None,
        kind: int = WIN_MD5) -> np.ndarray:
    """Chunk ends of the whole content-defined chunking step."""
    a = _u8(data)
    c = window_candidates(a, window, mask_bits, magic, nthreads, L, kind)
    return select(c, a.size, min_chunk, max_chunk, L)


def blockmap_hits(known_digests, query_digests) -> np.ndarray:
    """Similarity detection by block identifiers (Sec. 2.1: comparing hash values
    detects identical blocks; Sec. 4.3: the share of a new version's data found in
    chunks already stored): hit[i] is True when query digest i equals one of the
    known digests. Plain set membership over the full digest bytes."""
    seen = {bytes(d) for d in np.asarray(known_digests, dtype=np.uint8)}
    return np.array([bytes(d) in seen for d in np.asarray(query_digests, dtype=np.uint8)], dtype=bool)


def shared_bytes(known_digests, ends, query_digests) -> tuple[int, int]:
    """(number of query chunks found, bytes in them); chunk i of the queried version
    is [ends[i-1] (0 for i = 0), ends[i])."""
    hits = blockmap_hits(known_digests, query_digests)
    e = np.asarray(ends, dtype=np.int64)
    sizes = np.diff(np.concatenate([[0], e])) if e.size else np.zeros(0, np.int64)
    return int(hits.sum()), int(sizes[hits].sum()) if hits.size else 0


def shared_fraction(ends_v1, dig_v1, ends_v2, dig_v2) -> float:
    """Bytes of v2 in chunks whose digest also names a v1 chunk, over len(v2)."""
    seen = {bytes(d) for d in np.asarray(dig_v1)}
    e2 = np.asarray(ends_v2, dtype=np.int64)
    if e2.size == 0:
        return 0.0
    sizes = np.diff(np.concatenate([[0], e2]))
    shared = sum(int(s) for s, d in zip(sizes, np.asarray(dig_v2)) if bytes(d) in seen)
    return shared / float(e2[-1])
