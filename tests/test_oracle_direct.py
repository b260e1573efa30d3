"""Pins of direct hashing and the hash-of-hashes (Sec. 3.2.2) against hashlib."""
import hashlib

import numpy as np
import pytest

import oracle
from gen import inputs as G
from tests.pins import ref_digest


@pytest.mark.parametrize("algo", [oracle.MD5, oracle.SHA1])
@pytest.mark.parametrize("n,block", [(0, 4096), (1, 4096), (4096, 4096), (4097, 4096),
                                     (8 << 20, 4096), (300_000, 65536), (1000, 7), (5000, 64)])
def test_blocks_and_root(algo, n, block):
    data = G.uniform_bytes(n, seed=n + block).tobytes()
    dg, root = oracle.hash_blocks(algo, data, block)
    nblk = (n + block - 1) // block
    assert dg.shape[0] == nblk
    for i in range(nblk):
        assert dg[i].tobytes() == ref_digest(algo, data[i * block:(i + 1) * block]), i
    assert root == ref_digest(algo, b"".join(ref_digest(algo, data[i * block:(i + 1) * block])
                                             for i in range(nblk)))


def test_single_block_root_is_hash_of_hash():
    data = b"storage system accelerator" * 10
    _, root = oracle.hash_blocks(oracle.MD5, data, 4096)
    assert root == hashlib.md5(hashlib.md5(data).digest()).digest()


def test_empty_root_is_hash_of_empty():
    _, root = oracle.hash_blocks(oracle.SHA1, b"", 4096)
    assert root == hashlib.sha1(b"").digest()


@pytest.mark.parametrize("algo", [oracle.MD5, oracle.SHA1])
def test_chunks(algo):
    data = G.uniform_bytes(50_000, seed=3).tobytes()
    ends = np.array([1, 2, 100, 4000, 4000 + 64, 30_000, 50_000], np.uint64)
    dg = oracle.hash_chunks(algo, data, ends)
    s = 0
    for i, e in enumerate(ends):
        assert dg[i].tobytes() == ref_digest(algo, data[s:int(e)])
        s = int(e)


def _pmd_ref(algo, data, block, segment):
    """hashlib restatement: per block, the digest of its segment digests."""
    ids = []
    for lo in range(0, len(data), block):
        blk = data[lo:lo + block]
        segs = [ref_digest(algo, blk[a:a + segment]) for a in range(0, len(blk), segment)]
        ids.append(ref_digest(algo, b"".join(segs)))
    return ids


@pytest.mark.parametrize("algo", [oracle.MD5, oracle.SHA1])
@pytest.mark.parametrize("n,block,segment", [(0, 4096, 1024), (1, 4096, 1024), (4096, 4096, 1024),
                                             (4097, 4096, 1024), (300_001, 65536, 4096),
                                             (1 << 20, 1 << 20, 4096), (5000, 100, 10),
                                             (10_000, 64, 64)])
def test_two_level_ids(algo, n, block, segment):
    data = G.uniform_bytes(n, seed=n + block + segment).tobytes()
    ids = oracle.hash_blocks_pmd(algo, data, block, segment)
    assert [r.tobytes() for r in ids] == _pmd_ref(algo, data, block, segment)


def test_two_level_with_one_segment_is_hash_of_hash():
    data = G.uniform_bytes(3 * 4096 + 5, seed=77).tobytes()
    ids = oracle.hash_blocks_pmd(oracle.SHA1, data, 4096, 4096)
    for i, lo in enumerate(range(0, len(data), 4096)):
        assert ids[i].tobytes() == hashlib.sha1(hashlib.sha1(data[lo:lo + 4096]).digest()).digest()


def test_two_level_single_block_equals_root_of_segments():
    # one block covering the input: its id is the hash-of-hashes over the segments
    data = G.uniform_bytes(50_000, seed=78).tobytes()
    ids = oracle.hash_blocks_pmd(oracle.MD5, data, 1 << 16, 1024)
    segs = b"".join(hashlib.md5(data[a:a + 1024]).digest() for a in range(0, len(data), 1024))
    assert ids.shape[0] == 1 and ids[0].tobytes() == hashlib.md5(segs).digest()


def test_two_level_rejects_block_not_multiple_of_segment():
    L = oracle.lib()
    import numpy as _np
    a = _np.zeros(100, _np.uint8)
    ids = _np.zeros((2, 16), _np.uint8)
    assert L.hgo_hash_blocks_pmd(oracle.MD5, a.ctypes.data, 100, 96, 64, ids.ctypes.data) == -1
