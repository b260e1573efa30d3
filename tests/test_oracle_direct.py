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
