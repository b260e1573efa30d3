"""GPU parity of direct hashing (Sec. 2.1, Sec. 3.2.2) against the CPU oracle.

Digests are exact, so every comparison is byte for byte.
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


ALGOS = [oracle.MD5, oracle.SHA1]
SMALL = [(0, 4096), (1, 4096), (55, 4096), (56, 64), (63, 4096), (64, 4096), (4096, 4096),
         (4097, 4096), (1_000_003, 4096), (300_000, 65536), (3 << 20, 1 << 20), (5000, 7),
         (100_000, 64), (100_000, 100), (70_000, 120)]


@pytest.mark.parametrize("algo", ALGOS)
@pytest.mark.parametrize("n,block", SMALL)
@pytest.mark.parametrize("offset", [0, 1, 6, 12])
def test_blocks_small(hg, algo, n, block, offset):
    data = G.uniform_bytes(n, seed=n + block)
    d = to_device(data, offset)
    dg, root = hg.hash_blocks(d, block, algo)
    torch.cuda.synchronize()
    hg.sync()
    odg, oroot = oracle.hash_blocks(algo, data, block)
    assert np.array_equal(dg.cpu().numpy(), odg)
    assert root.cpu().numpy().tobytes() == oroot


@pytest.mark.parametrize("algo", ALGOS)
def test_config_direct_8mib(hg, algo):
    """8 MiB seeded uniform buffer, 2048 blocks of 4 KiB, digests + hash-of-hashes."""
    data = G.uniform_bytes(8 << 20, seed=1)
    dg, root = hg.hash_blocks(to_device(data), 4096, algo)
    odg, oroot = oracle.hash_blocks(algo, data, 4096)
    assert dg.shape[0] == 2048
    assert np.array_equal(dg.cpu().numpy(), odg)
    assert root.cpu().numpy().tobytes() == oroot
    hg.sync()


@pytest.fixture(scope="module")
def gib_uniform():
    return G.uniform_bytes(1 << 30, seed=4)


@pytest.mark.parametrize("algo", ALGOS)
@pytest.mark.parametrize("block", [4096, 65536, 1 << 20])
def test_config_1gib_uniform(hg, gib_uniform, algo, block):
    d = to_device(gib_uniform)
    dg, root = hg.hash_blocks(d, block, algo)
    odg, oroot = oracle.hash_blocks(algo, gib_uniform, block)
    assert np.array_equal(dg.cpu().numpy(), odg)
    assert root.cpu().numpy().tobytes() == oroot
    hg.sync()


def test_bad_arguments(hg):
    import paper_1202_3669_b300 as hgb
    d = to_device(G.uniform_bytes(100, 1))
    with pytest.raises(hgb.HashGPUError):
        hg.hash_blocks(d, 0, hgb.MD5)                      # block size 0
    out = torch.empty(64, dtype=torch.uint8, device="cuda")
    with pytest.raises(hgb.HashGPUError):
        hg.hash_blocks(d, 64, hgb.MD5, out=out[1:33])       # misaligned digests
    hg.sync()
