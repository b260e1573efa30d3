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
# (4096 * 64, 64), (4097 * 128 + 5, 128), (320_010, 64): exactly 4096 aligned
# blocks (half-warp chain layout) and just above it (four-warp CTAs)
SMALL = [(0, 4096), (1, 4096), (55, 4096), (56, 64), (63, 4096), (64, 4096), (4096, 4096),
         (4097, 4096), (1_000_003, 4096), (300_000, 65536), (3 << 20, 1 << 20), (5000, 7),
         (100_000, 64), (100_000, 100), (70_000, 120), (4096 * 64, 64), (4097 * 128 + 5, 128),
         (320_010, 64)]


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


# Enough blocks for the throughput kernels (148 x 512 = 75776 and up), an odd
# count (the two-block MD5 kernel's last thread hashes one block) and a short
# last block, at 32-byte (two-block MD5 kernel), 16-byte (one block per
# thread) and 8-byte (generic kernel) alignment; the roots take the host path.
@pytest.mark.parametrize("algo", ALGOS)
@pytest.mark.parametrize("block,extra", [(128, 77), (4096, 1234)])
@pytest.mark.parametrize("offset", [0, 16, 8])
def test_blocks_throughput_forms(hg, algo, block, extra, offset):
    nfull = 75777
    n = nfull * block + extra
    data = G.uniform_bytes(n, seed=block + extra)
    d = to_device(data, offset)
    assert d.data_ptr() % 32 == offset % 32
    dg, root = hg.hash_blocks(d, block, algo)
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


@pytest.mark.parametrize("algo", ALGOS)
def test_config_1gib_text_like(hg, algo):
    """1 GiB text-like (seed 5), 64 KiB blocks + hash-of-hashes."""
    data = G.text_like_bytes(1 << 30, seed=5)
    dg, root = hg.hash_blocks(to_device(data), 65536, algo)
    odg, oroot = oracle.hash_blocks(algo, data, 65536)
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


# ---------------------------------------------------------------- two-level identifiers
PMD_SMALL = [(0, 4096, 1024), (1, 4096, 1024), (4095, 4096, 1024), (4097, 4096, 1024),
             (1_000_003, 65536, 4096), (3 << 20, 1 << 20, 4096), (100_000, 700, 100),
             (70_000, 128, 64), (64, 64, 64), (200_000, 8192, 8192)]


@pytest.mark.parametrize("algo", ALGOS)
@pytest.mark.parametrize("n,block,segment", PMD_SMALL)
@pytest.mark.parametrize("offset", [0, 5])
def test_two_level_small(hg, algo, n, block, segment, offset):
    data = G.uniform_bytes(n, seed=n + block + segment)
    d = to_device(data, offset)
    ids = hg.hash_blocks_pmd(d, block, segment, algo)
    torch.cuda.synchronize()
    hg.sync()
    assert np.array_equal(ids.cpu().numpy(), oracle.hash_blocks_pmd(algo, data, block, segment))


@pytest.mark.parametrize("algo", ALGOS)
@pytest.mark.parametrize("block,segment", [(1 << 20, 4096), (65536, 4096)])
def test_two_level_1gib(hg, gib_uniform, algo, block, segment):
    d = to_device(gib_uniform)
    dl = 16 if algo == oracle.MD5 else 20
    seg = torch.empty(((1 << 30) // segment, dl), dtype=torch.uint8, device="cuda")
    ids = hg.hash_blocks_pmd(d, block, segment, algo, seg_out=seg)
    got = ids.cpu().numpy()
    # the segment digests are the plain fixed-block digests at the segment size
    sdg, _ = oracle.hash_blocks(algo, gib_uniform, segment, root=False)
    assert np.array_equal(seg.cpu().numpy(), sdg)
    want = oracle.hash_blocks_pmd(algo, gib_uniform, block, segment)
    assert np.array_equal(got, want)
    hg.sync()


def test_two_level_text_like(hg):
    data = G.text_like_bytes(5_000_017, seed=5)
    ids = hg.hash_blocks_pmd(to_device(data, 3), 1 << 20, 4096, oracle.SHA1)
    assert np.array_equal(ids.cpu().numpy(), oracle.hash_blocks_pmd(oracle.SHA1, data, 1 << 20, 4096))
    hg.sync()


def test_two_level_bad_arguments(hg):
    import paper_1202_3669_b300 as hgb
    d = to_device(G.uniform_bytes(10_000, 1))
    with pytest.raises(hgb.HashGPUError):
        hg.hash_blocks_pmd(d, 4096, 1000, hgb.MD5)           # block not a multiple of segment
    with pytest.raises(hgb.HashGPUError):
        hg.hash_blocks_pmd(d, 4096, 0, hgb.MD5)              # zero segment
    seg = torch.empty(64 * 16 + 8, dtype=torch.uint8, device="cuda")
    with pytest.raises(hgb.HashGPUError):
        hg.hash_blocks_pmd(d, 4096, 1024, hgb.MD5, seg_out=seg[4:])   # misaligned segment digests
    hg.sync()


def test_int_pipe_probe_runs():
    """The benchmark's integer-pipe probe (roofline denominators, its own library)
    launches and reports its operation count; bad arguments are refused."""
    import ctypes as C
    import os
    lib = C.CDLL(os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                              "paper_1202_3669_b300", "bench_probe", "libhgprobe.so"))
    lib.hgp_probe_int_pipe.argtypes = [C.c_int, C.c_int, C.c_uint32, C.c_uint32, C.c_void_p, C.c_void_p]
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    ops = C.c_uint64()
    s = torch.cuda.current_stream().cuda_stream
    for kind in range(5):
        assert lib.hgp_probe_int_pipe(0, kind, 64, 2, C.byref(ops), s) == 0
        assert ops.value == sms * 2 * 256 * 8 * 64 * (4 if kind == 3 else 1)
    assert lib.hgp_probe_int_pipe(0, 5, 64, 2, C.byref(ops), s) != 0
    torch.cuda.synchronize()
