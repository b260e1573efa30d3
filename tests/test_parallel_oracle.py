"""The parallel drivers the full-size GPU parity tests use around the oracle
(threads over chunk ranges and over files) give exactly the oracle's serial
results."""
import numpy as np

import oracle
from gen import inputs as G
from tests.gpu_util import oracle_digests_parallel, oracle_files


class _P:
    window, mask_bits, magic, min_chunk, max_chunk = 20, 9, 0x55, 256, 4096
    window_hash = oracle.WIN_MD5


def test_digests_parallel_equal_serial():
    data = G.uniform_bytes(3_000_000, seed=201)
    ends = oracle.cdc(data, 20, 9, 0x55, 256, 4096, nthreads=4)
    for algo in (oracle.MD5, oracle.SHA1):
        assert np.array_equal(oracle_digests_parallel(algo, data, ends, nthreads=5),
                              oracle.hash_chunks(algo, data, ends))
    assert oracle_digests_parallel(oracle.MD5, data[:0], ends[:0]).shape == (0, 16)


def test_files_parallel_equal_serial():
    sizes = np.array([0, 1, 20, 5000, 300_000, 9 << 20, 70_000, 0, 123_457])
    data, off = G.files_from_sizes(sizes, 202)
    res = oracle_files(data, off, _P, oracle.SHA1, nthreads=3)
    for f in range(sizes.size):
        body = data[off[f]:off[f + 1]]
        e = oracle.cdc(body, 20, 9, 0x55, 256, 4096)
        assert np.array_equal(res[f][0], e)
        assert np.array_equal(res[f][1], oracle.hash_chunks(oracle.SHA1, body, e))
