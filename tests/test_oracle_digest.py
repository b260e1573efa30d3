"""Pins of the oracle's MD5 / SHA-1 (RFC 1321, FIPS 180-4) against hashlib and coreutils."""
import hashlib
import shutil
import subprocess

import numpy as np
import pytest

import oracle
from gen import inputs as G
from tests.pins import ref_digest


@pytest.mark.parametrize("algo", [oracle.MD5, oracle.SHA1])
def test_every_length_0_to_2048(algo):
    buf = G.uniform_bytes(2048, seed=101).tobytes()
    L = oracle.lib()
    for n in range(0, 2049):
        assert oracle.digest(algo, buf[:n], L) == ref_digest(algo, buf[:n]), n


@pytest.mark.parametrize("algo", [oracle.MD5, oracle.SHA1])
@pytest.mark.parametrize("n", [1 << 20, 3 * (1 << 20) + 17])
def test_large_random(algo, n):
    buf = G.uniform_bytes(n, seed=n).tobytes()
    assert oracle.digest(algo, buf) == ref_digest(algo, buf)


@pytest.mark.parametrize("algo,tool", [(oracle.MD5, "md5sum"), (oracle.SHA1, "sha1sum")])
def test_coreutils(tmp_path, algo, tool):
    if shutil.which(tool) is None:
        pytest.skip(f"{tool} missing")
    data = G.text_like_bytes(100_003, seed=7).tobytes()
    p = tmp_path / "x.bin"
    p.write_bytes(data)
    out = subprocess.run([tool, str(p)], capture_output=True, text=True, check=True).stdout
    assert oracle.digest(algo, data).hex() == out.split()[0]


def test_constant_inputs():
    for v in (0, 0x80, 0xFF):
        for n in (55, 56, 63, 64, 119, 120, 4096):
            data = bytes([v]) * n
            assert oracle.md5(data) == hashlib.md5(data).digest()
            assert oracle.sha1(data) == hashlib.sha1(data).digest()
