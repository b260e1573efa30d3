"""The C-ABI library loads on the CPU host and exports everything include/*.h declares.

No compute is called here (there is no GPU on the build host); only calls that
touch no device memory.
"""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
INCLUDE = os.path.join(ROOT, "include")


def declared_functions():
    names = set()
    for f in os.listdir(INCLUDE):
        if not f.endswith(".h"):
            continue
        src = open(os.path.join(INCLUDE, f)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names |= set(re.findall(r"\b(hg_\w+)\s*\(", src))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("hg_hash_blocks", "hg_cdc_boundaries", "hg_hash_chunks", "hg_init", "hg_destroy"):
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_1202_3669_b300 import _lib
    lib = C.CDLL(_lib.LIB_PATH)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_symbol():
    from paper_1202_3669_b300 import _lib
    assert set(declared_functions()) <= set(_lib.SIGNATURES)


def test_host_only_calls():
    from paper_1202_3669_b300 import _lib
    L = _lib.lib
    assert L.hg_digest_len(0) == 16 and L.hg_digest_len(1) == 20 and L.hg_digest_len(7) == -1
    assert L.hg_strerror(-3) == b"output capacity too small"
    p = _lib.default_params()
    assert (p.window, p.mask_bits, p.magic, p.min_chunk, p.max_chunk) == (20, 13, 0x0F0F, 2048, 65536)


def test_server_default_config():
    """Default server limits (host code): 1 GiB per wave at most, waves closed at 256 MiB."""
    from paper_1202_3669_b300 import _lib
    cfg = _lib.hg_server_config()
    _lib.lib.hg_server_default_config(C.byref(cfg))
    assert C.sizeof(cfg) == 64
    assert (cfg.device_budget, cfg.max_wave_bytes, cfg.wave_target_bytes) == (32 << 30, 1 << 30, 256 << 20)
    assert (cfg.max_wave_requests, cfg.max_inflight_waves, cfg.cdc.window) == (4096, 3, 20)


def test_exit_handler_closes_children_before_contexts():
    """The binding's exit handler releases servers, streams, block maps and batches
    before the contexts they were made on (host logic, with stand-in objects)."""
    import paper_1202_3669_b300 as hgb
    order = []

    class Stub:
        def __init__(self, name):
            self.name = name

        def _release(self):
            order.append(self.name)

    ctx, child = Stub("context"), Stub("batch")
    hgb._contexts.add(ctx)
    hgb._children.add(child)
    try:
        hgb._close_all()
    finally:
        hgb._contexts.discard(ctx)
        hgb._children.discard(child)
    assert order.index("batch") < order.index("context")


def test_init_without_gpu_fails_cleanly():
    import torch
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    from paper_1202_3669_b300 import _lib
    h = C.c_void_p()
    assert _lib.lib.hg_init(C.byref(h), 0, 0) == _lib.HG_ECUDA
    assert h.value is None


def test_cdc_hash_plan_is_host_only():
    import paper_1202_3669_b300 as hgb
    assert hgb.cdc_hash_plan(0) == []
    for n in (1, 8192, (16 << 20) + 1, 64 << 20, 67100231, 1 << 30, 5 << 30):
        b = hgb.cdc_hash_plan(n)
        assert b[0] == 0 and b[-1] == n and all(x < y for x, y in zip(b, b[1:]))
        assert all(x % 8192 == 0 for x in b[:-1]) and len(b) - 1 <= 64
        if n <= (64 << 20):
            assert b == [0, n]                          # small buffers: one pass
        else:
            assert all(y - x >= (16 << 20) for x, y in zip(b, b[1:]))


def test_pinned_size_classes_and_null_context():
    """Pinned-pool size classes (host arithmetic only) and argument errors."""
    from paper_1202_3669_b300 import _lib
    L = _lib.lib
    assert L.hg_pinned_class(0) == 0
    assert L.hg_pinned_class(1) == 64 << 10
    assert L.hg_pinned_class(64 << 10) == 64 << 10
    assert L.hg_pinned_class((64 << 10) + 1) == 80 << 10
    assert L.hg_pinned_class(1 << 20) == 1 << 20
    assert L.hg_pinned_class((1 << 20) + 1) == (1 << 20) + (1 << 18)
    assert L.hg_pinned_class(3 << 20) == 3 << 20
    for n in (100, 70_000, 999_999, 5 << 20, (5 << 20) + 1, 123_456_789):
        c = L.hg_pinned_class(n)
        assert n <= c <= max(64 << 10, n + n // 4 + 1)
    assert L.hg_alloc_pinned(None, 100) is None
    assert L.hg_free_pinned(None, None) == _lib.HG_EINVAL


def test_host_digest_equals_hashlib():
    """The library's host MD5/SHA-1 (used for the hash-of-hashes) against OpenSSL via
    hashlib at every length 0..1100 and on a MiB-sized input; no device needed."""
    import hashlib

    import numpy as np

    from paper_1202_3669_b300 import _lib
    g = np.random.default_rng(7)
    buf = g.integers(0, 256, (1 << 20) + 77, dtype=np.uint8)
    out = np.zeros(20, np.uint8)
    for algo, ref, dl in ((0, hashlib.md5, 16), (1, hashlib.sha1, 20)):
        for n in list(range(0, 1101)) + [buf.size]:
            assert _lib.lib.hg_host_digest(algo, buf.ctypes.data if n else None, n,
                                           out.ctypes.data) == 0
            assert out[:dl].tobytes() == ref(buf[:n].tobytes()).digest(), (algo, n)
    assert _lib.lib.hg_host_digest(7, None, 0, out.ctypes.data) == _lib.HG_EINVAL
