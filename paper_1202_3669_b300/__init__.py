"""HashGPU on B300: direct hashing and content-defined chunking on the GPU.

`Context` wraps the C ABI (include/hashgpu.h) for torch CUDA tensors: torch
provides device memory and streams, the CUDA library does all the work. The
raw C functions are re-exported under their C names from `_lib`.
"""
from __future__ import annotations

import torch

from . import _lib
from ._lib import (HG_MD5, HG_SHA1, HashGPUError, check, default_params,  # noqa: F401
                   hg_cdc_boundaries, hg_cdc_candidates, hg_cdc_params, hg_destroy,
                   hg_digest_len, hg_hash_blocks, hg_hash_chunks, hg_init, hg_reserve,
                   hg_scratch_bytes, hg_sync, hg_window_bitmap)

MD5, SHA1 = HG_MD5, HG_SHA1
DIGEST_LEN = {MD5: 16, SHA1: 20}


def params(window=20, mask_bits=13, magic=0x0F0F, min_chunk=2048, max_chunk=65536) -> hg_cdc_params:
    p = hg_cdc_params()
    p.window, p.mask_bits, p.magic, p.reserved = window, mask_bits, magic, 0
    p.min_chunk, p.max_chunk = min_chunk, max_chunk
    return p


def _ptr(t: torch.Tensor | None) -> int | None:
    if t is None:
        return None
    return t.data_ptr() if t.numel() else None


def _stream(stream) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


class Context:
    """One library context on one CUDA device (scratch memory under a budget)."""

    def __init__(self, device: int = 0, budget: int = 0):
        if not torch.cuda.is_available():
            raise RuntimeError("HashGPU needs a CUDA device")
        self.device = torch.device("cuda", device)
        self.h = hg_init(device, budget)

    def close(self):
        if getattr(self, "h", None):
            hg_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def sync(self, stream=None) -> None:
        check(hg_sync(self.h, _stream(stream)), "device error")

    def reserve(self, max_bytes: int) -> None:
        check(hg_reserve(self.h, max_bytes), "hg_reserve")

    # ---------------------------------------------------------------------------------------
    def hash_blocks(self, data: torch.Tensor, block: int, algo: int = MD5, root: bool = True,
                    out: torch.Tensor | None = None, root_out: torch.Tensor | None = None,
                    stream=None):
        n = data.numel()
        nblk = (n + block - 1) // block if block > 0 else 0
        dl = DIGEST_LEN.get(algo, 16)
        if out is None:
            out = torch.empty((nblk, dl), dtype=torch.uint8, device=self.device)
        if root and root_out is None:
            root_out = torch.empty(dl, dtype=torch.uint8, device=self.device)
        check(hg_hash_blocks(self.h, algo, _ptr(data), n, block, _ptr(out),
                             _ptr(root_out) if root else None, _stream(stream)), "hg_hash_blocks")
        return out, (root_out if root else None)

    def window_bitmap(self, data: torch.Tensor, p: hg_cdc_params | None = None,
                      out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        p = p or default_params()
        n = data.numel()
        if out is None:
            out = torch.empty((n + 31) // 32, dtype=torch.int32, device=self.device)
        check(hg_window_bitmap(self.h, _ptr(data), n, p, _ptr(out), _stream(stream)),
              "hg_window_bitmap")
        return out

    def cdc_candidates(self, data: torch.Tensor, p: hg_cdc_params | None = None,
                       cap: int | None = None, stream=None):
        p = p or default_params()
        n = data.numel()
        cap = cap if cap is not None else n // 64 + 1024
        out = torch.empty(max(cap, 1), dtype=torch.int64, device=self.device)
        cnt = torch.zeros(1, dtype=torch.int64, device=self.device)
        check(hg_cdc_candidates(self.h, _ptr(data), n, p, _ptr(out), cap, _ptr(cnt),
                                _stream(stream)), "hg_cdc_candidates")
        return out, cnt

    def cdc_boundaries(self, data: torch.Tensor, p: hg_cdc_params | None = None,
                       cap: int | None = None, out: torch.Tensor | None = None,
                       count: torch.Tensor | None = None, stream=None):
        p = p or default_params()
        n = data.numel()
        if cap is None:
            cap = out.numel() if out is not None else n // p.min_chunk + 2
        if out is None:
            out = torch.empty(max(cap, 1), dtype=torch.int64, device=self.device)
        if count is None:
            count = torch.zeros(1, dtype=torch.int64, device=self.device)
        check(hg_cdc_boundaries(self.h, _ptr(data), n, p, _ptr(out), cap, _ptr(count),
                                _stream(stream)), "hg_cdc_boundaries")
        return out, count

    def hash_chunks(self, data: torch.Tensor, ends: torch.Tensor, algo: int = MD5,
                    count: torch.Tensor | None = None, out: torch.Tensor | None = None,
                    stream=None) -> torch.Tensor:
        nchunk = ends.numel()
        if out is None:
            out = torch.empty((nchunk, DIGEST_LEN[algo]), dtype=torch.uint8, device=self.device)
        check(hg_hash_chunks(self.h, algo, _ptr(data), data.numel(), _ptr(ends), nchunk,
                             _ptr(count), _ptr(out), _stream(stream)), "hg_hash_chunks")
        return out

    def cdc(self, data: torch.Tensor, algo: int = MD5, p: hg_cdc_params | None = None,
            stream=None):
        """Boundaries then per-chunk digests, chained on one stream without a host sync.
        Returns (ends, count, digests); ends/digests hold count valid rows."""
        ends, count = self.cdc_boundaries(data, p, stream=stream)
        dg = self.hash_chunks(data, ends, algo, count=count, stream=stream)
        return ends, count, dg
