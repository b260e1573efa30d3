"""HashGPU on B300: direct hashing and content-defined chunking on the GPU.

`Context` wraps the C ABI (include/hashgpu.h) for torch CUDA tensors: torch
provides device memory and streams, the CUDA library does all the work. The
raw C functions are re-exported under their C names from `_lib`.
"""
from __future__ import annotations

import atexit
import ctypes as C
import sys
import weakref

import numpy as np
import torch

from . import _lib
from ._lib import (HG_MD5, HG_SHA1, HashGPUError, check, default_params,  # noqa: F401
                   hg_batch_autotune, hg_batch_autotune_cached, hg_batch_cdc_hash, hg_batch_cdc_hash_graph, hg_batch_create,
                   hg_batch_destroy, hg_batch_get_tuning, hg_batch_set_tuning, hg_batch_slots,
                   hg_batch_sync, hg_batch_tuning, hg_cdc_boundaries, hg_cdc_boundaries_static,
                   hg_cdc_candidates, hg_cdc_params, hg_destroy, hg_digest_len, hg_hash_blocks,
                   hg_hash_blocks_pmd, hg_hash_chunks, hg_init, hg_reserve, hg_scratch_bytes, hg_sync, hg_window_bitmap,
                   HG_REQ_BLOCKS, HG_REQ_CDC, hg_cancel, hg_poll, hg_release, hg_request, hg_result,
                   hg_server_config, hg_server_create, hg_server_default_config, hg_server_destroy,
                   hg_server_get_stats, hg_server_replay, hg_server_stats, hg_server_wait_any,
                   hg_submit, hg_cdc_hash, hg_cdc_hash_plan, hg_cdc_hash_h2d, hg_stream_open,
                   hg_stream_feed, hg_stream_close, hg_stream_destroy, hg_blockmap_create,
                   hg_blockmap_insert, hg_blockmap_lookup, hg_blockmap_count, hg_blockmap_clear,
                   hg_blockmap_destroy, hg_alloc_pinned, hg_free_pinned,
                   hg_pinned_set_budget, hg_pinned_trim, hg_pinned_stats, hg_pinned_class,
                   hg_pinned_info)

MD5, SHA1 = HG_MD5, HG_SHA1
DIGEST_LEN = {MD5: 16, SHA1: 20}

# Library objects still open when the interpreter exits are closed by an exit
# handler, servers, streams, block maps and batches before the contexts they were
# made on, while the CUDA runtime and this module are still intact. Finalizers that
# run later, during interpreter teardown, do not call into the library.
_children: "weakref.WeakSet" = weakref.WeakSet()
_contexts: "weakref.WeakSet" = weakref.WeakSet()


@atexit.register
def _close_all() -> None:
    for group in (_children, _contexts):
        for obj in list(group):
            try:
                obj._release()
            except Exception:
                pass


def _finalizer_may_call() -> bool:
    return not sys.is_finalizing()


WIN_MD5, WIN_RABIN = 0, 1


def params(window=20, mask_bits=13, magic=0x0F0F, min_chunk=2048, max_chunk=65536,
           window_hash=WIN_MD5) -> hg_cdc_params:
    p = hg_cdc_params()
    p.window, p.mask_bits, p.magic, p.window_hash = window, mask_bits, magic, window_hash
    p.min_chunk, p.max_chunk = min_chunk, max_chunk
    return p


def cdc_hash_plan(n: int) -> list[int]:
    """Segment bounds hg_cdc_hash uses for an n-byte buffer."""
    k = hg_cdc_hash_plan(n, None, 0)
    b = np.zeros(k + 1, dtype=np.uint64)
    hg_cdc_hash_plan(n, b.ctypes.data, k + 1)
    return [int(x) for x in b] if k else []


def _ptr(t: torch.Tensor | None) -> int | None:
    if t is None:
        return None
    return t.data_ptr() if t.numel() else None


def _stream(stream) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


class PinnedBuffer:
    """A page-locked host buffer from a context's pool (hg_alloc_pinned).

    `tensor` is a uint8 CPU tensor of the requested length over the buffer. The
    driver treats the memory as page-locked (copies from and to it are one DMA and
    asynchronous), although torch's `is_pinned()` only knows its own allocator. It
    must not be used after `free()`, which gives the buffer back to the pool.
    """

    def __init__(self, ctx: "Context", nbytes: int):
        self.ctx, self.nbytes = ctx, int(nbytes)
        self.ptr = hg_alloc_pinned(ctx.h, self.nbytes)
        if not self.ptr:
            raise HashGPUError(_lib.HG_ENOMEM, "hg_alloc_pinned")
        raw = (C.c_uint8 * self.nbytes).from_address(self.ptr)
        self.tensor = torch.from_numpy(np.ctypeslib.as_array(raw))
        ctx._pinned.add(self)

    def numpy(self) -> np.ndarray:
        return self.tensor.numpy()

    def free(self) -> None:
        if self.ptr and self.ctx.h:
            check(hg_free_pinned(self.ctx.h, self.ptr), "hg_free_pinned")
        self.ctx._pinned.discard(self)
        self.ptr, self.tensor = None, None


class Context:
    """One library context on one CUDA device (scratch memory under a budget)."""

    def __init__(self, device: int = 0, budget: int = 0):
        if not torch.cuda.is_available():
            raise RuntimeError("HashGPU needs a CUDA device")
        self.device = torch.device("cuda", device)
        self.h = hg_init(device, budget)
        self._pinned = set()
        _contexts.add(self)

    def close(self):
        if getattr(self, "h", None):
            for b in list(getattr(self, "_pinned", ())):   # hg_destroy releases the pool
                b.ptr, b.tensor = None, None
            self._pinned = set()
            hg_destroy(self.h)
            self.h = None

    # ---------------------------------------------------------------------------------------
    def alloc_pinned(self, nbytes: int) -> PinnedBuffer:
        """A pinned host buffer of nbytes from this context's pool."""
        return PinnedBuffer(self, nbytes)

    def pinned_stats(self) -> dict:
        info = hg_pinned_info()
        check(hg_pinned_stats(self.h, info), "hg_pinned_stats")
        return {k: int(getattr(info, k)) for k, _ in info._fields_}

    def set_pinned_budget(self, nbytes: int) -> None:
        check(hg_pinned_set_budget(self.h, nbytes), "hg_pinned_set_budget")

    def trim_pinned(self) -> None:
        check(hg_pinned_trim(self.h), "hg_pinned_trim")

    def _release(self):
        self.close()

    def __del__(self):
        try:
            if _finalizer_may_call():
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

    def hash_blocks_pmd(self, data: torch.Tensor, block: int, segment: int, algo: int = MD5,
                        out: torch.Tensor | None = None, seg_out: torch.Tensor | None = None,
                        stream=None) -> torch.Tensor:
        """Two-level block identifiers (H of each block's segment digests)."""
        n = data.numel()
        nblk = (n + block - 1) // block if block > 0 else 0
        dl = DIGEST_LEN.get(algo, 16)
        if out is None:
            out = torch.empty((nblk, dl), dtype=torch.uint8, device=self.device)
        check(hg_hash_blocks_pmd(self.h, algo, _ptr(data), n, block, segment,
                                 _ptr(seg_out) if seg_out is not None else None, _ptr(out),
                                 _stream(stream)), "hg_hash_blocks_pmd")
        return out

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

    def cdc_hash(self, data: torch.Tensor, algo: int = MD5, p: hg_cdc_params | None = None,
                 out=None, stream=None):
        """Pipelined boundaries + digests (hg_cdc_hash). Returns (ends, count, digests)."""
        p = p or default_params()
        n = data.numel()
        cap = n // p.min_chunk + 2
        if out is None:
            out = (torch.empty(cap, dtype=torch.int64, device=self.device),
                   torch.zeros(1, dtype=torch.int64, device=self.device),
                   torch.empty((cap, DIGEST_LEN[algo]), dtype=torch.uint8, device=self.device))
        ends, count, dg = out
        check(hg_cdc_hash(self.h, algo, _ptr(data), n, p, _ptr(ends), ends.numel(), _ptr(count),
                          _ptr(dg), _stream(stream)), "hg_cdc_hash")
        return ends, count, dg

    def cdc_hash_from_host(self, host: torch.Tensor, dev: torch.Tensor, algo: int = MD5,
                           p: hg_cdc_params | None = None, out=None, stream=None):
        """hg_cdc_hash_h2d: copy the (pinned) host bytes into dev in pieces, overlapped with
        the chunking. Returns (ends, count, digests)."""
        p = p or default_params()
        n = host.numel()
        assert dev.numel() >= n
        cap = n // p.min_chunk + 2
        if out is None:
            out = (torch.empty(cap, dtype=torch.int64, device=self.device),
                   torch.zeros(1, dtype=torch.int64, device=self.device),
                   torch.empty((cap, DIGEST_LEN[algo]), dtype=torch.uint8, device=self.device))
        ends, count, dg = out
        check(hg_cdc_hash_h2d(self.h, algo, _ptr(host), _ptr(dev), n, p, _ptr(ends), ends.numel(),
                              _ptr(count), _ptr(dg), _stream(stream)), "hg_cdc_hash_h2d")
        return ends, count, dg

    def cdc(self, data: torch.Tensor, algo: int = MD5, p: hg_cdc_params | None = None,
            stream=None):
        """Boundaries then per-chunk digests, chained on one stream without a host sync.
        Returns (ends, count, digests); ends/digests hold count valid rows."""
        ends, count = self.cdc_boundaries(data, p, stream=stream)
        dg = self.hash_chunks(data, ends, algo, count=count, stream=stream)
        return ends, count, dg


class Batch:
    """Many files stored back to back in one device buffer, chunked and hashed in one pass.

    file_off: nfile + 1 byte offsets (file f = bytes [file_off[f], file_off[f+1])).
    Results use the slot layout of include/hashgpu.h: chunk i of file f ends at
    ends[slot_off[f] + i] (relative to the file start), with its digest in the same row.
    """

    def __init__(self, ctx: Context, file_off, p: hg_cdc_params | None = None):
        self.ctx = ctx
        self.p = p or default_params()
        self.file_off = np.ascontiguousarray(file_off, dtype=np.uint64)
        self.nfile = self.file_off.size - 1
        self.h = hg_batch_create(ctx.h, self.file_off.ctypes.data, self.nfile, self.p)
        _children.add(self)
        self.slot_off = np.zeros(self.nfile + 1, dtype=np.uint64)
        self.total_slots = hg_batch_slots(self.h, self.slot_off.ctypes.data)

    def close(self):
        if getattr(self, "h", None):
            hg_batch_destroy(self.h)
            self.h = None

    def _release(self):
        self.close()

    def __del__(self):
        try:
            if _finalizer_may_call():
                self.close()
        except Exception:
            pass

    def outputs(self, algo: int):
        dev = self.ctx.device
        return (torch.empty(max(1, self.total_slots), dtype=torch.int64, device=dev),
                torch.zeros(max(1, self.nfile), dtype=torch.int64, device=dev),
                torch.empty((max(1, self.total_slots), DIGEST_LEN[algo]), dtype=torch.uint8,
                            device=dev))

    def cdc_hash(self, data: torch.Tensor, algo: int = SHA1, out=None, graph: bool = False,
                 stream=None):
        ends, counts, dg = out if out is not None else self.outputs(algo)
        fn = hg_batch_cdc_hash_graph if graph else hg_batch_cdc_hash
        check(fn(self.h, algo, _ptr(data), _ptr(ends), _ptr(counts), _ptr(dg), _stream(stream)),
              "hg_batch_cdc_hash")
        return ends, counts, dg

    def sync(self, stream=None):
        check(hg_batch_sync(self.h, _stream(stream)), "batch device error")

    def tuning(self) -> hg_batch_tuning:
        t = hg_batch_tuning()
        check(hg_batch_get_tuning(self.h, t))
        return t

    def set_tuning(self, t: hg_batch_tuning):
        check(hg_batch_set_tuning(self.h, t), "hg_batch_set_tuning")

    def autotune(self, data: torch.Tensor, algo: int = SHA1, out=None, stream=None,
                 cache: str | None = None) -> hg_batch_tuning:
        """Tune this batch (hg_batch_autotune); with `cache` (a JSON Lines file) a tuning
        stored for the same GPU, parameters and batch shape is reused instead
        (hg_batch_autotune_cached). `self.tuned_from_cache` tells which happened."""
        ends, counts, dg = out if out is not None else self.outputs(algo)
        best = hg_batch_tuning()
        if cache is None:
            check(hg_batch_autotune(self.h, algo, _ptr(data), _ptr(ends), _ptr(counts), _ptr(dg),
                                    _stream(stream), best), "hg_batch_autotune")
            self.tuned_from_cache = False
        else:
            hit = C.c_int(0)
            check(hg_batch_autotune_cached(self.h, algo, _ptr(data), _ptr(ends), _ptr(counts),
                                           _ptr(dg), _stream(stream), cache, best, hit),
                  "hg_batch_autotune_cached")
            self.tuned_from_cache = bool(hit.value)
        return best

    def file_results(self, f: int, ends: torch.Tensor, counts: torch.Tensor, dg: torch.Tensor):
        """(ends, digests) of file f as numpy arrays (host copies)."""
        k = int(counts[f].item())
        a = int(self.slot_off[f])
        return (ends[a:a + k].cpu().numpy().astype(np.uint64), dg[a:a + k].cpu().numpy())


class Server:
    """Request server with continuous batching (one progress thread per server).

    Requests reference host memory (numpy arrays or pinned torch tensors) that
    must stay alive until the request completes; `submit` keeps a reference.
    """

    def __init__(self, ctx: Context, device_budget: int | None = None,
                 max_wave_bytes: int | None = None, max_wave_requests: int | None = None,
                 max_inflight_waves: int | None = None, p: hg_cdc_params | None = None,
                 wave_target_bytes: int | None = None):
        cfg = hg_server_config()
        hg_server_default_config(cfg)
        if device_budget is not None:
            cfg.device_budget = device_budget
        if max_wave_bytes is not None:
            cfg.max_wave_bytes = max_wave_bytes
        if max_wave_requests is not None:
            cfg.max_wave_requests = max_wave_requests
        if max_inflight_waves is not None:
            cfg.max_inflight_waves = max_inflight_waves
        if wave_target_bytes is not None:
            cfg.wave_target_bytes = wave_target_bytes
        if p is not None:
            cfg.cdc = p
        self.cfg = cfg
        self.ctx = ctx
        self.h = hg_server_create(ctx.h, cfg)
        _children.add(self)
        self._keep: dict[int, object] = {}

    @staticmethod
    def _host_ptr(data):
        if isinstance(data, torch.Tensor):
            return data.data_ptr() if data.numel() else None, data.numel()
        a = np.ascontiguousarray(data)
        return (a.ctypes.data if a.size else None), a.size

    def make_request(self, data, kind: int = HG_REQ_CDC, algo: int = MD5, block: int = 0,
                     want_root: bool = False) -> hg_request:
        ptr, n = self._host_ptr(data)
        r = hg_request()
        r.kind, r.algo, r.h_data, r.n, r.block, r.want_root, r.reserved = \
            kind, algo, ptr, n, block, int(want_root), 0
        return r

    def submit(self, data, kind: int = HG_REQ_CDC, algo: int = MD5, block: int = 0,
               want_root: bool = False) -> int:
        r = self.make_request(data, kind, algo, block, want_root)
        rc, t = hg_submit(self.h, r)
        check(rc, "hg_submit")
        self._keep[t] = data
        return t

    def cancel(self, ticket: int) -> int:
        return hg_cancel(self.h, ticket)

    def poll(self, ticket: int, timeout_us: int = -1, release: bool = True):
        """dict of the result, or None if not done within timeout_us."""
        res = hg_result()
        rc = hg_poll(self.h, ticket, res, timeout_us)
        if rc == _lib.HG_EAGAIN:
            return None
        check(rc, "hg_poll")
        dl = DIGEST_LEN[res.algo]
        k = res.count
        out = {"status": res.status, "count": k,
               "ends": np.ctypeslib.as_array(res.ends, (k,)).copy() if res.ends else None,
               "digests": (np.ctypeslib.as_array(res.digests, (k * dl,)).reshape(k, dl).copy()
                           if res.digests else np.zeros((0, dl), np.uint8)),
               "root": bytes(res.root[:dl]),
               "t_submit_ns": res.t_submit_ns, "t_admit_ns": res.t_admit_ns,
               "t_done_ns": res.t_done_ns}
        if release:
            hg_release(self.h, ticket)
            self._keep.pop(ticket, None)
        return out

    def wait_any(self, max_n: int = 1024, timeout_us: int = -1) -> list[int]:
        buf = np.zeros(max_n, np.uint64)
        rc, n = hg_server_wait_any(self.h, buf.ctypes.data, max_n, timeout_us)
        check(rc, "hg_server_wait_any")
        return buf[:n].tolist()

    def stats(self) -> dict:
        st = hg_server_stats()
        check(hg_server_get_stats(self.h, st))
        return {k: getattr(st, k) for k, _ in st._fields_}

    def replay(self, reqs: list, arrivals_ns: np.ndarray):
        """Open-loop replay of (request, arrival) pairs; returns (latencies_ns, span_ns)."""
        arr = (hg_request * len(reqs))(*reqs)
        t = np.ascontiguousarray(arrivals_ns, dtype=np.uint64)
        lat = np.zeros(len(reqs), np.uint64)
        rc, span = hg_server_replay(self.h, C.cast(arr, C.c_void_p).value, t.ctypes.data,
                                    len(reqs), lat.ctypes.data)
        check(rc, "hg_server_replay")
        return lat, span

    def close(self):
        if getattr(self, "h", None):
            hg_server_destroy(self.h)
            self.h = None
            self._keep.clear()

    def _release(self):
        self.close()

    def __del__(self):
        try:
            if _finalizer_may_call():
                self.close()
        except Exception:
            pass


class CdcStream:
    """Chunk a stream fed in device buffers of any size (hg_stream_*); results in stream offsets."""

    def __init__(self, ctx: Context, algo: int = MD5, p: hg_cdc_params | None = None,
                 max_feed: int = 64 << 20):
        self.ctx, self.algo = ctx, algo
        self.p = p or default_params()
        self.max_feed = max_feed
        self.h = hg_stream_open(ctx.h, algo, self.p, max_feed)
        _children.add(self)
        self.cap = (max_feed + self.p.max_chunk + self.p.window) // self.p.min_chunk + 2
        dev = ctx.device
        self._ends = torch.empty(self.cap, dtype=torch.int64, device=dev)
        self._cnt = torch.zeros(1, dtype=torch.int64, device=dev)
        self._dg = torch.empty((self.cap, DIGEST_LEN[algo]), dtype=torch.uint8, device=dev)

    def _take(self):
        k = int(self._cnt.item())
        return self._ends[:k].clone(), self._dg[:k].clone()

    def feed(self, data: torch.Tensor, stream=None):
        """Feed bytes; returns (ends, digests) of the chunks this feed decided."""
        check(hg_stream_feed(self.h, _ptr(data), data.numel(), _ptr(self._ends), self.cap,
                             _ptr(self._cnt), _ptr(self._dg), _stream(stream)), "hg_stream_feed")
        return self._take()

    def close(self, stream=None):
        check(hg_stream_close(self.h, _ptr(self._ends), self.cap, _ptr(self._cnt), _ptr(self._dg),
                              _stream(stream)), "hg_stream_close")
        out = self._take()
        hg_stream_destroy(self.h)
        self.h = None
        return out

    def _release(self):
        if self.h:
            hg_stream_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            if _finalizer_may_call():
                self._release()
        except Exception:
            pass


class BlockMap:
    """Device hash table of distinct digests (hg_blockmap_*): similarity detection."""

    def __init__(self, ctx: Context, algo: int = MD5, capacity: int = 1 << 20):
        self.ctx, self.algo = ctx, algo
        self.h = hg_blockmap_create(ctx.h, algo, capacity)
        _children.add(self)

    def insert(self, digests: torch.Tensor, count: torch.Tensor | None = None, stream=None):
        check(hg_blockmap_insert(self.h, _ptr(digests), digests.shape[0] if digests.dim() else 0,
                                 _ptr(count) if count is not None else None, _stream(stream)),
              "hg_blockmap_insert")

    def lookup(self, digests: torch.Tensor, ends: torch.Tensor | None = None,
               count: torch.Tensor | None = None, want_hits: bool = True, stream=None):
        """(hits uint8[n] or None, result int64[2] = {found, bytes found})."""
        n = digests.shape[0]
        hits = torch.empty(max(n, 1), dtype=torch.uint8, device=self.ctx.device) if want_hits else None
        res = torch.empty(2, dtype=torch.int64, device=self.ctx.device)
        check(hg_blockmap_lookup(self.h, _ptr(digests), _ptr(ends) if ends is not None else None, n,
                                 _ptr(count) if count is not None else None,
                                 _ptr(hits) if hits is not None else None, _ptr(res), _stream(stream)),
              "hg_blockmap_lookup")
        return (hits[:n] if hits is not None else None), res

    def count(self, stream=None) -> torch.Tensor:
        out = torch.empty(1, dtype=torch.int64, device=self.ctx.device)
        check(hg_blockmap_count(self.h, _ptr(out), _stream(stream)), "hg_blockmap_count")
        return out

    def clear(self, stream=None):
        check(hg_blockmap_clear(self.h, _stream(stream)), "hg_blockmap_clear")

    def close(self):
        if self.h:
            hg_blockmap_destroy(self.h)
            self.h = None

    def _release(self):
        self.close()

    def __del__(self):
        try:
            if _finalizer_may_call():
                self.close()
        except Exception:
            pass
