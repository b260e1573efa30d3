"""ctypes binding of libhashgpu.so (include/hashgpu.h).

The raw functions keep the C names and argument order (pointers are passed
as integers). Nothing here computes anything: every step runs in the CUDA
library, and importing this module fails loudly when the library is missing.
"""
from __future__ import annotations

import ctypes as C
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libhashgpu.so")

HG_OK, HG_EINVAL, HG_ENOMEM, HG_ECAPACITY, HG_ETIMEDOUT = 0, -1, -2, -3, -4
HG_ECUDA, HG_EAGAIN, HG_ECANCELED, HG_EUNSUPPORTED, HG_EBOUNDS = -5, -6, -7, -8, -9
HG_MD5, HG_SHA1 = 0, 1

# every exported symbol the header declares, with (restype, argtypes)
_vp, _u64, _u32, _i32, _sz = C.c_void_p, C.c_uint64, C.c_uint32, C.c_int, C.c_size_t


class hg_batch_tuning(C.Structure):
    _fields_ = [("window_ctas_per_sm", C.c_int32), ("hash_threads", C.c_int32),
                ("hash_ctas_per_sm", C.c_int32), ("reserved", C.c_int32),
                ("long_chunk_bytes", C.c_uint64)]


class hg_cdc_params(C.Structure):
    _fields_ = [("window", C.c_uint32), ("mask_bits", C.c_uint32), ("magic", C.c_uint32),
                ("window_hash", C.c_uint32), ("min_chunk", C.c_uint64), ("max_chunk", C.c_uint64)]


HG_REQ_CDC, HG_REQ_BLOCKS = 0, 1


class hg_request(C.Structure):
    _fields_ = [("kind", C.c_int32), ("algo", C.c_int32), ("h_data", C.c_void_p),
                ("n", C.c_uint64), ("block", C.c_uint64), ("want_root", C.c_int32),
                ("reserved", C.c_int32)]


class hg_result(C.Structure):
    _fields_ = [("status", C.c_int32), ("algo", C.c_int32), ("count", C.c_uint64),
                ("ends", C.POINTER(C.c_uint64)), ("digests", C.POINTER(C.c_uint8)),
                ("root", C.c_uint8 * 20), ("t_submit_ns", C.c_uint64),
                ("t_admit_ns", C.c_uint64), ("t_done_ns", C.c_uint64)]


class hg_server_config(C.Structure):
    _fields_ = [("device_budget", C.c_uint64), ("max_wave_bytes", C.c_uint64),
                ("max_wave_requests", C.c_uint32), ("max_inflight_waves", C.c_uint32),
                ("cdc", hg_cdc_params), ("wave_target_bytes", C.c_uint64)]


class hg_pinned_info(C.Structure):
    _fields_ = [(k, C.c_uint64) for k in ("budget_bytes", "held_bytes", "in_use_bytes",
                                          "host_allocs", "reuses", "buffers")]


class hg_server_stats(C.Structure):
    _fields_ = [(k, C.c_uint64) for k in ("submitted", "completed", "cancelled", "waves",
                                          "bytes_done", "arena_used", "arena_bytes", "queued")]


SIGNATURES = {
    "hg_cdc_default_params": (None, [C.POINTER(hg_cdc_params)]),
    "hg_strerror": (C.c_char_p, [_i32]),
    "hg_digest_len": (_i32, [_i32]),
    "hg_host_digest": (_i32, [_i32, _vp, _u64, _vp]),
    "hg_init": (_i32, [C.POINTER(_vp), _i32, _sz]),
    "hg_destroy": (_i32, [_vp]),
    "hg_reserve": (_i32, [_vp, _u64]),
    "hg_sync": (_i32, [_vp, _vp]),
    "hg_scratch_bytes": (_u64, [_vp]),
    "hg_hash_blocks": (_i32, [_vp, _i32, _vp, _u64, _u64, _vp, _vp, _vp]),
    "hg_hash_blocks_pmd": (_i32, [_vp, _i32, _vp, _u64, _u64, _u64, _vp, _vp, _vp]),
    "hg_blockmap_create": (_i32, [_vp, _i32, _u64, _vp]),
    "hg_blockmap_insert": (_i32, [_vp, _vp, _u64, _vp, _vp]),
    "hg_blockmap_lookup": (_i32, [_vp, _vp, _vp, _u64, _vp, _vp, _vp, _vp]),
    "hg_blockmap_count": (_i32, [_vp, _vp, _vp]),
    "hg_blockmap_clear": (_i32, [_vp, _vp]),
    "hg_blockmap_destroy": (_i32, [_vp]),
    "hg_blockmap_set_wait_limit": (_i32, [_vp, _u32]),
    "hg_blockmap_inject_claim": (_i32, [_vp, _vp, _vp]),
    "hg_window_bitmap": (_i32, [_vp, _vp, _u64, C.POINTER(hg_cdc_params), _vp, _vp]),
    "hg_cdc_candidates": (_i32, [_vp, _vp, _u64, C.POINTER(hg_cdc_params), _vp, _u64, _vp, _vp]),
    "hg_cdc_boundaries": (_i32, [_vp, _vp, _u64, C.POINTER(hg_cdc_params), _vp, _u64, _vp, _vp]),
    "hg_hash_chunks": (_i32, [_vp, _i32, _vp, _u64, _vp, _u64, _vp, _vp, _vp]),
    "hg_cdc_hash": (_i32, [_vp, _i32, _vp, _u64, C.POINTER(hg_cdc_params), _vp, _u64, _vp, _vp, _vp]),
    "hg_cdc_hash_plan": (_u32, [_u64, _vp, _u32]),
    "hg_cdc_hash_h2d": (_i32, [_vp, _i32, _vp, _vp, _u64, C.POINTER(hg_cdc_params), _vp, _u64, _vp, _vp, _vp]),
    "hg_stream_open": (_i32, [_vp, _i32, C.POINTER(hg_cdc_params), _u64, C.POINTER(_vp)]),
    "hg_stream_feed": (_i32, [_vp, _vp, _u64, _vp, _u64, _vp, _vp, _vp]),
    "hg_stream_close": (_i32, [_vp, _vp, _u64, _vp, _vp, _vp]),
    "hg_stream_destroy": (_i32, [_vp]),
    "hg_batch_create": (_i32, [_vp, _vp, _u32, C.POINTER(hg_cdc_params), C.POINTER(_vp)]),
    "hg_batch_destroy": (_i32, [_vp]),
    "hg_batch_slots": (_u64, [_vp, _vp]),
    "hg_batch_cdc_hash": (_i32, [_vp, _i32, _vp, _vp, _vp, _vp, _vp]),
    "hg_batch_cdc_hash_graph": (_i32, [_vp, _i32, _vp, _vp, _vp, _vp, _vp]),
    "hg_batch_sync": (_i32, [_vp, _vp]),
    "hg_batch_get_tuning": (_i32, [_vp, _vp]),
    "hg_batch_set_tuning": (_i32, [_vp, _vp]),
    "hg_batch_autotune": (_i32, [_vp, _i32, _vp, _vp, _vp, _vp, _vp, _vp]),
    "hg_batch_autotune_cached": (_i32, [_vp, _i32, _vp, _vp, _vp, _vp, _vp, C.c_char_p, _vp,
                                        C.POINTER(C.c_int)]),
    "hg_server_default_config": (None, [C.POINTER(hg_server_config)]),
    "hg_server_create": (_i32, [_vp, C.POINTER(hg_server_config), C.POINTER(_vp)]),
    "hg_server_destroy": (_i32, [_vp]),
    "hg_submit": (_i32, [_vp, C.POINTER(hg_request), C.POINTER(C.c_uint64)]),
    "hg_cancel": (_i32, [_vp, _u64]),
    "hg_poll": (_i32, [_vp, _u64, C.POINTER(hg_result), C.c_int64]),
    "hg_release": (_i32, [_vp, _u64]),
    "hg_server_wait_any": (_i32, [_vp, _vp, _u32, C.c_int64, C.POINTER(C.c_uint32)]),
    "hg_server_get_stats": (_i32, [_vp, C.POINTER(hg_server_stats)]),
    "hg_server_replay": (_i32, [_vp, _vp, _vp, _u32, _vp, C.POINTER(C.c_uint64)]),
    "hg_cdc_boundaries_static": (_i32, [_vp, _u64, C.POINTER(hg_cdc_params), _vp, _u64, _vp, _vp]),
    "hg_alloc_pinned": (_vp, [_vp, _sz]),
    "hg_free_pinned": (_i32, [_vp, _vp]),
    "hg_pinned_set_budget": (_i32, [_vp, _u64]),
    "hg_pinned_trim": (_i32, [_vp]),
    "hg_pinned_stats": (_i32, [_vp, C.POINTER(hg_pinned_info)]),
    "hg_pinned_class": (_u64, [_u64]),
}


def load(path: str = LIB_PATH) -> C.CDLL:
    if not os.path.exists(path):
        raise ImportError(
            f"{path} is missing: build the CUDA library first "
            "(python -c 'import __graft_entry__ as g; g.build()')")
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


lib = load()


class HashGPUError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        msg = lib.hg_strerror(status).decode()
        super().__init__(f"{what}: {msg} ({status})" if what else f"{msg} ({status})")


def check(status: int, what: str = "") -> int:
    if status != HG_OK:
        raise HashGPUError(status, what)
    return status


def default_params() -> hg_cdc_params:
    p = hg_cdc_params()
    lib.hg_cdc_default_params(C.byref(p))
    return p


# ---- raw C names, same argument order -------------------------------------------------------
def hg_init(device: int = 0, budget: int = 0) -> int:
    h = _vp()
    check(lib.hg_init(C.byref(h), device, budget), "hg_init")
    return h.value


def hg_destroy(ctx: int) -> int:
    return lib.hg_destroy(ctx)


def hg_reserve(ctx: int, max_bytes: int) -> int:
    return lib.hg_reserve(ctx, max_bytes)


def hg_sync(ctx: int, stream: int | None) -> int:
    return lib.hg_sync(ctx, stream)


def hg_scratch_bytes(ctx: int) -> int:
    return lib.hg_scratch_bytes(ctx)


def hg_digest_len(algo: int) -> int:
    return lib.hg_digest_len(algo)


def hg_hash_blocks(ctx, algo, d_in, n, block, d_digests, d_root, stream) -> int:
    return lib.hg_hash_blocks(ctx, algo, d_in, n, block, d_digests, d_root, stream)


def hg_hash_blocks_pmd(ctx, algo, d_in, n, block, segment, d_seg_digests, d_ids, stream) -> int:
    return lib.hg_hash_blocks_pmd(ctx, algo, d_in, n, block, segment, d_seg_digests, d_ids, stream)


def hg_window_bitmap(ctx, d_in, n, params, d_bitmap, stream) -> int:
    return lib.hg_window_bitmap(ctx, d_in, n, C.byref(params), d_bitmap, stream)


def hg_cdc_candidates(ctx, d_in, n, params, d_cands, cap, d_count, stream) -> int:
    return lib.hg_cdc_candidates(ctx, d_in, n, C.byref(params), d_cands, cap, d_count, stream)


def hg_cdc_boundaries(ctx, d_in, n, params, d_ends, cap, d_count, stream) -> int:
    return lib.hg_cdc_boundaries(ctx, d_in, n, C.byref(params), d_ends, cap, d_count, stream)


def hg_hash_chunks(ctx, algo, d_in, n, d_ends, nchunk, d_count, d_digests, stream) -> int:
    return lib.hg_hash_chunks(ctx, algo, d_in, n, d_ends, nchunk, d_count, d_digests, stream)


def hg_alloc_pinned(ctx, nbytes) -> int | None:
    return lib.hg_alloc_pinned(ctx, nbytes)


def hg_free_pinned(ctx, p) -> int:
    return lib.hg_free_pinned(ctx, p)


def hg_pinned_set_budget(ctx, nbytes) -> int:
    return lib.hg_pinned_set_budget(ctx, nbytes)


def hg_pinned_trim(ctx) -> int:
    return lib.hg_pinned_trim(ctx)


def hg_pinned_stats(ctx, out) -> int:
    return lib.hg_pinned_stats(ctx, C.byref(out))


def hg_pinned_class(nbytes) -> int:
    return lib.hg_pinned_class(nbytes)


def hg_cdc_boundaries_static(d_in, n, params, d_ends, cap, d_count, stream) -> int:
    return lib.hg_cdc_boundaries_static(d_in, n, C.byref(params), d_ends, cap, d_count, stream)


def hg_batch_create(ctx, h_file_off_ptr, nfile, params) -> int:
    h = _vp()
    check(lib.hg_batch_create(ctx, h_file_off_ptr, nfile, C.byref(params), C.byref(h)),
          "hg_batch_create")
    return h.value


def hg_batch_destroy(batch) -> int:
    return lib.hg_batch_destroy(batch)


def hg_batch_slots(batch, h_slot_off_ptr) -> int:
    return lib.hg_batch_slots(batch, h_slot_off_ptr)


def hg_batch_cdc_hash(batch, algo, d_data, d_ends, d_counts, d_digests, stream) -> int:
    return lib.hg_batch_cdc_hash(batch, algo, d_data, d_ends, d_counts, d_digests, stream)


def hg_batch_cdc_hash_graph(batch, algo, d_data, d_ends, d_counts, d_digests, stream) -> int:
    return lib.hg_batch_cdc_hash_graph(batch, algo, d_data, d_ends, d_counts, d_digests, stream)


def hg_batch_sync(batch, stream) -> int:
    return lib.hg_batch_sync(batch, stream)


def hg_batch_get_tuning(batch, tuning) -> int:
    return lib.hg_batch_get_tuning(batch, C.byref(tuning))


def hg_batch_set_tuning(batch, tuning) -> int:
    return lib.hg_batch_set_tuning(batch, C.byref(tuning))


def hg_batch_autotune(batch, algo, d_data, d_ends, d_counts, d_digests, stream, best) -> int:
    return lib.hg_batch_autotune(batch, algo, d_data, d_ends, d_counts, d_digests, stream,
                                 C.byref(best) if best is not None else None)


def hg_batch_autotune_cached(batch, algo, d_data, d_ends, d_counts, d_digests, stream, cache_path,
                             best, from_cache) -> int:
    return lib.hg_batch_autotune_cached(batch, algo, d_data, d_ends, d_counts, d_digests, stream,
                                        cache_path.encode() if isinstance(cache_path, str) else cache_path,
                                        C.byref(best) if best is not None else None,
                                        C.byref(from_cache) if from_cache is not None else None)


def hg_server_default_config(cfg) -> None:
    lib.hg_server_default_config(C.byref(cfg))


def hg_server_create(ctx, cfg) -> int:
    h = _vp()
    check(lib.hg_server_create(ctx, C.byref(cfg), C.byref(h)), "hg_server_create")
    return h.value


def hg_server_destroy(srv) -> int:
    return lib.hg_server_destroy(srv)


def hg_submit(srv, req) -> tuple[int, int]:
    t = C.c_uint64()
    rc = lib.hg_submit(srv, C.byref(req), C.byref(t))
    return rc, t.value


def hg_cancel(srv, ticket) -> int:
    return lib.hg_cancel(srv, ticket)


def hg_poll(srv, ticket, res, timeout_us) -> int:
    return lib.hg_poll(srv, ticket, C.byref(res), timeout_us)


def hg_release(srv, ticket) -> int:
    return lib.hg_release(srv, ticket)


def hg_server_wait_any(srv, tickets_ptr, max_n, timeout_us) -> tuple[int, int]:
    n = C.c_uint32()
    rc = lib.hg_server_wait_any(srv, tickets_ptr, max_n, timeout_us, C.byref(n))
    return rc, n.value


def hg_server_get_stats(srv, st) -> int:
    return lib.hg_server_get_stats(srv, C.byref(st))


def hg_server_replay(srv, reqs_ptr, arrivals_ptr, nreq, lat_ptr) -> tuple[int, int]:
    span = C.c_uint64()
    rc = lib.hg_server_replay(srv, reqs_ptr, arrivals_ptr, nreq, lat_ptr, C.byref(span))
    return rc, span.value


def hg_cdc_hash(ctx, algo, d_in, n, params, d_ends, cap, d_count, d_digests, stream) -> int:
    return lib.hg_cdc_hash(ctx, algo, d_in, n, C.byref(params), d_ends, cap, d_count, d_digests,
                           stream)


def hg_cdc_hash_plan(n, bounds_ptr, max_n) -> int:
    return lib.hg_cdc_hash_plan(n, bounds_ptr, max_n)


def hg_cdc_hash_h2d(ctx, algo, h_in, d_in, n, params, d_ends, cap, d_count, d_digests, stream) -> int:
    return lib.hg_cdc_hash_h2d(ctx, algo, h_in, d_in, n, C.byref(params), d_ends, cap, d_count,
                               d_digests, stream)


def hg_blockmap_create(ctx, algo, capacity) -> int:
    h = _vp()
    check(lib.hg_blockmap_create(ctx, algo, capacity, C.byref(h)), "hg_blockmap_create")
    return h.value


def hg_blockmap_insert(m, d_digests, count, d_count, stream) -> int:
    return lib.hg_blockmap_insert(m, d_digests, count, d_count, stream)


def hg_blockmap_lookup(m, d_digests, d_ends, count, d_count, d_hits, d_result, stream) -> int:
    return lib.hg_blockmap_lookup(m, d_digests, d_ends, count, d_count, d_hits, d_result, stream)


def hg_blockmap_count(m, d_out, stream) -> int:
    return lib.hg_blockmap_count(m, d_out, stream)


def hg_blockmap_clear(m, stream) -> int:
    return lib.hg_blockmap_clear(m, stream)


def hg_blockmap_destroy(m) -> int:
    return lib.hg_blockmap_destroy(m)


def hg_stream_open(ctx, algo, params, max_feed) -> int:
    h = _vp()
    check(lib.hg_stream_open(ctx, algo, C.byref(params), max_feed, C.byref(h)), "hg_stream_open")
    return h.value


def hg_stream_feed(st, d_data, n, d_ends, cap, d_count, d_digests, stream) -> int:
    return lib.hg_stream_feed(st, d_data, n, d_ends, cap, d_count, d_digests, stream)


def hg_stream_close(st, d_ends, cap, d_count, d_digests, stream) -> int:
    return lib.hg_stream_close(st, d_ends, cap, d_count, d_digests, stream)


def hg_stream_destroy(st) -> int:
    return lib.hg_stream_destroy(st)
