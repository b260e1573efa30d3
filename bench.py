#!/usr/bin/env python3
"""Benchmark of the HashGPU hot path on B300.

Workload (one step): content-defined chunking of two versions of a file --
a 64 MiB seeded uniform base and a second version made by seeded edits
touching 1 % of its bytes (insert/delete/overwrite runs of 1..512 bytes) --
with a 20-byte MD5 window at every offset, boundaries where the low 13 bits
of the window hash equal 0x0F0F, chunks between 2 KiB and 64 KiB, then the
MD5 digest of every chunk (Sec. 2.1, Sec. 3.2.2, Fig. 3). The two versions
run on two streams, each with its own library context.

value: hashed GB/s (input bytes of both versions per step / device time per
step), inputs resident in HBM, L2 flushed between steps.
e2e:   the same through hg_cdc_hash_h2d, with the versions in pinned host
memory: the call copies each version to the device in pieces overlapped with
the chunking; the D2H of counts, boundaries + digests is inside the timed
region too.
The line also carries the roofline of the dominant kernel (the window-hash
kernel), the CPU oracle baseline, the fixed-block direct-hashing throughputs
(1 GiB, MD5/SHA-1, 4 KiB / 64 KiB / 1 MiB blocks, two-level identifiers) and the clocks
seen while timing.

--impl reference times the CPU oracle on the host cores on bounded samples of
the same workload (there is no reference implementation to install).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "hashed GB/s (CDC: 20-byte MD5 window + min/max boundaries + per-chunk MD5)"
# hg_cdc_hash is the public call timed; hg_cdc_boundaries + hg_hash_chunks (the
# same kernels without segment pipelining) is reported beside it.
UNIT = "GB/s"
WORKLOAD = "cdc_64MiB_base_plus_1pct_edited_version"
# Algorithmic cost of one window hash in two-input 32-bit integer operations (the
# roofline unit): one MD5 compression per window; 44 steps whose message word is a
# constant fold it with the step constant (4 operations), the steps on data words take
# 5, the hash stops after the step that last writes word A, and the window assembly
# (funnel shifts) and the candidate test add about 8: about 270 per window (one per
# input byte). Against the integer issue rate (4 schedulers x 32 lanes per SM per
# clock); a kernel could pass 1.0 only by fusing two-input operations into three-input
# instructions beyond what the count assumes.
OPS_PER_WINDOW = 270
ISSUE_LANES_PER_SM_CLK = 128
# Per-chunk MD5 adds about 5.1 operations per byte (64 steps x 5 + 4 final adds per
# 64 bytes), so the whole chunking step costs about 275 operations per input byte.
OPS_PER_BYTE_CDC_STEP = OPS_PER_WINDOW + 5.1
OPS_PER_BYTE_MD5, OPS_PER_BYTE_SHA1 = 5.1, 9.6
# Instructions per 64-byte block that only the integer ALU pipe runs, whatever the adds'
# placement: MD5 one logic op and one rotate-add per step (64 steps); SHA-1 80 logic ops,
# 80 rotate-adds, 80 rotates of b, 64 x 3 schedule ops (two 3-input XORs, a rotate) and
# 16 byte swaps. Against the ALU pipe's 64 lanes per SM per clock they bound the block
# kernels whatever is moved to the FMA pipe (a secondary roofline beside the issue rate's).
ALU_ONLY_PER_BLOCK_MD5, ALU_ONLY_PER_BLOCK_SHA1 = 128, 448
# The integer ALU pipe alone (logic, funnel shift, rotate-add issue only there) takes
# one warp instruction every other clock per scheduler: 64 lanes per SM per clock.
ALU_LANES_PER_SM_CLK = 64
# the window kernel's own sources: its counters in profiles/ hold only while these are unchanged
WINDOW_KERNEL_SRC = [os.path.join(ROOT, "paper_1202_3669_b300", "csrc", f)
                     for f in ("hg_window.cu", "hg_window.cuh", "hg_device.cuh")]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-extras", action="store_true", help="skip the direct/batch/serve/CPU legs")
    ap.add_argument("--leg", default=None,
                    choices=["direct", "batch", "serve", "rabin", "blockmap", "configs", "alu", "blocks"],
                    help="run only this extra leg (for profiling) and print its result")
    ap.add_argument("--batch-files", type=int, default=4096,
                    help="batch leg: use only the first N files of the 4096-file workload")
    return ap.parse_args()


def workload():
    from gen import inputs as G
    base = G.uniform_bytes(64 << 20, seed=2)
    v2, _ = G.edited_version(base, seed=3)
    return [base, v2]


# ------------------------------------------------------------------ clocks --------------------
class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons while timing."""
    Q = ("index,pci.bus_id,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, bus_id: str | None):
        self.bus = (bus_id or "").lower()
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                       "-lms", "100"], stdout=self.f, stderr=subprocess.DEVNULL)
        except FileNotFoundError:
            self.p = None
        time.sleep(0.25)

    def stop(self) -> dict:
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.15)
        self.p.terminate()
        self.p.wait()
        self.f.seek(0)
        rows = [r.split(", ") for r in self.f.read().strip().splitlines() if r.count(",") >= 9]
        os.unlink(self.f.name)
        if self.bus:
            mine = [r for r in rows if r[1].lower().endswith(self.bus[-12:])]
            rows = mine or rows
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        idx0 = rows[0][0]
        rows = [r for r in rows if r[0] == idx0]
        sm = [float(r[2]) for r in rows]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[6 + k].strip() == "Active"})
        loaded = [s for s in sm if s > 0.5 * max(sm)] or sm
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": float(rows[0][3]),
                "reasons": reasons, "samples": len(rows),
                "power_w_max": max(float(r[4]) for r in rows if r[4].replace('.', '', 1).isdigit()) if rows else None}


# ------------------------------------------------------------------ helpers -------------------
def max_over_ranks(times_ms, world, device=None):
    """Per-step times of this rank -> the maximum over all ranks (replicas run the same
    workload, so the slowest rank sets the job's time). No-op on one rank."""
    if world <= 1:
        return [float(t) for t in times_ms]
    import torch
    import torch.distributed as dist
    t = torch.tensor(times_ms, dtype=torch.float64,
                     device=device if dist.get_backend() == "nccl" else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t.cpu()]


def replica_throughput(bytes_per_rank, world, step_ms):
    """Whole-job GB/s: every rank hashes bytes_per_rank per step (weak scaling)."""
    return world * bytes_per_rank / (step_ms / 1e3) / 1e9

def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6400.0, "sm_max_mhz": 2032.0}, "fallback"


def source_hash(srcs) -> str:
    """First 16 hex digits of the SHA-256 of the source files, concatenated in order."""
    h = hashlib.sha256()
    for src in srcs:
        with open(src, "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def kernel_traffic(kernel: str, srcs):
    """DRAM bytes per launch from a committed ncu summary, if it was taken on these sources."""
    p = os.path.join(ROOT, "profiles", f"{kernel}.traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        rec = json.load(f)
    h = source_hash(srcs)
    if rec.get("source_sha256_16") != h:
        return None
    return rec


def cpu_info() -> dict:
    """Host CPU model and the threads the oracle baselines use."""
    model = None
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    return {"model": model, "nproc": os.cpu_count() or 1}


def _threads_map(fn, items, nthreads):
    import concurrent.futures as cf
    with cf.ThreadPoolExecutor(nthreads) as ex:
        return list(ex.map(fn, items))


def _oracle_blocks_n(oracle, L, algo, data, block, nthreads):
    """Fixed-block digests + root with the oracle, blocks split over threads (each
    thread one contiguous range of whole blocks); the root hashes the digest list."""
    nblk = (data.size + block - 1) // block
    cuts = np.linspace(0, nblk, min(nblk, nthreads) + 1).astype(np.int64)
    parts = _threads_map(lambda k: oracle.hash_blocks(algo, data[cuts[k] * block:cuts[k + 1] * block],
                                                      block, root=False, L=L)[0],
                         range(cuts.size - 1), nthreads)
    dg = np.concatenate(parts)
    return dg, oracle.digest(algo, dg.tobytes(), L=L)


def _time_rate(fn, nbytes, reps=3):
    """Wall-clock median of reps runs."""
    ts = []
    for _ in range(reps):
        t0 = time.perf_counter()
        fn()
        ts.append(time.perf_counter() - t0)
    dt = statistics.median(ts)
    return {"GBps": nbytes / dt / 1e9, "seconds": dt, "bytes": int(nbytes), "runs": reps}


def cpu_baseline(versions, budget_s: float = 12.0):
    """The oracle as it stands, on the host cores, on bounded samples of each
    configuration: the main chunking workload on all threads (the headline baseline) and
    on one thread, plus the 8 MiB fixed-block configuration, fixed blocks and chunking of
    the 1 GiB inputs (samples), each on one thread and fanned out over all threads
    (independent block ranges; window ranges inside the oracle)."""
    import oracle
    from gen import inputs as G
    nthreads = os.cpu_count() or 1
    L = oracle.lib()
    # calibrate on growing prefixes (thread start-up dominates tiny probes), then size the
    # sample to about budget_s seconds; the whole workload is the upper bound
    probe_n, rate = 1 << 20, 0.0
    while True:
        probe = versions[0][:probe_n]
        t0 = time.perf_counter()
        e = oracle.cdc(probe, nthreads=nthreads, L=L)
        oracle.hash_chunks(oracle.MD5, probe, e, L=L)
        dt = time.perf_counter() - t0
        rate = probe.size / max(1e-6, dt)
        if dt >= 0.5 or probe_n >= versions[0].size:
            break
        probe_n = min(versions[0].size, probe_n * 4)
    nbytes = int(min(versions[0].size, max(1 << 20, rate * budget_s / 2)))
    total, t0 = 0, time.perf_counter()
    for v in versions:
        s = v[:nbytes]
        e = oracle.cdc(s, nthreads=nthreads, L=L)
        oracle.hash_chunks(oracle.MD5, s, e, L=L)
        total += s.size
    dt = time.perf_counter() - t0
    # the same oracle on one thread, on a smaller sample (about a quarter of the budget)
    n1 = int(min(versions[0].size, max(1 << 18, rate / nthreads * budget_s / 8)))
    t1 = time.perf_counter()
    for v in versions:
        s1 = v[:n1]
        e = oracle.cdc(s1, nthreads=1, L=L)
        oracle.hash_chunks(oracle.MD5, s1, e, L=L)
    dt1 = time.perf_counter() - t1
    single = {"value": 2 * n1 / dt1 / 1e9, "unit": UNIT, "cores": 1, "seconds": dt1,
              "sample": f"first {n1} bytes of each version"}

    # the other configurations, on samples sized from the rates above
    configs = {}
    small = G.uniform_bytes(8 << 20, seed=1)
    for algo, name in ((oracle.MD5, "md5"), (oracle.SHA1, "sha1")):
        configs[f"blocks_8MiB_4KiB_{name}_with_root"] = {
            "1_thread": _time_rate(lambda: oracle.hash_blocks(algo, small, 4096, L=L), small.size),
            f"{nthreads}_threads": _time_rate(lambda: _oracle_blocks_n(oracle, L, algo, small, 4096, nthreads),
                                              small.size)}
    u = G.uniform_bytes(64 << 20, seed=4)          # a 64 MiB sample drawn as the 1 GiB input is
    for algo, name in ((oracle.MD5, "md5"), (oracle.SHA1, "sha1")):
        for block, label in ((4096, "4KiB"), (1 << 20, "1MiB")):
            configs[f"blocks_1GiB_uniform_{label}_{name}"] = {
                "1_thread": _time_rate(lambda: oracle.hash_blocks(algo, u[:16 << 20], block, L=L), 16 << 20),
                f"{nthreads}_threads": _time_rate(
                    lambda: _oracle_blocks_n(oracle, L, algo, u, block, nthreads), u.size)}
    ncdc = int(min(16 << 20, max(1 << 20, rate * budget_s / 8)))
    n1c = int(max(1 << 17, n1 // 4))
    t = G.text_like_bytes(ncdc, seed=5)
    for dist, data in (("uniform", u[:ncdc]), ("text", t)):
        def cdc_all(d=data):
            e = oracle.cdc(d, nthreads=nthreads, L=L)
            oracle.hash_chunks(oracle.MD5, d, e, L=L)

        def cdc_one(d=data[:n1c]):
            e = oracle.cdc(d, nthreads=1, L=L)
            oracle.hash_chunks(oracle.MD5, d, e, L=L)
        configs[f"cdc_1GiB_{dist}_md5"] = {"1_thread": _time_rate(cdc_one, n1c),
                                         f"{nthreads}_threads": _time_rate(cdc_all, data.size)}
    return {"value": total / dt / 1e9, "unit": UNIT, "cores": nthreads, "kind": "oracle",
            "single_thread": single, "cpu": cpu_info(), "configs": configs,
            "sample": f"first {nbytes} bytes of each of the two versions ({total} bytes), "
                      f"window candidates on {nthreads} threads + selection + per-chunk MD5",
            "seconds": dt}


# ------------------------------------------------------------------ reference arm -------------
def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    versions = workload()
    import oracle
    nthreads = os.cpu_count() or 1
    per_step = (2 << 20)          # bytes of each version per step: a bounded sample
    times = []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        for v in versions:
            s = v[:per_step]
            e = oracle.cdc(s, nthreads=nthreads)
            oracle.hash_chunks(oracle.MD5, s, e)
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            times.append(dt)
        if sum(times) > 150:      # keep the run within a few minutes
            break
    t = sum(times) / len(times)
    val = 2 * per_step / t / 1e9
    out = {"metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus, "steps": len(times),
           "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
           "impl": "reference",
           "config": {"workload": WORKLOAD, "sample_bytes_per_version": per_step},
           "cpu_baseline": {"value": val, "unit": UNIT, "cores": nthreads, "kind": "oracle",
                            "sample": f"first {per_step} bytes of each version per step"},
           "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


# ------------------------------------------------------------------ our arm -------------------
def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    import torch
    import torch.distributed as dist

    import paper_1202_3669_b300 as hgb

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)

    def barrier():
        if world > 1:
            dist.barrier()

    if args.leg:
        ctx = hgb.Context(local)
        flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
        if args.leg == "direct":
            res = direct_leg(hgb, ctx, dev, flush)
        elif args.leg == "batch":
            res = batch_leg(hgb, ctx, dev, flush, nfiles=args.batch_files)
        elif args.leg == "rabin":
            res = rabin_leg(hgb, dev, flush)
        elif args.leg == "blockmap":
            res = blockmap_leg(hgb, ctx, dev, flush)
        elif args.leg == "configs":
            res = configs_leg(hgb, ctx, dev, flush)
        elif args.leg == "alu":
            res = alu_leg(dev)
        elif args.leg == "blocks":
            res = blocks_leg(hgb, ctx, dev)
        else:
            bl = batch_leg(hgb, ctx, dev, flush)
            res = serve_leg(hgb, ctx, bl["batched_graph_GBps"], bl["per_file_GBps"])
        print(json.dumps({"leg": args.leg, "result": res}), flush=True)
        return
    versions = workload()
    nbytes = sum(v.size for v in versions)
    p = hgb.default_params()
    ctxs = [hgb.Context(local) for _ in versions]
    streams = [torch.cuda.Stream(dev) for _ in versions]
    d_in = [torch.from_numpy(v).to(dev) for v in versions]
    cap = [v.size // p.min_chunk + 2 for v in versions]
    ends = [torch.empty(c, dtype=torch.int64, device=dev) for c in cap]
    cnts = [torch.zeros(1, dtype=torch.int64, device=dev) for _ in versions]
    dgs = [torch.empty((c, 16), dtype=torch.uint8, device=dev) for c in cap]
    for c, v in zip(ctxs, versions):
        c.reserve(v.size)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)    # > 126 MB L2
    main_s = torch.cuda.current_stream(dev)

    def step(src):
        ev0 = torch.cuda.Event()
        ev0.record(main_s)
        for i in range(len(versions)):
            s = streams[i]
            s.wait_event(ev0)
            ctxs[i].cdc_hash(src[i], hgb.MD5, p, out=(ends[i], cnts[i], dgs[i]), stream=s)
        for s in streams:
            main_s.wait_stream(s)

    # hg_cdc_hash: five kernels per segment (window, scan, compact, select, chunk digests)
    launches_per_step = sum(5 * (len(hgb.cdc_hash_plan(v.size)) - 1) for v in versions)
    for _ in range(args.warmup):
        step(d_in)
    torch.cuda.synchronize()
    for c in ctxs:
        c.sync()

    bus = None
    try:
        bus = torch.cuda.get_device_properties(dev).pci_bus_id
    except Exception:
        pass
    clk = ClockSampler(bus)
    clk.start()
    barrier()
    torch.cuda.synchronize()
    ms = []
    for _ in range(args.steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(main_s)
        step(d_in)
        b.record(main_s)
        ms.append((a, b))
    torch.cuda.synchronize()
    barrier()
    step_ms = [a.elapsed_time(b) for a, b in ms]
    t_dev = sum(step_ms) / len(step_ms)

    # the same work through the two unpipelined calls, for comparison
    def step_two_calls(src):
        ev0 = torch.cuda.Event()
        ev0.record(main_s)
        for i in range(len(versions)):
            s = streams[i]
            s.wait_event(ev0)
            ctxs[i].cdc_boundaries(src[i], p, cap=cap[i], out=ends[i], count=cnts[i], stream=s)
            ctxs[i].hash_chunks(src[i], ends[i], hgb.MD5, count=cnts[i], out=dgs[i], stream=s)
        for s in streams:
            main_s.wait_stream(s)

    step_two_calls(d_in)
    tw = []
    for _ in range(20):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(main_s)
        step_two_calls(d_in)
        b.record(main_s)
        tw.append((a, b))
    torch.cuda.synchronize()
    t_two = sum(a.elapsed_time(b) for a, b in tw) / len(tw)

    # e2e: pinned host inputs -> device -> boundaries + digests -> pinned host; the pinned
    # buffers come from the library's pool (hg_alloc_pinned)
    def pinned(ctx, nbytes, dtype, shape):
        b = ctx.alloc_pinned(nbytes)
        return b, b.tensor.view(dtype)[:int(np.prod(shape))].view(shape)
    pool = []
    h_in, h_ends, h_cnt, h_dg = [], [], [], []
    for i, v in enumerate(versions):
        b, t = pinned(ctxs[i], v.size, torch.uint8, (v.size,))
        t.numpy()[:] = v
        pool.append(b)
        h_in.append(t)
        for lst, nb, dt, shp in ((h_ends, cap[i] * 8, torch.int64, (cap[i],)), (h_cnt, 8, torch.int64, (1,)),
                                 (h_dg, cap[i] * 16, torch.uint8, (cap[i], 16))):
            b, t = pinned(ctxs[i], nb, dt, shp)
            pool.append(b)
            lst.append(t)
    d_in2 = [torch.empty_like(x) for x in d_in]
    h2d = sum(v.size for v in versions)
    d2h = sum(e.numel() * 8 + 8 + d.numel() for e, d in zip(h_ends, h_dg))
    # plain pinned host -> device copy rate, for context of the e2e figure
    a, bq = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    d_in2[0].copy_(h_in[0], non_blocking=True)
    a.record(main_s)
    for _ in range(5):
        d_in2[0].copy_(h_in[0], non_blocking=True)
    bq.record(main_s)
    torch.cuda.synchronize()
    h2d_gbps = 5 * versions[0].size / (a.elapsed_time(bq) / 1e3) / 1e9

    def e2e_step():
        ev0 = torch.cuda.Event()
        ev0.record(main_s)
        for i in range(len(versions)):
            s = streams[i]
            s.wait_event(ev0)
            ctxs[i].cdc_hash_from_host(h_in[i], d_in2[i], hgb.MD5, p, out=(ends[i], cnts[i], dgs[i]),
                                       stream=s)
            with torch.cuda.stream(s):
                h_cnt[i].copy_(cnts[i], non_blocking=True)
                h_ends[i].copy_(ends[i], non_blocking=True)
                h_dg[i].copy_(dgs[i], non_blocking=True)
        for s in streams:
            main_s.wait_stream(s)

    for _ in range(3):
        e2e_step()
    torch.cuda.synchronize()
    e2e_steps = max(10, args.steps // 4)
    barrier()
    ev = []
    for _ in range(e2e_steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(main_s)
        e2e_step()
        b.record(main_s)
        ev.append((a, b))
    torch.cuda.synchronize()
    t_e2e = sum(a.elapsed_time(b) for a, b in ev) / len(ev)
    stages = stage_breakdown(versions, streams, main_s, flush, h_in, d_in2, (ends, cnts, dgs),
                             (h_ends, h_cnt, h_dg), e2e_step, t_dev, t_e2e)
    pool_stats = [c.pinned_stats() for c in ctxs]
    clocks = clk.stop()
    for c in ctxs:
        c.sync()

    # the e2e result must be the device result
    for i in range(len(versions)):
        k = int(h_cnt[i].item())
        assert k == int(cnts[i].item())
        assert torch.equal(h_ends[i][:k], ends[i][:k].cpu())

    # dominant kernel alone: the window-hash kernel on the base version, same stream discipline
    wl = []
    bm = torch.empty((versions[0].size + 31) // 32, dtype=torch.int32, device=dev)
    for i in range(args.warmup + 20):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(main_s)
        ctxs[0].window_bitmap(d_in[0], p, out=bm, stream=main_s)
        b.record(main_s)
        if i >= args.warmup:
            wl.append((a, b))
    torch.cuda.synchronize()
    t_win = sum(a.elapsed_time(b) for a, b in wl) / len(wl) / 1e3
    windows = versions[0].size - (p.window - 1)
    peaks, peak_kind = measured_peaks()
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    sm_max = float(peaks.get("sm_max_mhz", 2032.0))
    issue_peak = sm_count * ISSUE_LANES_PER_SM_CLK * sm_max * 1e6 / 1e12
    alu_peak = sm_count * ALU_LANES_PER_SM_CLK * sm_max * 1e6 / 1e12
    achieved = windows * OPS_PER_WINDOW / t_win / 1e12
    tr = kernel_traffic("k_window_bitmap", WINDOW_KERNEL_SRC)
    counters = (tr or {}).get("per_window", {})
    roofline = {"bound": "alu", "kernel": "k_window_bitmap<20>", "achieved": achieved,
                "peak": issue_peak, "unit": "Tops/s (two-input int32 operations)",
                "frac": achieved / issue_peak,
                "peak_kind": (f"int32 issue rate: {sm_count} SMs x {ISSUE_LANES_PER_SM_CLK} lanes/clk x "
                              f"{sm_max:.0f} MHz (max SM clock, {peak_kind} clock); algorithmic count "
                              f"{OPS_PER_WINDOW} two-input operations per window"),
                "ops_per_window": OPS_PER_WINDOW, "windows_per_launch": windows,
                "launch_ms": t_win * 1e3, "window_GBps": versions[0].size / t_win / 1e9,
                "traffic": (tr["dram_bytes_per_launch"] * versions[0].size / tr["input_bytes"]) if tr else None}
    if counters.get("alu_pipe_inst"):
        # secondary: the instructions ncu counted on each pipe, against each pipe's peak
        roofline["alu_pipe_frac"] = windows * counters["alu_pipe_inst"] / t_win / 1e12 / alu_peak
        roofline["issue_frac"] = windows * counters["all_inst"] / t_win / 1e12 / issue_peak
        roofline["counted_per_window"] = counters
    if clocks.get("sm_mhz"):
        roofline["frac_at_observed_clock"] = achieved / (issue_peak * clocks["sm_mhz"] / sm_max)
    # the integer pipes' rates measured by the probe (per operation class), beside the peak used
    roofline["measured_int_pipe"] = alu_leg(dev)
    # the whole chunking step (windows + selection + per-chunk MD5) against its bound
    step_bound = issue_peak * 1e12 / OPS_PER_BYTE_CDC_STEP / 1e9
    cdc_step_roofline = {"bound": "alu", "achieved": nbytes / (t_dev / 1e3) / 1e9,
                         "peak": step_bound, "unit": "GB/s",
                         "frac": nbytes / (t_dev / 1e3) / 1e9 / step_bound,
                         "peak_kind": f"int32 issue rate / {OPS_PER_BYTE_CDC_STEP:.1f} operations per byte"}

    # shared-chunk fraction between the versions (from this run's device results)
    k0, k1 = int(cnts[0].item()), int(cnts[1].item())
    s0 = {bytes(r) for r in dgs[0][:k0].cpu().numpy()}
    e1 = ends[1][:k1].cpu().numpy()
    sz1 = np.diff(np.concatenate([[0], e1]))
    shared = sum(int(s) for s, r in zip(sz1, dgs[1][:k1].cpu().numpy()) if bytes(r) in s0) / versions[1].size

    extras = {}
    if not args.no_extras and rank == 0:
        extras["direct"] = direct_leg(hgb, ctxs[0], dev, flush)
        extras["rabin"] = rabin_leg(hgb, dev, flush)
        extras["blockmap"] = blockmap_leg(hgb, ctxs[0], dev, flush)
        extras["configs"] = configs_leg(hgb, ctxs[0], dev, flush)
        extras["batch"] = batch_leg(hgb, ctxs[0], dev, flush)
        extras["serve"] = serve_leg(hgb, ctxs[0], extras["batch"]["batched_graph_GBps"],
                                    extras["batch"]["per_file_GBps"])
        extras["cpu_baseline"] = cpu_baseline(versions)

    # max over ranks
    t_dev_all, t_e2e_all = max_over_ranks([t_dev, t_e2e], world, dev)
    if rank == 0:
        value = replica_throughput(nbytes, world, t_dev_all)
        out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
               "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_dev_all,
               "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
               "data": "synthetic",
               "config": {"workload": WORKLOAD, "bytes_per_step_per_gpu": nbytes,
                          "version_bytes": [int(v.size) for v in versions],
                          "window": p.window, "mask_bits": p.mask_bits, "magic": p.magic,
                          "min_chunk": p.min_chunk, "max_chunk": p.max_chunk, "digest": "md5",
                          "chunks": [k0, k1], "shared_fraction": shared,
                          "l2": "flushed between steps (256 MiB memset)",
                          "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
               "e2e": {"value": replica_throughput(nbytes, world, t_e2e_all), "unit": UNIT,
                       "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                       "pinned_h2d_copy_GBps": h2d_gbps,
                       "link_frac": replica_throughput(nbytes, world, t_e2e_all) / world / h2d_gbps,
                       "bound": "host link: the pinned host-to-device copy rate measured in this run",
                       "pinned_from": "hg_alloc_pinned pool",
                       "pinned_pool": {"host_allocs": sum(x["host_allocs"] for x in pool_stats),
                                       "held_bytes": sum(x["held_bytes"] for x in pool_stats)},
                       "stages": stages},
               "gpu_launches": launches_per_step * args.steps,
               "roofline": roofline,
               "cdc_step_roofline": cdc_step_roofline,
               "cpu_baseline": extras.get("cpu_baseline"),
               "clocks": clocks,
               "step_ms_p50": statistics.median(step_ms), "step_ms_max": max(step_ms),
               "unpipelined": {"GBps": nbytes / (t_two / 1e3) / 1e9, "ms_per_step": t_two,
                               "calls": "hg_cdc_boundaries + hg_hash_chunks"}}
        for k in ("direct", "configs", "rabin", "blockmap", "batch", "serve"):
            if k in extras:
                out[k] = extras[k]
        print(json.dumps(out), flush=True)
    if world > 1:
        dist.destroy_process_group()


# hg_cdc_hash_h2d copies an input of up to 480 MiB in 8 MiB pieces
H2D_PIECE = 8 << 20


def stage_breakdown(versions, streams, main_s, flush, h_in, d_in, dev_out, host_out, e2e_step,
                    t_kernel_ms, t_e2e_ms, reps=10):
    """Per-stage times of the e2e step, each stage alone (the paper's stage breakdown of a
    GPU hashing call, Table 1 / Fig. 4: allocation, copy in, kernel, copy out, host work):
    h2d = both versions' inputs host -> device in the library's pieces, each version on its
    stream; kernel = the device-resident step timed above; d2h = the result copies alone;
    host = the host time to enqueue one e2e step. Nothing is allocated inside the step (the
    pinned pool and the reserved device scratch are reused), so the allocation stage is 0.
    overlap_saved_ms = h2d + kernel + d2h - e2e; tail_after_h2d_ms = e2e - h2d."""
    import torch
    ends, cnts, dgs = dev_out
    h_ends, h_cnt, h_dg = host_out

    def fork(body):
        ev0 = torch.cuda.Event()
        ev0.record(main_s)
        for i, s in enumerate(streams):
            s.wait_event(ev0)
            with torch.cuda.stream(s):
                body(i)
        for s in streams:
            main_s.wait_stream(s)

    def h2d(i):
        for lo in range(0, versions[i].size, H2D_PIECE):
            d_in[i][lo:lo + H2D_PIECE].copy_(h_in[i][lo:lo + H2D_PIECE], non_blocking=True)

    def d2h(i):
        h_cnt[i].copy_(cnts[i], non_blocking=True)
        h_ends[i].copy_(ends[i], non_blocking=True)
        h_dg[i].copy_(dgs[i], non_blocking=True)

    def timed(body):
        fork(body)
        torch.cuda.synchronize()
        ev = []
        for _ in range(reps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(main_s)
            fork(body)
            b.record(main_s)
            ev.append((a, b))
        torch.cuda.synchronize()
        return statistics.median(a.elapsed_time(b) for a, b in ev)

    t_h2d, t_d2h = timed(h2d), timed(d2h)
    host = []
    for _ in range(reps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e2e_step()
        host.append((time.perf_counter() - t0) * 1e3)
    torch.cuda.synchronize()
    return {"alloc_ms": 0.0, "h2d_ms": t_h2d, "kernel_ms": t_kernel_ms, "d2h_ms": t_d2h,
            "host_enqueue_ms": statistics.median(host), "e2e_ms": t_e2e_ms,
            "overlap_saved_ms": t_h2d + t_kernel_ms + t_d2h - t_e2e_ms,
            "tail_after_h2d_ms": t_e2e_ms - t_h2d,
            "note": "each stage timed alone (CUDA events, median); h2d in 8 MiB pieces per version"}


def direct_leg(hgb, ctx, dev, flush):
    """Fixed-block MD5 / SHA-1 over 1 GiB of uniform bytes at 4 KiB, 64 KiB and 1 MiB blocks
    (digests only; at 4 KiB also digests + hash-of-hashes), and two-level identifiers of
    1 MiB blocks over 4 KiB segments; kernel time with CUDA events, L2 flushed between
    launches."""
    import torch
    from gen import inputs as G
    data = torch.from_numpy(G.uniform_bytes(1 << 30, seed=4)).to(dev)
    res = {}
    peaks, kind = measured_peaks()
    s = torch.cuda.current_stream(dev)

    def timed(fn, reps=8, warm=3):
        ts = []
        for i in range(reps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(s)
            fn()
            b.record(s)
            if i >= warm:
                ts.append((a, b))
        torch.cuda.synchronize()
        t = sum(a.elapsed_time(b) for a, b in ts) / len(ts) / 1e3
        return {"GBps": (1 << 30) / t / 1e9, "ms": t * 1e3,
                "hbm_frac": (1 << 30) / t / 1e9 / peaks["hbm_gbs"]}

    # bound of a fixed-block digest: min(HBM, int32 issue rate / operations per byte)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    issue = sms * ISSUE_LANES_PER_SM_CLK * float(peaks.get("sm_max_mhz", 2032.0)) * 1e6

    alu_pipe = sms * ALU_LANES_PER_SM_CLK * float(peaks.get("sm_max_mhz", 2032.0)) * 1e6

    def with_bound(r, ops_per_byte, alu_only_per_block):
        alu = issue / ops_per_byte / 1e9
        bound = min(peaks["hbm_gbs"], alu)
        r["roofline"] = {"bound": "hbm" if peaks["hbm_gbs"] <= alu else "alu", "peak_GBps": bound,
                         "frac": r["GBps"] / bound}
        # secondary: the ALU pipe alone, on the instructions nothing else can run
        pipe = alu_pipe / (alu_only_per_block / 64.0) / 1e9
        r["roofline"]["alu_pipe_bound_GBps"] = pipe
        r["roofline"]["frac_of_alu_pipe_bound"] = r["GBps"] / pipe
        return r

    # read-only HBM stream (a reduction over the 1 GiB input), context for the digest kernels
    ro = []
    for i in range(6):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(s)
        data.view(torch.int64).sum()
        b.record(s)
        if i >= 2:
            ro.append((a, b))
    torch.cuda.synchronize()
    res["hbm_read_only_GBps"] = (1 << 30) / (min(x.elapsed_time(y) for x, y in ro) / 1e3) / 1e9

    for algo, name in ((hgb.MD5, "md5"), (hgb.SHA1, "sha1")):
        dl = 16 if algo == hgb.MD5 else 20
        out = torch.empty(((1 << 30) // 4096, dl), dtype=torch.uint8, device=dev)
        rt = torch.empty(dl, dtype=torch.uint8, device=dev)
        opb = OPS_PER_BYTE_MD5 if algo == hgb.MD5 else OPS_PER_BYTE_SHA1
        aob = ALU_ONLY_PER_BLOCK_MD5 if algo == hgb.MD5 else ALU_ONLY_PER_BLOCK_SHA1
        # the rate of one serial digest chain: one 16 MiB block, one lane
        one = timed(lambda: ctx.hash_blocks(data[:16 << 20], 16 << 20, algo, root=False, out=out[:1]),
                    reps=4, warm=1)
        chain_rate = (16 << 20) / (one["ms"] / 1e3) / 1e9
        res[f"{name}_chain_GBps_per_chain"] = chain_rate
        for block, label in ((4096, "4KiB"), (65536, "64KiB"), (1 << 20, "1MiB")):
            r = with_bound(timed(lambda: ctx.hash_blocks(data, block, algo, root=False, out=out)), opb, aob)
            # with few blocks each is one serial chain: at most nblk chains at the single-chain rate
            chain = ((1 << 30) // block) * chain_rate
            if chain < r["roofline"]["peak_GBps"]:
                r["roofline"] = {"bound": "chain latency", "peak_GBps": chain, "frac": r["GBps"] / chain,
                                 "note": f"{(1 << 30) // block} chains x {chain_rate:.3f} GB/s per chain"}
            res[f"{name}_{label}"] = r
        r = timed(lambda: ctx.hash_blocks(data, 4096, algo, root=True, out=out, root_out=rt),
                  reps=5, warm=2)
        r["root_ms"] = r["ms"] - res[f"{name}_4KiB"]["ms"]
        r["root_share"] = r["root_ms"] / r["ms"]
        r["root_note"] = "hash-of-hashes over 4 MiB (MD5) / 5 MiB (SHA-1) of digests on a host core"
        res[f"{name}_4KiB_with_root"] = r
        ids = torch.empty(((1 << 30) >> 20, dl), dtype=torch.uint8, device=dev)
        res[f"{name}_1MiB_two_level_4KiB"] = timed(
            lambda: ctx.hash_blocks_pmd(data, 1 << 20, 4096, algo, out=ids, seg_out=out))
    ctx.sync()
    res["note"] = (f"1 GiB uniform bytes (seed 4); 262144 / 16384 / 1024 blocks; chain rate = one "
                   f"16 MiB block digested by one lane; two-level = "
                   f"H(4 KiB segment digests) per 1 MiB block; HBM peak {peaks['hbm_gbs']} GB/s ({kind})")
    return res


def blocks_leg(hgb, ctx, dev, reps=3):
    """Fixed-block digests of 1 GiB of uniform bytes in 4 KiB blocks, reps launches of MD5
    then reps of SHA-1, without the root (a short, fixed launch sequence for profiling)."""
    import torch
    from gen import inputs as G
    data = torch.from_numpy(G.uniform_bytes(1 << 30, seed=4)).to(dev)
    s = torch.cuda.current_stream(dev)
    res = {}
    for algo, name, dl in ((hgb.MD5, "md5", 16), (hgb.SHA1, "sha1", 20)):
        out = torch.empty(((1 << 30) // 4096, dl), dtype=torch.uint8, device=dev)
        ts = []
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(s)
            ctx.hash_blocks(data, 4096, algo, root=False, out=out)
            b.record(s)
            ts.append((a, b))
        torch.cuda.synchronize()
        res[name] = {"ms": [x.elapsed_time(y) for x, y in ts]}
    ctx.sync()
    return res


def probe_lib():
    """The benchmark's integer-pipe probe library (built beside its source)."""
    import ctypes as C
    path = os.path.join(ROOT, "paper_1202_3669_b300", "bench_probe", "libhgprobe.so")
    if not os.path.exists(path):
        import importlib.util
        spec = importlib.util.spec_from_file_location(
            "_hg_build", os.path.join(ROOT, "paper_1202_3669_b300", "build.py"))
        mod = importlib.util.module_from_spec(spec)
        spec.loader.exec_module(mod)
        mod.build_probe()
    lib = C.CDLL(path)
    lib.hgp_probe_int_pipe.argtypes = [C.c_int, C.c_int, C.c_uint32, C.c_uint32, C.c_void_p, C.c_void_p]
    return lib


def alu_leg(dev, iters=65536):
    """Integer-pipe throughput probe: 8 CTAs x 256 threads per SM, 8 independent chains per
    thread, per operation class; lanes per clock per SM at the maximum SM clock (the clock
    the bench runs at, sampled alongside)."""
    import ctypes as C

    import torch
    lib = probe_lib()
    s = torch.cuda.current_stream(dev)
    peaks, _ = measured_peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2032.0))
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    out = {}
    ops = C.c_uint64()
    for kind, name in ((0, "lop3"), (1, "iadd3"), (2, "shf_funnel"), (3, "md5_op_mix"),
                       (4, "mad_by_runtime_1")):
        ts = []
        for i in range(5):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(s)
            assert lib.hgp_probe_int_pipe(dev.index or 0, kind, iters, 8, C.byref(ops), s.cuda_stream) == 0
            b.record(s)
            if i >= 2:
                ts.append((a, b))
        torch.cuda.synchronize()
        t = statistics.median(x.elapsed_time(y) for x, y in ts) / 1e3
        out[name] = {"Tops": ops.value / t / 1e12, "lanes_per_sm_clk": ops.value / t / (sms * sm_max * 1e6)}
    out["note"] = f"{sms} SMs at {sm_max:.0f} MHz; md5_op_mix counts 4 ops per MD5-like step"
    return out


def configs_leg(hgb, ctx, dev, flush):
    """The other measured configurations: 8 MiB / 4 KiB blocks in one call (digests + hash-of-
    hashes, MD5 and SHA-1), and 1 GiB chunking (uniform seed 4, text-like seed 5) kernel-only
    and end to end from a pinned host buffer, plus 1 GiB fixed-block digests end to end (host
    pieces copied on two streams, each piece hashed as it lands). Median of the timed runs,
    L2 flushed before each."""
    import torch
    from gen import inputs as G
    s = torch.cuda.current_stream(dev)

    def med(fn, reps=10, warm=2):
        ts = []
        for i in range(reps + warm):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(s)
            fn()
            b.record(s)
            if i >= warm:
                ts.append((a, b))
        torch.cuda.synchronize()
        return statistics.median(a.elapsed_time(b) for a, b in ts) / 1e3

    res = {}
    small = torch.from_numpy(G.uniform_bytes(8 << 20, seed=1)).to(dev)
    for algo, name in ((hgb.MD5, "md5"), (hgb.SHA1, "sha1")):
        dl = 16 if algo == hgb.MD5 else 20
        out = torch.empty((2048, dl), dtype=torch.uint8, device=dev)
        rt = torch.empty(dl, dtype=torch.uint8, device=dev)
        t = med(lambda: ctx.hash_blocks(small, 4096, algo, root=True, out=out, root_out=rt))
        res[f"blocks_8MiB_4KiB_{name}_with_root"] = {"ms": t * 1e3, "GBps": (8 << 20) / t / 1e9}
    del small
    n = 1 << 30
    d = torch.empty(n, dtype=torch.uint8, device=dev)
    cap = n // 2048 + 2
    outs = (torch.empty(cap, dtype=torch.int64, device=dev), torch.zeros(1, dtype=torch.int64, device=dev),
            torch.empty((cap, 16), dtype=torch.uint8, device=dev))
    h_ends = torch.empty(cap, dtype=torch.int64).pin_memory()
    h_dg = torch.empty((cap, 16), dtype=torch.uint8).pin_memory()
    h_cnt = torch.empty(1, dtype=torch.int64).pin_memory()
    p = hgb.default_params()
    for dist, gen in (("uniform", lambda: G.uniform_bytes(n, seed=4)),
                      ("text", lambda: G.text_like_bytes(n, seed=5))):
        host = torch.from_numpy(gen()).pin_memory()
        d.copy_(host)
        t_k = med(lambda: ctx.cdc_hash(d, hgb.MD5, p, out=outs, stream=s))

        def e2e():
            ctx.cdc_hash_from_host(host, d, hgb.MD5, p, out=outs, stream=s)
            h_cnt.copy_(outs[1], non_blocking=True)
            h_ends.copy_(outs[0], non_blocking=True)
            h_dg.copy_(outs[2], non_blocking=True)
        t_e = med(e2e, reps=5)
        ctx.sync()
        res[f"cdc_1GiB_{dist}_md5"] = {"kernel_GBps": n / t_k / 1e9, "kernel_ms": t_k * 1e3,
                                           "e2e_GBps": n / t_e / 1e9, "e2e_ms": t_e * 1e3,
                                           "chunks": int(outs[1].item())}
        if dist == "uniform":
            streams = [torch.cuda.Stream(dev) for _ in range(2)]
            piece = 64 << 20
            for algo, name in ((hgb.MD5, "md5"), (hgb.SHA1, "sha1")):
                dl = 16 if algo == hgb.MD5 else 20
                dg = torch.empty((n // 4096, dl), dtype=torch.uint8, device=dev)
                h_out = torch.empty((n // 4096, dl), dtype=torch.uint8).pin_memory()

                def blocks_e2e():
                    ev0 = torch.cuda.Event()
                    ev0.record(s)
                    for k in range(n // piece):
                        st = streams[k % 2]
                        st.wait_event(ev0)
                        with torch.cuda.stream(st):
                            d[k * piece:(k + 1) * piece].copy_(host[k * piece:(k + 1) * piece],
                                                              non_blocking=True)
                            seg = dg[k * piece // 4096:(k + 1) * piece // 4096]
                            ctx.hash_blocks(d[k * piece:(k + 1) * piece], 4096, algo, root=False,
                                            out=seg, stream=st)
                            h_out[k * piece // 4096:(k + 1) * piece // 4096].copy_(seg, non_blocking=True)
                    for st in streams:
                        s.wait_stream(st)
                t_b = med(blocks_e2e, reps=5)
                res[f"blocks_1GiB_uniform_4KiB_{name}_e2e"] = {"GBps": n / t_b / 1e9, "ms": t_b * 1e3}
        del host
    ctx.sync()
    res["note"] = ("blocks_8MiB: one hg_hash_blocks call with the root (latency-bound: 2048 chains "
                   "+ one serial root); cdc_1GiB: hg_cdc_hash on device input vs hg_cdc_hash_h2d from pinned "
                   "host memory (+ D2H of ends and digests); fixed-block e2e: 64 MiB pieces copied and "
                   "hashed on two streams, digests copied back (root not included)")
    return res


def rabin_leg(hgb, dev, flush, steps=50):
    """The chunking step of the main workload with the Rabin fingerprint window (48 bytes,
    LBFS-style) instead of the MD5 window: whole step (both versions, two streams), the
    window kernel alone on the base version, and the shared-chunk fraction."""
    import torch
    versions = workload()
    p = hgb.params(window=48, window_hash=hgb.WIN_RABIN)
    ctxs = [hgb.Context(dev.index or 0) for _ in versions]
    streams = [torch.cuda.Stream(dev) for _ in versions]
    d_in = [torch.from_numpy(v).to(dev) for v in versions]
    cap = [v.size // p.min_chunk + 2 for v in versions]
    outs = [(torch.empty(c, dtype=torch.int64, device=dev), torch.zeros(1, dtype=torch.int64, device=dev),
             torch.empty((c, 16), dtype=torch.uint8, device=dev)) for c in cap]
    main_s = torch.cuda.current_stream(dev)

    def step():
        ev0 = torch.cuda.Event()
        ev0.record(main_s)
        for i in range(len(versions)):
            streams[i].wait_event(ev0)
            ctxs[i].cdc_hash(d_in[i], hgb.MD5, p, out=outs[i], stream=streams[i])
        for st in streams:
            main_s.wait_stream(st)

    def timed(fn, n):
        ts = []
        for i in range(n + 3):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(main_s)
            fn()
            b.record(main_s)
            if i >= 3:
                ts.append((a, b))
        torch.cuda.synchronize()
        return sum(a.elapsed_time(b) for a, b in ts) / len(ts) / 1e3

    t_step = timed(step, steps)
    bm = torch.empty((versions[0].size + 31) // 32, dtype=torch.int32, device=dev)
    t_win = timed(lambda: ctxs[0].window_bitmap(d_in[0], p, out=bm, stream=main_s), 20)
    for c in ctxs:
        c.sync()
    k0, k1 = int(outs[0][1].item()), int(outs[1][1].item())
    s0 = {bytes(r) for r in outs[0][2][:k0].cpu().numpy()}
    e1 = outs[1][0][:k1].cpu().numpy()
    sz1 = np.diff(np.concatenate([[0], e1]))
    shared = sum(int(z) for z, r in zip(sz1, outs[1][2][:k1].cpu().numpy()) if bytes(r) in s0)
    nbytes = sum(v.size for v in versions)
    return {"GBps": nbytes / t_step / 1e9, "ms_per_step": t_step * 1e3,
            "window_kernel_GBps": versions[0].size / t_win / 1e9, "window_kernel_ms": t_win * 1e3,
            "chunks": [k0, k1], "shared_fraction": shared / versions[1].size,
            "params": {"window": 48, "mask_bits": 13, "magic": 0x0F0F, "min": 2048, "max": 65536,
                       "window_hash": "rabin (degree-31 polynomial 0x9E3779BB)", "digest": "md5"}}


def blockmap_leg(hgb, ctx, dev, flush, n=1 << 24):
    """Device block map: insert n random MD5-sized digests, then look up n digests of which
    half are stored (chunk sizes given, so found bytes are summed too). Kernel time with CUDA
    events; digests per second."""
    import torch
    g = np.random.default_rng(13)
    known = torch.from_numpy(g.integers(0, 256, (n, 16), dtype=np.uint8)).to(dev)
    pick = torch.from_numpy(g.integers(0, n, n // 2)).to(dev)
    fresh = torch.from_numpy(g.integers(0, 256, (n - n // 2, 16), dtype=np.uint8)).to(dev)
    queries = torch.cat([known[pick], fresh])
    ends = torch.cumsum(torch.from_numpy(g.integers(1, 65536, n)).to(dev), 0)
    s = torch.cuda.current_stream(dev)
    ins, look = [], []
    m = hgb.BlockMap(ctx, hgb.MD5, capacity=n)
    for i in range(4):
        m.clear(stream=s)
        flush.zero_()
        a, b, c = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        a.record(s)
        m.insert(known, stream=s)
        b.record(s)
        hits, res = m.lookup(queries, ends=ends, want_hits=True, stream=s)
        c.record(s)
        if i:
            ins.append((a, b))
            look.append((b, c))
    torch.cuda.synchronize()
    ctx.sync()
    found = int(res[0].item())
    m.close()
    t_ins = sum(x.elapsed_time(y) for x, y in ins) / len(ins) / 1e3
    t_look = sum(x.elapsed_time(y) for x, y in look) / len(look) / 1e3
    return {"digests": n, "insert_Mdigests_per_s": n / t_ins / 1e6, "insert_ms": t_ins * 1e3,
            "lookup_Mdigests_per_s": n / t_look / 1e6, "lookup_ms": t_look * 1e3,
            "found": found, "slots": 2 * n,
            "note": "random 16-byte digests; table 2n slots x 24 B; lookups half hits"}


def batch_leg(hgb, ctx, dev, flush, nfiles=4096):
    """4096 files, log-normal sizes (median 64 KiB, sigma 2.4, 512 B..256 MiB, about 3.6 GiB),
    chunking + per-chunk SHA-1: one batched pass (graph replay, autotuned) against one launch
    sequence per file on one stream with the same kernels."""
    import torch
    from gen import inputs as G
    seed, sizes = G.batch_workload_seed()
    sizes = sizes[:nfiles]
    data, off = G.files_from_sizes(sizes, seed + 1000)
    d = torch.from_numpy(data).to(dev)
    total = int(off[-1])
    del data
    b = hgb.Batch(ctx, off)
    out = b.outputs(hgb.SHA1)
    s = torch.cuda.current_stream(dev)
    best = b.autotune(d, hgb.SHA1, out=out)

    def timed(fn, reps):
        ts = []
        for _ in range(reps):
            flush.zero_()
            a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(s)
            fn()
            e.record(s)
            ts.append((a, e))
        torch.cuda.synchronize()
        return sum(a.elapsed_time(e) for a, e in ts) / len(ts) / 1e3

    b.cdc_hash(d, hgb.SHA1, out=out, graph=True)
    t_graph = timed(lambda: b.cdc_hash(d, hgb.SHA1, out=out, graph=True), 5)
    t_plain = timed(lambda: b.cdc_hash(d, hgb.SHA1, out=out), 5)
    b.sync()
    chunks = int(out[1].sum().item())
    # one launch sequence per file: boundaries then chunk digests, same kernels
    p = hgb.default_params()
    caps = [int(sz) // p.min_chunk + 2 for sz in sizes]
    ends = torch.empty(max(caps), dtype=torch.int64, device=dev)
    cnt = torch.zeros(1, dtype=torch.int64, device=dev)
    dg = torch.empty((max(caps), 20), dtype=torch.uint8, device=dev)
    ctx.reserve(int(max(sizes)))
    views = [d[int(off[f]):int(off[f + 1])] for f in range(len(sizes))]

    def per_file():
        for f, v in enumerate(views):
            ctx.cdc_boundaries(v, p, cap=caps[f], out=ends, count=cnt, stream=s)
            ctx.hash_chunks(v, ends[:caps[f]], hgb.SHA1, count=cnt, out=dg, stream=s)

    per_file()
    t_file = timed(per_file, 2)
    ctx.sync()
    return {"files": len(sizes), "bytes": total, "seed": seed, "chunks": chunks,
            "batched_graph_GBps": total / t_graph / 1e9, "batched_GBps": total / t_plain / 1e9,
            "per_file_GBps": total / t_file / 1e9, "batched_over_per_file": t_file / t_graph,
            "ms": {"graph": t_graph * 1e3, "plain": t_plain * 1e3, "per_file": t_file * 1e3},
            "tuning": {"window_ctas_per_sm": best.window_ctas_per_sm,
                       "hash_threads": best.hash_threads, "hash_ctas_per_sm": best.hash_ctas_per_sm,
                       "long_chunk_bytes": best.long_chunk_bytes},
            "note": "per-file: hg_cdc_boundaries + hg_hash_chunks per file on one stream"}


def serve_leg(hgb, ctx, capacity_gbps, per_file_gbps=None, fracs=(0.1, 0.4, 0.7, 1.0, 1.2),
              max_req=20000, seconds=2.5):
    """Open-loop Poisson arrivals; request sizes log-normal as in the batch workload; 70 %
    chunking + MD5, 30 % 64 KiB-block SHA-1 with root; 32 GiB device budget. Payloads come
    from a 1 GiB buffer of the library's pinned pool (request i reads a seeded slice);
    latency is completion minus scheduled arrival.

    Two sweeps: the five rates as fractions of the batched capacity (device-resident
    batch, the configuration's definition), and the same fractions of the served ceiling
    (the throughput the server sustains when offered more than it can take, which the
    host link bounds). p99 is reported for each; `p99_at_3x` is the p99 at the highest
    rate that is sustained (achieved >= 95 % of offered) at >= 3x the per-file-launch
    throughput."""
    import torch
    from gen import inputs as G
    pool_bytes = 1 << 30
    sctx = hgb.Context(ctx.device.index, budget=40 << 30)      # the server's own context
    pbuf = sctx.alloc_pinned(pool_bytes)
    pbuf.numpy()[:] = G.uniform_bytes(pool_bytes, seed=77)
    base = pbuf.ptr
    srv = hgb.Server(sctx, device_budget=32 << 30, max_wave_bytes=1 << 30)
    sizes_all = G.lognormal_sizes(200000, seed=78)
    mean_size = float(sizes_all.mean())

    def run(rate_gbps, k, secs=seconds):
        lam = rate_gbps * 1e9 / mean_size
        n = int(min(max_req, max(200, lam * secs)))
        g = G.rng(80 + k)
        sizes = G.lognormal_sizes(n, seed=90 + k)
        offs = (g.random(n) * (pool_bytes - sizes)).astype(np.int64)
        kinds = g.random(n) < 0.7
        reqs = []
        for i in range(n):
            r = hgb.hg_request()
            r.h_data = base + int(offs[i])
            r.n = int(sizes[i])
            if kinds[i]:
                r.kind, r.algo, r.block, r.want_root = hgb.HG_REQ_CDC, hgb.MD5, 0, 0
            else:
                r.kind, r.algo, r.block, r.want_root = hgb.HG_REQ_BLOCKS, hgb.SHA1, 65536, 1
            reqs.append(r)
        arrivals = (G.poisson_arrivals(lam, n, seed=100 + k) * 1e9).astype(np.uint64)
        lat, span = srv.replay(reqs, arrivals)
        lat_ms = lat.astype(np.float64) / 1e6
        total = int(sizes.sum())
        return {"requests": n, "offered_GBps": total / (arrivals[-1] / 1e9) / 1e9,
                "achieved_GBps": total / (span / 1e9) / 1e9,
                "p50_ms": float(np.percentile(lat_ms, 50)),
                "p99_ms": float(np.percentile(lat_ms, 99)),
                "mean_request_bytes": total / n}

    out = {"capacity_GBps": capacity_gbps, "budget_bytes": 32 << 30, "rates": []}
    for k, frac in enumerate(fracs):
        out["rates"].append({"frac": frac, "of": "batched capacity", **run(frac * capacity_gbps, k)})
    # the served ceiling: offered twice the batched capacity, what the server sustains
    sat = run(2.0 * capacity_gbps, 20, secs=1.5)
    ceiling = sat["achieved_GBps"]
    out["served_ceiling_GBps"] = ceiling
    out["rates_vs_served_ceiling"] = []
    for k, frac in enumerate(fracs):
        out["rates_vs_served_ceiling"].append({"frac": frac, "of": "served ceiling",
                                               **run(frac * ceiling, 10 + k)})
    if per_file_gbps:
        ok = [r for r in out["rates"] + out["rates_vs_served_ceiling"]
              if r["achieved_GBps"] >= 0.95 * r["offered_GBps"] and r["achieved_GBps"] >= 3 * per_file_gbps]
        if ok:
            best = max(ok, key=lambda r: r["achieved_GBps"])
            out["p99_at_3x"] = {"achieved_GBps": best["achieved_GBps"], "p99_ms": best["p99_ms"],
                                "p50_ms": best["p50_ms"], "per_file_GBps": per_file_gbps,
                                "ratio_to_per_file": best["achieved_GBps"] / per_file_gbps}
    out["waves"] = srv.stats()["waves"]
    out["pinned_pool"] = sctx.pinned_stats()
    srv.close()
    pbuf.free()
    sctx.close()
    return out


if __name__ == "__main__":
    main()
