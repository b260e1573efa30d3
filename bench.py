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
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "hashed GB/s (CDC: 20-byte MD5 window + min/max boundaries + per-chunk MD5)"
# hg_cdc_hash is the public call timed; hg_cdc_boundaries + hg_hash_chunks (the
# same kernels without segment pipelining) is reported beside it.
UNIT = "GB/s"
WORKLOAD = "cdc_64MiB_base_plus_1pct_edited_version"
# Algorithmic cost of one window hash in integer-ALU instructions (3-input logic op,
# 3-input add and the rotate-add each count one): 42 operations with a constant
# message word x 3 + 19 with a data word x 4, + 3.75 funnel shifts to assemble
# the window, + 4 for the test and bit collection = 208 (ncu counted 194 ALU-pipe + 10
# FMA-pipe instructions per window).
ALU_OPS_PER_WINDOW = 208
ALU_LANES_PER_SM_CLK = 64     # integer ALU pipe: one warp instruction per 2 clocks per scheduler
TWO_INPUT_OPS_PER_WINDOW = 270  # the same work counted in 2-input operations
ISSUE_LANES_PER_SM_CLK = 128  # 4 schedulers x 32 lanes
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
                    choices=["direct", "batch", "serve", "rabin", "blockmap", "configs", "alu"],
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


def cpu_baseline(versions, budget_s: float = 12.0):
    """The oracle as it stands, on the host cores, on a bounded sample of the workload."""
    import oracle
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
    return {"value": total / dt / 1e9, "unit": UNIT, "cores": nthreads, "kind": "oracle",
            "single_thread": single,
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
            res = alu_leg(hgb, ctx, dev)
        else:
            res = serve_leg(hgb, ctx, batch_leg(hgb, ctx, dev, flush)["batched_graph_GBps"])
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

    # e2e: pinned host inputs -> device -> boundaries + digests -> pinned host
    h_in = [torch.from_numpy(v).pin_memory() for v in versions]
    h_ends = [torch.empty(c, dtype=torch.int64).pin_memory() for c in cap]
    h_cnt = [torch.empty(1, dtype=torch.int64).pin_memory() for _ in versions]
    h_dg = [torch.empty((c, 16), dtype=torch.uint8).pin_memory() for c in cap]
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
    peak_tops = sm_count * ALU_LANES_PER_SM_CLK * sm_max * 1e6 / 1e12
    achieved = windows * ALU_OPS_PER_WINDOW / t_win / 1e12
    issue_peak = sm_count * ISSUE_LANES_PER_SM_CLK * sm_max * 1e6 / 1e12
    tr = kernel_traffic("k_window_bitmap", WINDOW_KERNEL_SRC)
    roofline = {"bound": "alu", "kernel": "k_window_bitmap<20>", "achieved": achieved,
                "peak": peak_tops, "unit": "Tops/s (int32 ALU-pipe instructions)",
                "frac": achieved / peak_tops,
                "peak_kind": f"{sm_count} SMs x {ALU_LANES_PER_SM_CLK} lanes/clk (integer ALU pipe) x "
                             f"{sm_max:.0f} MHz (max SM clock, {peak_kind} clock); recipe unit counts",
                "ops_per_window": ALU_OPS_PER_WINDOW, "windows_per_launch": windows,
                "launch_ms": t_win * 1e3, "window_GBps": versions[0].size / t_win / 1e9,
                "frac_two_input_count_vs_issue_peak": windows * TWO_INPUT_OPS_PER_WINDOW / t_win / 1e12 / issue_peak,
                "traffic": (tr["dram_bytes_per_launch"] * versions[0].size / tr["input_bytes"]) if tr else None}
    if clocks.get("sm_mhz"):
        roofline["frac_at_observed_clock"] = achieved / (peak_tops * clocks["sm_mhz"] / sm_max)
    # the integer pipe's rate measured by a probe (per operation class), beside the peak used
    roofline["measured_int_pipe"] = alu_leg(hgb, ctxs[0], dev)

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
        extras["serve"] = serve_leg(hgb, ctxs[0], extras["batch"]["batched_graph_GBps"])
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
                       "pinned_h2d_copy_GBps": h2d_gbps},
               "gpu_launches": launches_per_step * args.steps,
               "roofline": roofline,
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

    for algo, name in ((hgb.MD5, "md5"), (hgb.SHA1, "sha1")):
        dl = 16 if algo == hgb.MD5 else 20
        out = torch.empty(((1 << 30) // 4096, dl), dtype=torch.uint8, device=dev)
        rt = torch.empty(dl, dtype=torch.uint8, device=dev)
        for block, label in ((4096, "4KiB"), (65536, "64KiB"), (1 << 20, "1MiB")):
            res[f"{name}_{label}"] = timed(
                lambda: ctx.hash_blocks(data, block, algo, root=False, out=out))
        res[f"{name}_4KiB_with_root"] = timed(
            lambda: ctx.hash_blocks(data, 4096, algo, root=True, out=out, root_out=rt), reps=5, warm=2)
        ids = torch.empty(((1 << 30) >> 20, dl), dtype=torch.uint8, device=dev)
        res[f"{name}_1MiB_two_level_4KiB"] = timed(
            lambda: ctx.hash_blocks_pmd(data, 1 << 20, 4096, algo, out=ids, seg_out=out))
    ctx.sync()
    res["note"] = (f"1 GiB uniform bytes (seed 4); 262144 / 16384 / 1024 blocks; two-level = "
                   f"H(4 KiB segment digests) per 1 MiB block; HBM peak {peaks['hbm_gbs']} GB/s ({kind})")
    return res


def alu_leg(hgb, ctx, dev, iters=65536):
    """Integer-pipe throughput probe (hg_probe_int_pipe): 8 CTAs x 256 threads per SM, 8
    independent chains per thread, per operation class; lanes per clock per SM at the
    maximum SM clock (the clock the bench runs at, sampled alongside)."""
    import torch
    s = torch.cuda.current_stream(dev)
    peaks, _ = measured_peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2032.0))
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    out = {}
    for kind, name in ((0, "lop3"), (1, "iadd3"), (2, "shf_funnel"), (3, "md5_op_mix")):
        ts = []
        for i in range(5):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(s)
            ops = ctx.probe_int_pipe(kind, iters, 8, stream=s)
            b.record(s)
            if i >= 2:
                ts.append((a, b))
        torch.cuda.synchronize()
        t = statistics.median(x.elapsed_time(y) for x, y in ts) / 1e3
        out[name] = {"Tops": ops / t / 1e12, "lanes_per_sm_clk": ops / t / (sms * sm_max * 1e6)}
    ctx.sync()
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
    c1 = torch.from_numpy(G.uniform_bytes(8 << 20, seed=1)).to(dev)
    for algo, name in ((hgb.MD5, "md5"), (hgb.SHA1, "sha1")):
        dl = 16 if algo == hgb.MD5 else 20
        out = torch.empty((2048, dl), dtype=torch.uint8, device=dev)
        rt = torch.empty(dl, dtype=torch.uint8, device=dev)
        t = med(lambda: ctx.hash_blocks(c1, 4096, algo, root=True, out=out, root_out=rt))
        res[f"c1_8MiB_4KiB_{name}_with_root"] = {"ms": t * 1e3, "GBps": (8 << 20) / t / 1e9}
    del c1
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
        res[f"c3_1GiB_{dist}_cdc_md5"] = {"kernel_GBps": n / t_k / 1e9, "kernel_ms": t_k * 1e3,
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
                res[f"c3_1GiB_uniform_4KiB_{name}_e2e"] = {"GBps": n / t_b / 1e9, "ms": t_b * 1e3}
        del host
    ctx.sync()
    res["note"] = ("c1: one hg_hash_blocks call with the root (latency-bound: 2048 chains + one "
                   "serial root); c3: hg_cdc_hash on device input vs hg_cdc_hash_h2d from pinned "
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


def serve_leg(hgb, ctx, capacity_gbps, fracs=(0.1, 0.4, 0.7, 1.0, 1.2), max_req=20000,
              seconds=2.5):
    """Open-loop Poisson arrivals at fractions of the batched capacity; request sizes log-normal
    as in the batch workload; 70 % chunking + MD5, 30 % 64 KiB-block SHA-1 with root; 32 GiB
    device budget. Payloads come from a 1 GiB pinned pool (request i reads a seeded slice);
    latency is completion minus scheduled arrival."""
    import torch
    from gen import inputs as G
    pool_bytes = 1 << 30
    pool = torch.from_numpy(G.uniform_bytes(pool_bytes, seed=77)).pin_memory()
    base = pool.data_ptr()
    sctx = hgb.Context(ctx.device.index, budget=40 << 30)      # the server's own context
    srv = hgb.Server(sctx, device_budget=32 << 30, max_wave_bytes=1 << 30)
    out = {"capacity_GBps": capacity_gbps, "budget_bytes": 32 << 30, "rates": []}
    sizes_all = G.lognormal_sizes(200000, seed=78)
    mean_size = float(sizes_all.mean())
    for k, frac in enumerate(fracs):
        lam = frac * capacity_gbps * 1e9 / mean_size
        n = int(min(max_req, max(200, lam * seconds)))
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
        out["rates"].append({"frac": frac, "requests": n, "offered_GBps": total / (arrivals[-1] / 1e9) / 1e9,
                             "achieved_GBps": total / (span / 1e9) / 1e9,
                             "p50_ms": float(np.percentile(lat_ms, 50)),
                             "p99_ms": float(np.percentile(lat_ms, 99)),
                             "mean_request_bytes": total / n})
    out["waves"] = srv.stats()["waves"]
    srv.close()
    sctx.close()
    return out


if __name__ == "__main__":
    main()
