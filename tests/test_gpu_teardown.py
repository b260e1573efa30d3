"""Process exit with library objects still open.

A program may end without closing its contexts, batches, servers, streams or block
maps. The binding closes whatever is still open in an exit handler (children before
the contexts they were made on), while the CUDA runtime is intact; finalizers that
run later, during interpreter teardown, do not call into the library. A process
that left several contexts and autotuned batches open once crashed (SIGSEGV) after
its last statement; this runs such a program in a child process and wants a clean
exit.
"""
import os
import subprocess
import sys
import textwrap

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PROGRAM = textwrap.dedent("""
    import sys
    sys.path.insert(0, {root!r})
    import numpy as np, torch
    import paper_1202_3669_b300 as hgb
    from gen import inputs as G
    dev = torch.device("cuda", 0)
    sizes = G.lognormal_sizes(256, seed=31, hi=4 << 20)
    data, off = G.files_from_sizes(sizes, 32)
    d = torch.from_numpy(data).to(dev)
    k = len(sizes) // 2
    ctxs = [hgb.Context(0) for _ in range(3)]
    offs = [off, off[:k + 1], off[k:] - off[k]]
    views = [d, d[:int(off[k])], d[int(off[k]):]]
    batches = []
    for c, o, v in zip(ctxs, offs, views):
        b = hgb.Batch(c, o)
        out = b.outputs(hgb.SHA1)
        b.autotune(v, hgb.SHA1, out=out)
        b.cdc_hash(v, hgb.SHA1, out=out, graph=True)
        batches.append((b, out))
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    batches[1][0].cdc_hash(views[1], hgb.SHA1, out=batches[1][1], graph=True, stream=s1)
    batches[2][0].cdc_hash(views[2], hgb.SHA1, out=batches[2][1], graph=True, stream=s2)
    srv = hgb.Server(ctxs[0], device_budget=1 << 30, max_wave_bytes=64 << 20)
    t = srv.submit(G.uniform_bytes(100_000, 33), hgb.HG_REQ_CDC, hgb.MD5)
    srv.poll(t)
    st = hgb.CdcStream(ctxs[1], hgb.MD5, max_feed=1 << 20)
    st.feed(d[:1 << 20])
    bm = hgb.BlockMap(ctxs[2], hgb.MD5, capacity=1 << 12)
    e, c, g = ctxs[2].cdc_hash(d[:4 << 20], hgb.MD5)
    bm.insert(g, c)
    pb = ctxs[0].alloc_pinned(1 << 20)
    torch.cuda.synchronize()
    print("end of program", flush=True)
""")


def test_exit_with_objects_open():
    r = subprocess.run([sys.executable, "-X", "faulthandler", "-c", PROGRAM.format(root=ROOT)],
                       capture_output=True, text=True, timeout=600)
    assert "end of program" in r.stdout, r.stdout + r.stderr
    assert r.returncode == 0, f"exit status {r.returncode}\n{r.stderr[-2000:]}"
