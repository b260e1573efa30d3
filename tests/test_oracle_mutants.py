"""The pins are sensitive: plausible mistakes planted in a copy of the oracle fail them.

Each mutant is a one-token change to a copy of the oracle's C source (a wrong
rotation, a dropped term, a swapped byte order, an off-by-one cut, an
exclusive bound), compiled on the CPU into a throw-away library. The same pin
checks that the real oracle passes must reject every mutant.
"""
import json
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle
from gen import inputs as G
from tests.pins import brute_window_cuts, brute_window_cuts_with, check_chunking, ref_digest

ORACLE_DIR = os.path.dirname(os.path.abspath(oracle.__file__))
HERE = os.path.dirname(os.path.abspath(__file__))

MUTANTS = [
    ("md5.c", "{7, 12, 17, 22}", "{7, 12, 17, 23}"),                 # wrong rotation
    ("md5.c", "return (x & z) | (y & ~z);", "return (x & y) | (y & ~z);"),  # wrong G
    ("md5.c", "tail[rem] = 0x80;", "tail[rem] = 0x01;"),              # wrong padding bit
    ("md5.c", "tail[tlen - 8 + j] = (uint8_t)(bits >> (8 * j));",
              "tail[tlen - 1 - j] = (uint8_t)(bits >> (8 * j));"),   # length byte order
    ("md5.c", "k = (3 * i + 5) % 16;", "k = (3 * i + 3) % 16;"),       # wrong word index
    ("md5.c", "st[0] += a; st[1] += b;", "st[0] += a; st[1] += c;"),   # wrong feed-forward
    ("sha1.c", "c = rotl(b, 30);", "c = rotl(b, 29);"),
    ("sha1.c", "W[t] = rotl(W[t - 3] ^ W[t - 8] ^ W[t - 14] ^ W[t - 16], 1);",
               "W[t] = W[t - 3] ^ W[t - 8] ^ W[t - 14] ^ W[t - 16];"),  # SHA-0 schedule
    ("sha1.c", "+ e + Kc[t / 20]", "+ Kc[t / 20]"),                     # dropped term
    ("direct.c", "hgo_digest(algo, digests, nblk * (uint64_t)dl, root);",
                 "hgo_digest(algo, digests, (nblk ? nblk - 1 : 0) * (uint64_t)dl, root);"),
    ("direct.c", "uint64_t hi = lo + block < n ? lo + block : n;",
                 "uint64_t hi = lo + block;"),                          # pads the short block
    ("direct.c", "uint64_t b = a + segment < blk_end ? a + segment : blk_end;",
                 "uint64_t b = a + segment;"),                          # pads the short segment
    ("direct.c", "hgo_digest(algo, buf, nseg * (uint64_t)dl, ids + i * (uint64_t)dl);",
                 "hgo_digest(algo, buf, (nseg - 1) * (uint64_t)dl, ids + i * (uint64_t)dl);"),
    ("direct.c", "for (uint64_t a = lo; a < blk_end; a += segment) {",
                 "for (uint64_t a = 0; a < blk_end - lo; a += segment) {"),  # segments from 0
    ("rabin.c", "for (int j = 7; j >= 0; j--) {", "for (int j = 0; j < 8; j++) {"),   # bit order
    ("rabin.c", "if (r & 0x80000000u) r ^= HGO_RABIN_POLY;",
                "if (r & 0x40000000u) r ^= HGO_RABIN_POLY;"),           # wrong degree
    ("rabin.c", "r = (r << 1) | ((msg[i] >> j) & 1u);",
                "r = (r << 1) ^ ((msg[len - 1 - i] >> j) & 1u);"),      # bytes reversed
    ("cdc.c", "uint32_t h = kind == HGO_WIN_RABIN ? hgo_rabin_fingerprint(w, window)",
              "uint32_t h = kind == HGO_WIN_RABIN ? hgo_rabin_fingerprint(w + 1, window - 1)"),
    ("cdc.c", "j->cuts[j->count++] = p + 1;", "j->cuts[j->count++] = p;"),  # cut before window
    ("cdc.c", "return (uint32_t)d[0] | ((uint32_t)d[1] << 8)", "return (uint32_t)d[3] | ((uint32_t)d[2] << 8)"),
    ("cdc.c", "cands[k] < s + min_chunk", "cands[k] <= s + min_chunk"),  # exclusive min
    ("cdc.c", "while (k < ncand && cands[k] < s + min_chunk) k++;",
              "while (k < ncand && cands[k] <= s) k++;"),              # min ignored
    ("cdc.c", "else if (s + max_chunk < n) cut = s + max_chunk;",
              "else if (s + max_chunk < n) cut = s + max_chunk - 1;"),
]


def build_mutant(tmp_path, fname, old, new):
    d = tmp_path / "m"
    d.mkdir()
    for f in os.listdir(ORACLE_DIR):
        if f.endswith((".c", ".h")):
            shutil.copy(os.path.join(ORACLE_DIR, f), d / f)
    src = (d / fname).read_text()
    assert src.count(old) == 1, (fname, old)
    (d / fname).write_text(src.replace(old, new))
    out = d / "libmut.so"
    subprocess.run(["gcc", "-std=c99", "-O1", "-fPIC", "-shared", "-pthread",
                    "-D_POSIX_C_SOURCE=200809L", "-o", str(out),
                    *[str(d / f) for f in ("md5.c", "sha1.c", "direct.c", "cdc.c", "rabin.c")], "-lm"],
                   check=True)
    return oracle.lib(str(out))


def pins_pass(L) -> bool:
    """The pin checks of the oracle test-suite, at small sizes."""
    buf = G.uniform_bytes(300, seed=101).tobytes()
    for algo in (oracle.MD5, oracle.SHA1):
        for n in range(0, 300):
            if oracle.digest(algo, buf[:n], L) != ref_digest(algo, buf[:n]):
                return False
    data = G.uniform_bytes(5000, seed=9).tobytes()
    for algo in (oracle.MD5, oracle.SHA1):
        dg, root = oracle.hash_blocks(algo, data, 1024, L=L)
        parts = [ref_digest(algo, data[i:i + 1024]) for i in range(0, 5000, 1024)]
        if [r.tobytes() for r in dg] != parts or root != ref_digest(algo, b"".join(parts)):
            return False
        ids = oracle.hash_blocks_pmd(algo, data, 2100, 300, L=L)
        want = []
        for lo in range(0, 5000, 2100):
            blk = data[lo:lo + 2100]
            want.append(ref_digest(algo, b"".join(ref_digest(algo, blk[a:a + 300])
                                                  for a in range(0, len(blk), 300))))
        if [r.tobytes() for r in ids] != want:
            return False
    # Rabin window: hand-reduced values and GF(2) linearity, candidates per window
    if oracle.rabin_fingerprint(b"\x80\0\0\0", L) != 0x1E3779BB:
        return False
    if oracle.rabin_fingerprint(b"\x01\0\0\0\0", L) != 0x3C6EF376:
        return False
    if oracle.rabin_fingerprint(b"\x12\x34\x56", L) != 0x123456:
        return False
    a, b = G.uniform_bytes(64, 21), G.uniform_bytes(64, 22)
    if oracle.rabin_fingerprint(a ^ b, L) != oracle.rabin_fingerprint(a, L) ^ oracle.rabin_fingerprint(b, L):
        return False
    small_r = G.uniform_bytes(1200, seed=23).tobytes()
    if oracle.window_candidates(small_r, 24, 3, 2, L=L, kind=oracle.WIN_RABIN).tolist() != \
            brute_window_cuts_with(small_r, 24, 3, 2, lambda w: oracle.rabin_fingerprint(w, L)):
        return False
    small = G.uniform_bytes(1500, seed=5).tobytes()
    if oracle.window_candidates(small, 20, 4, 5, L=L).tolist() != brute_window_cuts(small, 20, 4, 5):
        return False
    with open(os.path.join(HERE, "golden", "select_cases.json")) as f:
        for c in json.load(f)["cases"]:
            got = oracle.select(np.array(c["cands"], np.uint64), c["n"], c["min"], c["max"], L=L)
            if got.tolist() != c["ends"]:
                return False
    return True


def test_real_oracle_passes_pins():
    assert pins_pass(oracle.lib())


@pytest.mark.parametrize("fname,old,new", MUTANTS, ids=[f"{m[0]}:{i}" for i, m in enumerate(MUTANTS)])
def test_mutant_fails_pins(tmp_path, fname, old, new):
    L = build_mutant(tmp_path, fname, old, new)
    assert not pins_pass(L)
