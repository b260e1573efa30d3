"""Build libhashgpu.so in-tree with nvcc for sm_103a (B300)."""
from __future__ import annotations

import concurrent.futures as cf
import os
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(PKG, "libhashgpu.so")
# the benchmark's integer-pipe probe: its own library, not part of the hashing library
PROBE_SRC = os.path.join(PKG, "bench_probe", "hg_probe.cu")
PROBE_LIB = os.path.join(PKG, "bench_probe", "libhgprobe.so")
BUILD = os.path.join(PKG, "_build")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O2,-Wall",
              "-I", INCLUDE, "-I", CSRC, *ARCH]


def sources() -> list[str]:
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))


def headers() -> list[str]:
    hs = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    return hs + [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE) if f.endswith(".h")]


# The debug variant (HG_DEBUG): kernels check the indexes of their global accesses
# and report HG_EBOUNDS instead of touching memory out of range.
LIB_DEBUG = os.path.join(PKG, "libhashgpu_debug.so")
BUILD_DEBUG = os.path.join(PKG, "_build_debug")


def _compile(src: str, verbose: bool, debug: bool = False) -> str:
    obj = os.path.join(BUILD_DEBUG if debug else BUILD, os.path.basename(src) + ".o")
    newest = max(os.path.getmtime(p) for p in [src, *headers(), __file__])
    if os.path.exists(obj) and os.path.getmtime(obj) >= newest:
        return obj
    cmd = ["nvcc", *NVCC_FLAGS, *(["-DHG_DEBUG"] if debug else []),
           *(["-Xptxas", "-v"] if verbose else []), "-c", src, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
    if verbose:
        sys.stderr.write(r.stderr)
    return obj


def build(force: bool = False, verbose: bool = False, debug: bool = False) -> str:
    bdir, lib = (BUILD_DEBUG, LIB_DEBUG) if debug else (BUILD, LIB)
    os.makedirs(bdir, exist_ok=True)
    if force:
        for f in os.listdir(bdir):
            os.remove(os.path.join(bdir, f))
    with cf.ThreadPoolExecutor(max_workers=os.cpu_count() or 4) as ex:
        objs = list(ex.map(lambda s: _compile(s, verbose, debug), sources()))
    if not os.path.exists(lib) or any(os.path.getmtime(o) > os.path.getmtime(lib) for o in objs):
        tmp = lib + ".tmp"
        cmd = ["nvcc", "-shared", *ARCH, "-o", tmp, *objs, "-cudart", "static"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, lib)
    return lib


def build_probe(force: bool = False) -> str:
    """Build the benchmark's probe library (libhgprobe.so) beside its source."""
    if force or not os.path.exists(PROBE_LIB) or os.path.getmtime(PROBE_LIB) < max(
            os.path.getmtime(PROBE_SRC), os.path.getmtime(__file__)):
        tmp = PROBE_LIB + ".tmp"
        cmd = ["nvcc", "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", *ARCH, "-shared",
               PROBE_SRC, "-o", tmp, "-cudart", "static"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, PROBE_LIB)
    return PROBE_LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
    print(build(force="--force" in sys.argv, debug=True))
    print(build_probe(force="--force" in sys.argv))
