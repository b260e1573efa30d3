"""Compile the C oracle into oracle/liboracle.so (test infrastructure only)."""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SOURCES = ["md5.c", "sha1.c", "direct.c", "cdc.c", "rabin.c"]
LIB = os.path.join(HERE, "liboracle.so")


def build(force: bool = False, out: str = LIB, cflags=None) -> str:
    srcs = [os.path.join(HERE, s) for s in SOURCES]
    deps = srcs + [os.path.join(HERE, "hg_oracle.h")]
    if not force and os.path.exists(out) and all(
            os.path.getmtime(out) >= os.path.getmtime(d) for d in deps):
        return out
    cmd = ["gcc", "-std=c99", "-O2", "-fPIC", "-shared", "-pthread",
           "-D_POSIX_C_SOURCE=200809L", "-Wall", "-Wextra", "-Werror",
           *(cflags or []), "-o", out, *srcs, "-lm"]
    subprocess.run(cmd, check=True)
    return out


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
