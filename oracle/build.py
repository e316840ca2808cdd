"""Compile the CPU oracle (plain C, gcc) into oracle/_build/liborc.so.

Test infrastructure: the CUDA library does not use this.  Flags keep the
arithmetic plain on every host: no fast-math and no contraction of a*b+c
into fused multiply-adds, so x86-64 and aarch64 round identically.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "mlb_oracle.c")
BODY = os.path.join(HERE, "mlb_oracle_body.h")
OUT_DIR = os.path.join(HERE, "_build")
OUT = os.path.join(OUT_DIR, "liborc.so")

CFLAGS = ["-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
          "-fPIC", "-shared", "-Wall", "-Wno-unused-function"]


def compile_oracle(src: str = SRC, out: str = OUT, include_dir: str = HERE,
                   defines: dict | None = None) -> str:
    os.makedirs(os.path.dirname(out), exist_ok=True)
    cmd = ["gcc", *CFLAGS, "-I", include_dir]
    for k, v in (defines or {}).items():
        cmd.append(f"-D{k}={v}")
    cmd += [src, "-o", out + ".tmp", "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(out + ".tmp", out)
    return out


def build(force: bool = False) -> str:
    """Build liborc.so if missing or older than its sources."""
    if not force and os.path.exists(OUT):
        t = os.path.getmtime(OUT)
        if t >= os.path.getmtime(SRC) and t >= os.path.getmtime(BODY):
            return OUT
    return compile_oracle()


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
