"""Compile the CPU oracle (plain C, gcc) into oracle/_build/liborc.so and
its multi-core build (OpenMP, fixed-block reductions) liborc_par.so.

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
OUT_PAR = os.path.join(OUT_DIR, "liborc_par.so")

CFLAGS = ["-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
          "-fPIC", "-shared", "-Wall", "-Wno-unused-function", "-Wno-unknown-pragmas"]


def compile_oracle(src: str = SRC, out: str = OUT, include_dir: str = HERE,
                   defines: dict | None = None, openmp: bool = False) -> str:
    os.makedirs(os.path.dirname(out), exist_ok=True)
    cmd = ["gcc", *CFLAGS, "-I", include_dir]
    if openmp:
        cmd.append("-fopenmp")
    for k, v in (defines or {}).items():
        cmd.append(f"-D{k}={v}")
    cmd += [src, "-o", out + ".tmp", "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(out + ".tmp", out)
    return out


def _fresh(out: str) -> bool:
    if not os.path.exists(out):
        return False
    t = os.path.getmtime(out)
    return t >= os.path.getmtime(SRC) and t >= os.path.getmtime(BODY)


def build(force: bool = False) -> str:
    """Build liborc.so (sequential) and liborc_par.so (multi-core build,
    fixed-block reductions) if missing or older than their sources."""
    if force or not _fresh(OUT):
        compile_oracle()
    if force or not _fresh(OUT_PAR):
        compile_oracle(out=OUT_PAR, defines={"ORC_PAR": 1}, openmp=True)
    return OUT


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
