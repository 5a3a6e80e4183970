"""Compile the C part of the oracle (test infrastructure) with gcc.

The flags matter: -ffp-contract=off forbids fused multiply-add contraction and
no -ffast-math is given, so every float operation rounds on its own exactly as
the oracle's fixed float sequences specify, on x86-64 and on aarch64 alike.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "pt2d_oracle.c")
LIB = os.path.join(HERE, "liboracle_pt2d.so")

CFLAGS = ["-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
          "-Wall", "-Wextra"]


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", *CFLAGS, SRC, "-o", tmp, "-lm"]
    if verbose:
        print(" ".join(cmd), file=sys.stderr)
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


def compile_variant(source_text: str, out_path: str) -> str:
    """Compile a modified copy of the oracle source (used to plant a mistake
    on purpose and check that the pinning tests catch it)."""
    src = out_path + ".c"
    with open(src, "w") as fh:
        fh.write(source_text)
    subprocess.run(["gcc", *CFLAGS, src, "-o", out_path, "-lm"], check=True)
    return out_path


if __name__ == "__main__":
    print(build(force=True, verbose=True))
