"""Builds the FP64 CPU oracle (plain C, gcc, OpenMP when available) in-tree.

TEST INFRASTRUCTURE: the oracle is the reference the CUDA library is checked against.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "gbd_oracle.c")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "liboracle.so")


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile oracle/gbd_oracle.c into oracle/_build/liboracle.so; returns its path."""
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    tmp = LIB + f".tmp{os.getpid()}"
    base = ["gcc", "-std=gnu11", "-O2", "-fPIC", "-shared", "-o", tmp, SRC, "-lm"]
    for extra in (["-fopenmp"], []):
        cmd = base[:2] + extra + base[2:]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if verbose:
            print(" ".join(cmd), r.stdout, r.stderr, file=sys.stderr)
        if r.returncode == 0:
            os.replace(tmp, LIB)
            return LIB
    raise RuntimeError(f"oracle build failed:\n{r.stderr}")


if __name__ == "__main__":
    print(build(force=True, verbose=True))
