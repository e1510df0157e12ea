"""Compile the C oracle into oracle/_build/librts_oracle.so (gcc, OpenMP).

Test infrastructure: the oracle is built so that tests, the smoke check and
the benchmark's CPU-baseline leg can call it; nothing in the product library
links against it.
"""
from __future__ import annotations

import hashlib
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "librts_oracle.so")
SRC = [os.path.join(HERE, "rts_oracle.c")]
HDR = [os.path.join(HERE, "rts_oracle.h")]


def _digest() -> str:
    h = hashlib.sha256()
    for f in SRC + HDR:
        h.update(open(f, "rb").read())
    return h.hexdigest()


def _stale() -> bool:
    if not os.path.exists(LIB) or not os.path.exists(LIB + ".srchash"):
        return True
    return open(LIB + ".srchash").read().strip() != _digest()


def build_oracle(force: bool = False) -> str:
    """Build the oracle shared library if missing or out of date; return its path."""
    if not force and not _stale():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    tmp = LIB + ".tmp.%d" % os.getpid()
    # -O2 without -ffast-math: IEEE double arithmetic in program order.
    cmd = ["gcc", "-std=c11", "-O2", "-fopenmp", "-fPIC", "-shared", "-Wall", "-Wextra",
           "-o", tmp] + SRC + ["-lm"]
    digest = _digest()
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    with open(LIB + ".srchash", "w") as f:
        f.write(digest + "\n")
    return LIB


if __name__ == "__main__":
    print(build_oracle(force=True))
