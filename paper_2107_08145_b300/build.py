"""Build the CUDA library librts.so for sm_103a (B300) in-tree.

    python -m paper_2107_08145_b300.build [--force] [--ptxas-v]

The library is a plain C ABI (include/rts.h) compiled with nvcc; the Python
package loads it with ctypes.
"""
from __future__ import annotations

import glob
import hashlib
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "librts.so")
SRC = os.path.join(HERE, "csrc", "rts_api.cu")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _inputs():
    return sorted(glob.glob(os.path.join(HERE, "csrc", "*.cu*")) + [os.path.join(ROOT, "include", "rts.h")])


def source_hash() -> str:
    """Hash of every source the library is built from (and of the command)."""
    h = hashlib.sha256(" ".join(nvcc_command("out")).encode())
    for f in _inputs():
        h.update(f.encode())
        h.update(open(f, "rb").read())
    return h.hexdigest()


def _stale() -> bool:
    if not os.path.exists(LIB) or not os.path.exists(LIB + ".srchash"):
        return True
    return open(LIB + ".srchash").read().strip() != source_hash()


def nvcc_command(out: str, extra=()):
    return (["nvcc"] + ARCH + ["-O3", "-lineinfo", "-std=c++17", "-shared", "-Xcompiler", "-fPIC",
                               "-I", os.path.join(ROOT, "include"), "-o", out, SRC] + list(extra))


def build(force: bool = False, verbose_ptxas: bool = False) -> str:
    if not force and not _stale():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    tmp = LIB + ".tmp.%d" % os.getpid()
    extra = ["-Xptxas", "-v"] if verbose_ptxas else []
    digest = source_hash()
    subprocess.run(nvcc_command(tmp, extra), check=True)
    os.replace(tmp, LIB)
    with open(LIB + ".srchash", "w") as f:
        f.write(digest + "\n")
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose_ptxas="--ptxas-v" in sys.argv))
