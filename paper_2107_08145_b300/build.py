"""Build the CUDA library librts.so for sm_103a (B300) in-tree.

    python -m paper_2107_08145_b300.build [--force] [--ptxas-v]

The library is a plain C ABI (include/rts.h) compiled with nvcc; the Python
package loads it with ctypes. Every csrc/*.cu file is one translation unit
(the host API and the light kernels in rts_api.cu, the sweep instantiations
in files of their own); they are compiled in parallel and linked into one
shared object.
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
CSRC = os.path.join(HERE, "csrc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC"]


def _units():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _inputs():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu*")) + glob.glob(os.path.join(CSRC, "*.h")) +
                  [os.path.join(ROOT, "include", "rts.h")])


def compile_command(src: str, out: str, extra=()):
    return ["nvcc"] + ARCH + FLAGS + ["-I", os.path.join(ROOT, "include"), "-c", "-o", out, src] + list(extra)


def link_command(objs, out: str):
    return ["nvcc"] + ARCH + ["-shared", "-o", out] + list(objs)


def source_hash() -> str:
    """Hash of every source the library is built from (and of the commands)."""
    h = hashlib.sha256(" ".join(compile_command("src", "out") + link_command([], "out")).encode())
    for f in _inputs():
        h.update(os.path.relpath(f, ROOT).encode())
        h.update(open(f, "rb").read())
    return h.hexdigest()


def _deps(src: str, seen=None):
    """The file and every local header it includes, recursively."""
    import re
    seen = set() if seen is None else seen
    if src in seen or not os.path.exists(src):
        return seen
    seen.add(src)
    for inc in re.findall(r'^#include "([^"]+)"', open(src).read(), re.M):
        for d in (os.path.dirname(src), os.path.join(ROOT, "include")):
            f = os.path.join(d, inc)
            if os.path.exists(f):
                _deps(f, seen)
                break
    return seen


def _obj_hash(src: str, extra) -> str:
    h = hashlib.sha256(" ".join(compile_command(src, "out", extra)).encode())
    for f in sorted(_deps(src)):
        h.update(os.path.relpath(f, ROOT).encode())
        h.update(open(f, "rb").read())
    return h.hexdigest()


def _stale() -> bool:
    if not os.path.exists(LIB) or not os.path.exists(LIB + ".srchash"):
        return True
    return open(LIB + ".srchash").read().strip() != source_hash()


def build(force: bool = False, verbose_ptxas: bool = False) -> str:
    if not force and not _stale():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    digest = source_hash()
    extra = ["-Xptxas", "-v"] if verbose_ptxas else []
    objs, procs = [], []
    for src in _units():
        obj = os.path.join(BUILD, os.path.splitext(os.path.basename(src))[0] + ".o")
        objs.append(obj)
        oh = _obj_hash(src, extra)
        # an object is rebuilt only when its source, its headers or the command changed
        if not force and os.path.exists(obj) and os.path.exists(obj + ".hash") and \
                open(obj + ".hash").read().strip() == oh:
            continue
        procs.append((src, obj, oh, subprocess.Popen(compile_command(src, obj, extra))))
    failed = [src for src, _, _, p in procs if p.wait() != 0]
    if failed:
        raise RuntimeError("nvcc failed for " + ", ".join(os.path.basename(f) for f in failed))
    for _, obj, oh, _ in procs:
        with open(obj + ".hash", "w") as f:
            f.write(oh + "\n")
    tmp = LIB + ".tmp.%d" % os.getpid()
    subprocess.run(link_command(objs, tmp), check=True)
    os.replace(tmp, LIB)
    with open(LIB + ".srchash", "w") as f:
        f.write(digest + "\n")
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose_ptxas="--ptxas-v" in sys.argv))
