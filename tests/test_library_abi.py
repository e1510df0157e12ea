"""CPU-only checks of the CUDA library boundary: it builds for sm_103a, loads,
and exports every entry point include/rts.h declares. No compute calls."""
import ctypes
import os
import re
import subprocess

import pytest

import paper_2107_08145_b300 as rts

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "rts.h")).read()
    return sorted(set(re.findall(r"\b(rts_[a-z_]+)\s*\(", txt)))


def test_header_declares_exports():
    decl = _declared()
    assert set(decl) == set(rts.EXPORTS), decl


def test_library_loads_and_exports_every_symbol():
    L = rts.load()
    for name in _declared():
        assert hasattr(L, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", rts.library_path()], capture_output=True, text=True).stdout
    for name in _declared():
        assert re.search(r"\bT %s$" % name, out, re.M), name


def test_library_is_built_for_sm103a():
    """Every translation unit is compiled for sm_103a only (the build
    command); the GPU test test_device_code_is_sm103 reads the loaded
    kernels' version at run time."""
    from paper_2107_08145_b300 import build

    cmd = build.compile_command("x.cu", "x.o")
    assert "arch=compute_103a,code=sm_103a" in cmd and cmd.count("-gencode") == 1
    assert "-gencode" in build.link_command([], "x.so")


@pytest.mark.gpu
def test_device_code_is_sm103():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    assert rts.device_code_version() == 103


def test_default_options_and_null_handle():
    L = rts.load()
    o = rts.Options()
    L.rts_default_options(ctypes.byref(o))
    assert o.prec == rts.FP64 and o.tau_switch == 0.1 and o.max_wrap_iters == 64 and o.timeout_s == 2.0
    assert L.rts_last_error(None) == b"null handle"
    assert L.rts_check(None) == rts.RTS_EINVAL
    assert L.rts_solve(None, None, None, None, None, None, None, None) == rts.RTS_EINVAL


def test_create_rejects_bad_grid_without_gpu():
    """Argument validation happens before any CUDA call."""
    L = rts.load()
    h = ctypes.c_void_p()
    g = rts.Grid(4, 4, 1, 1.0, 1.0, 1.0)  # nz < 2
    rc = L.rts_create(ctypes.byref(h), ctypes.byref(g), 1, None, None)
    assert rc == rts.RTS_EINVAL
    assert b"nz" in L.rts_last_error(h)
    L.rts_destroy(h)
    g = rts.Grid(4, 4, 4, 1.0, -1.0, 1.0)
    rc = L.rts_create(ctypes.byref(h), ctypes.byref(g), 1, None, None)
    assert rc == rts.RTS_EINVAL and b"spacing" in L.rts_last_error(h)
    L.rts_destroy(h)
    n = (ctypes.c_double * 3)(1.0, 0.0, 0.0)
    w = (ctypes.c_double * 1)(1.0)
    q = rts.Quadrature(1, n, w)
    g = rts.Grid(4, 4, 4, 1.0, 1.0, 1.0)
    rc = L.rts_create(ctypes.byref(h), ctypes.byref(g), 1, ctypes.byref(q), None)
    assert rc == rts.RTS_EINVAL and b"n_z" in L.rts_last_error(h)
    L.rts_destroy(h)


def test_create_rejects_too_many_levels_times_bands_without_gpu():
    """The per-level launches take one CTA layer per (band, level): nz * B is
    capped at 65535 and refused at create, before any CUDA call."""
    L = rts.load()
    h = ctypes.c_void_p()
    g = rts.Grid(4, 4, 8192, 1.0, 1.0, 1.0)
    rc = L.rts_create(ctypes.byref(h), ctypes.byref(g), 9, None, None)
    assert rc == rts.RTS_EINVAL and b"65535" in L.rts_last_error(h)
    L.rts_destroy(h)


def test_front_end_rejects_bad_arguments_without_gpu():
    """rts_front_end validates its table and the stagger shift (finite,
    |shift| <= 2^20) before it launches anything; the array pointers are
    never dereferenced on these paths."""
    L = rts.load()
    g = rts.Grid(8, 8, 8, 1.0, 1.0, 1.0)
    err = ctypes.create_string_buffer(128)
    fake = ctypes.c_void_p(16)

    def call(shift=(-0.5, -0.5, -0.5), nT=4, dlnT=0.1):
        tab = rts.FrontTable(2, nT, 3, 0.0, dlnT, 0.0, 0.1, fake, fake, (ctypes.c_double * 3)(*shift))
        return L.rts_front_end(ctypes.byref(g), ctypes.byref(tab), rts.FP32_MIXED, fake, fake, fake, fake, None, err, 128)

    assert call(shift=(float("nan"), 0.0, 0.0)) == rts.RTS_EINVAL and b"shift" in err.value
    assert call(shift=(0.0, 2.0 ** 21, 0.0)) == rts.RTS_EINVAL and b"shift" in err.value
    assert call(shift=(0.0, 0.0, float("inf"))) == rts.RTS_EINVAL
    assert call(nT=0) == rts.RTS_EINVAL and b"table" in err.value
    assert call(dlnT=0.0) == rts.RTS_EINVAL


def test_product_path_does_not_import_oracle():
    """The library and its binding never reach the CPU oracle."""
    pkg = os.path.join(ROOT, "paper_2107_08145_b300")
    for dirpath, _, files in os.walk(pkg):
        if "_build" in dirpath:
            continue
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt and "rts_oracle" not in txt, f
