"""FP64 CPU oracle of the short-characteristics radiation transport solve.

TEST INFRASTRUCTURE ONLY. Only tests/, __graft_entry__.smoke() and the
benchmark's CPU-baseline leg may import this package. The CUDA library never
uses it and shares no code with it.

The arithmetic lives in rts_oracle.c (plain C, IEEE double); this module only
marshals numpy arrays through ctypes.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from .build import build_oracle

BC_ZERO, BC_EQUAL_S, BC_EXPLICIT = 0, 1, 2
OK, EINVAL, ENOMEM, ENOCONV = 0, 1, 2, 5

_lib = None


class _Problem(C.Structure):
    _fields_ = [
        ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
        ("dx", C.c_double), ("dy", C.c_double), ("dz", C.c_double),
        ("nbands", C.c_int), ("ndir", C.c_int),
        ("n", C.POINTER(C.c_double)), ("w", C.POINTER(C.c_double)),
        ("tau_switch", C.c_double), ("wrap_tol", C.c_double), ("max_wrap_iters", C.c_int),
        ("bottom_kind", C.c_int), ("top_kind", C.c_int),
        ("bottom_I", C.POINTER(C.c_double)), ("top_I", C.POINTER(C.c_double)),
    ]


class DirGeom(C.Structure):
    _fields_ = [
        ("axis", C.c_int), ("sa", C.c_int), ("b1", C.c_int), ("b2", C.c_int),
        ("s1", C.c_int), ("s2", C.c_int), ("ds", C.c_double), ("d1", C.c_double),
        ("d2", C.c_double), ("beta", C.c_double * 4), ("up", C.c_int),
    ]


def lib():
    global _lib
    if _lib is None:
        path = build_oracle()
        L = C.CDLL(path)
        dp = C.POINTER(C.c_double)
        ip = C.POINTER(C.c_int)
        L.orc_a4_quadrature.argtypes = [dp, dp]
        L.orc_direction_geometry.argtypes = [C.POINTER(_Problem), C.c_int, C.POINTER(DirGeom)]
        L.orc_segment_weights.argtypes = [C.c_double, dp, dp, dp]
        L.orc_sweep_direction.argtypes = [C.POINTER(_Problem), C.c_int, C.c_int, dp, dp, dp, ip]
        L.orc_divergence.argtypes = [C.c_int, C.c_int, C.c_int, C.c_double, C.c_double, C.c_double, dp, dp]
        L.orc_solve.argtypes = [C.POINTER(_Problem), dp, dp, dp, dp, dp, dp, dp, dp, dp, dp, ip, C.c_int]
        L.orc_adjoint.argtypes = [C.POINTER(_Problem), dp, dp, dp, dp, dp, dp, dp, dp, C.c_int]
        for f in ("orc_direction_geometry", "orc_sweep_direction", "orc_solve", "orc_adjoint"):
            getattr(L, f).restype = C.c_int
        _lib = L
    return _lib


def _p(a):
    if a is None:
        return C.POINTER(C.c_double)()
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(C.POINTER(C.c_double))


def a4_quadrature():
    """Default 24-direction set: (n [24,3], w [24])."""
    n = np.zeros((24, 3))
    w = np.zeros(24)
    lib().orc_a4_quadrature(_p(n), _p(w))
    return n, w


class OracleError(RuntimeError):
    def __init__(self, code, what):
        super().__init__(f"oracle {what} failed with status {code}")
        self.code = code


class Problem:
    """Grid, quadrature, boundary conditions and options of one solve."""

    def __init__(self, nx, ny, nz, nbands=1, dx=1.0, dy=1.0, dz=1.0, n=None, w=None,
                 tau_switch=0.1, wrap_tol=1e-15, max_wrap_iters=200,
                 bottom=BC_EQUAL_S, top=BC_ZERO, bottom_I=None, top_I=None):
        if n is None:
            n, w = a4_quadrature()
        self.n = np.ascontiguousarray(n, dtype=np.float64).reshape(-1, 3)
        self.w = np.ascontiguousarray(w, dtype=np.float64).reshape(-1)
        self.nx, self.ny, self.nz, self.nbands = nx, ny, nz, nbands
        self.dx, self.dy, self.dz = dx, dy, dz
        self.tau_switch, self.wrap_tol, self.max_wrap_iters = tau_switch, wrap_tol, max_wrap_iters
        self.bottom, self.top = bottom, top
        self.bottom_I = None if bottom_I is None else np.ascontiguousarray(bottom_I, dtype=np.float64)
        self.top_I = None if top_I is None else np.ascontiguousarray(top_I, dtype=np.float64)

    @property
    def ndir(self):
        return self.n.shape[0]

    @property
    def nup(self):
        return int((self.n[:, 2] > 0).sum())

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx)

    def _c(self):
        s = _Problem()
        s.nx, s.ny, s.nz = self.nx, self.ny, self.nz
        s.dx, s.dy, s.dz = self.dx, self.dy, self.dz
        s.nbands, s.ndir = self.nbands, self.ndir
        s.n, s.w = _p(self.n), _p(self.w)
        s.tau_switch, s.wrap_tol, s.max_wrap_iters = self.tau_switch, self.wrap_tol, self.max_wrap_iters
        s.bottom_kind, s.top_kind = self.bottom, self.top
        s.bottom_I, s.top_I = _p(self.bottom_I), _p(self.top_I)
        return s

    # -- single pieces -------------------------------------------------------
    def geometry(self, d):
        g = DirGeom()
        rc = lib().orc_direction_geometry(C.byref(self._c()), d, C.byref(g))
        if rc:
            raise OracleError(rc, "geometry")
        return g

    def sweep(self, band, d, chi_b, S_b):
        """Intensity of direction d, band index `band` ([nz,ny,nx]) and wrap count."""
        chi_b = np.ascontiguousarray(chi_b, dtype=np.float64)
        S_b = np.ascontiguousarray(S_b, dtype=np.float64)
        I = np.zeros(self.shape)
        it = C.c_int(0)
        rc = lib().orc_sweep_direction(C.byref(self._c()), band, d, _p(chi_b), _p(S_b), _p(I), C.byref(it))
        if rc:
            raise OracleError(rc, "sweep")
        return I, it.value

    # -- whole solve -----------------------------------------------------------
    def solve(self, chi, S, debug=False, nthreads=1):
        """Forward solve. chi, S: [B,nz,ny,nx] float64.

        Returns dict with I_top [B,nup,ny,nx], J, Q [nz,ny,nx], F [3,nz,ny,nx],
        wrap_iters [B,ndir]; with debug also Jb, Fb, QJb, QFb per band."""
        chi = np.ascontiguousarray(chi, dtype=np.float64)
        S = np.ascontiguousarray(S, dtype=np.float64)
        B = self.nbands
        assert chi.shape == (B,) + self.shape and S.shape == chi.shape
        out = dict(
            I_top=np.zeros((B, self.nup, self.ny, self.nx)),
            J=np.zeros(self.shape), F=np.zeros((3,) + self.shape), Q=np.zeros(self.shape),
        )
        if debug:
            out.update(Jb=np.zeros((B,) + self.shape), Fb=np.zeros((B, 3) + self.shape),
                       QJb=np.zeros((B,) + self.shape), QFb=np.zeros((B,) + self.shape))
        its = np.zeros((B, self.ndir), dtype=np.int32)
        rc = lib().orc_solve(
            C.byref(self._c()), _p(chi), _p(S), _p(out["I_top"]), _p(out["J"]), _p(out["F"]), _p(out["Q"]),
            _p(out.get("Jb")), _p(out.get("Fb")), _p(out.get("QJb")), _p(out.get("QFb")),
            its.ctypes.data_as(C.POINTER(C.c_int)), int(nthreads))
        if rc:
            raise OracleError(rc, "solve")
        out["wrap_iters"] = its
        return out

    def adjoint(self, chi, S, gI_top=None, gJ=None, gF=None, gQ=None, nthreads=1):
        """Gradients (g_logchi, g_S) [B,nz,ny,nx] of <g,outputs>."""
        chi = np.ascontiguousarray(chi, dtype=np.float64)
        S = np.ascontiguousarray(S, dtype=np.float64)
        f = lambda a: None if a is None else np.ascontiguousarray(a, dtype=np.float64)  # noqa: E731
        g_logchi = np.zeros_like(chi)
        g_S = np.zeros_like(S)
        rc = lib().orc_adjoint(C.byref(self._c()), _p(chi), _p(S), _p(f(gI_top)), _p(f(gJ)), _p(f(gF)),
                               _p(f(gQ)), _p(g_logchi), _p(g_S), int(nthreads))
        if rc:
            raise OracleError(rc, "adjoint")
        return g_logchi, g_S


def segment_weights(x):
    e, wu, wp = C.c_double(), C.c_double(), C.c_double()
    lib().orc_segment_weights(float(x), C.byref(e), C.byref(wu), C.byref(wp))
    return e.value, wu.value, wp.value


def neg_divergence(F, dx=1.0, dy=1.0, dz=1.0):
    """-div F for F [3,nz,ny,nx] with the oracle's stencil."""
    F = np.ascontiguousarray(F, dtype=np.float64)
    _, nz, ny, nx = F.shape
    out = np.zeros((nz, ny, nx))
    lib().orc_divergence(nx, ny, nz, dx, dy, dz, _p(F), _p(out))
    return out


def default_threads():
    """Threads for the oracle's OpenMP loop (capped: each holds one N-sized array)."""
    return max(1, min(32, os.cpu_count() or 1))
