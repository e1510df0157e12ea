"""B300-native short-characteristics radiation transport solver (RTS).

A thin ctypes binding over the C ABI in include/rts.h (librts.so, built from
csrc/ for sm_103a). Every step of the solve runs in the library's CUDA
kernels; this module only marshals torch tensors (device memory, streams) into
the ABI. If the library cannot be loaded, importing the solver raises: there
is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

from .build import LIB, build as _build

RTS_OK, RTS_EINVAL, RTS_ENOMEM, RTS_ECUDA, RTS_ETIMEOUT, RTS_ENOCONV, RTS_ENONFINITE = range(7)
FP64, FP32_MIXED, FP32_COMPENSATED = 0, 1, 2
BC_ZERO, BC_EQUAL_S, BC_EXPLICIT = 0, 1, 2
FLAG_HOST_IO = 1
FLAG_TIMING = 2
FLAG_ADJOINT = 4
FLAG_HOST_IO_ASYNC = 8
FLAG_LOG_CHI = 16
FLAG_SCATTER = 32

_PREC = {"fp64": FP64, "fp32": FP32_MIXED, "fp32_mixed": FP32_MIXED, "fp32_compensated": FP32_COMPENSATED}
_BC = {"zero": BC_ZERO, "equal_s": BC_EQUAL_S}
SWEEP_AUTO, SWEEP_SHARED, SWEEP_REGISTER = 0, 1, 2
_SWEEP = {"auto": SWEEP_AUTO, "shared": SWEEP_SHARED, "register": SWEEP_REGISTER}


class Grid(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("dx", C.c_double), ("dy", C.c_double), ("dz", C.c_double)]


class Quadrature(C.Structure):
    _fields_ = [("ndir", C.c_int), ("n", C.POINTER(C.c_double)), ("w", C.POINTER(C.c_double))]


class Options(C.Structure):
    _fields_ = [("prec", C.c_int), ("tau_switch", C.c_double), ("wrap_tol", C.c_double),
                ("max_wrap_iters", C.c_int), ("tile_rows", C.c_int), ("threads", C.c_int),
                ("flags", C.c_int), ("timeout_s", C.c_double), ("stream", C.c_void_p),
                ("adjoint_chunk_bands", C.c_int), ("sweep_kernel", C.c_int)]


class Stats(C.Structure):
    _fields_ = [("n_units", C.c_int), ("n_tiles", C.c_int), ("max_warmup_steps", C.c_int),
                ("mean_warmup_steps", C.c_double), ("device_status", C.c_int), ("grid", C.c_int),
                ("tile_rows", C.c_int), ("kernels_per_solve", C.c_int), ("timed_solves", C.c_int),
                ("ms_transpose", C.c_float), ("ms_sweep", C.c_float), ("ms_reduce", C.c_float),
                ("ms_qstep", C.c_float), ("timed_adjoints", C.c_int), ("ms_adjoint", C.c_float * 4),
                ("sweep_kernel", C.c_int), ("adjoint_chunk_bands", C.c_int)]


class FrontTable(C.Structure):
    _fields_ = [("nbands", C.c_int), ("nT", C.c_int), ("nR", C.c_int), ("lnT0", C.c_double), ("dlnT", C.c_double),
                ("lnR0", C.c_double), ("dlnR", C.c_double), ("ln_kappa", C.c_void_p), ("ln_B", C.c_void_p),
                ("shift", C.c_double * 3)]


class Boundary(C.Structure):
    _fields_ = [("bottom", C.c_int), ("top", C.c_int), ("bottom_I", C.c_void_p), ("top_I", C.c_void_p),
                ("wrap_seed", C.c_void_p), ("seed_in", C.c_int), ("seed_tol", C.c_double)]


_lib = None

# every symbol include/rts.h declares
EXPORTS = ("rts_default_options", "rts_create", "rts_solve", "rts_solve_host", "rts_check",
           "rts_get_stats", "rts_last_error", "rts_num_up", "rts_destroy", "rts_solve_noalloc", "rts_adjoint",
           "rts_create_batched", "rts_solve_batched", "rts_batched_layout", "rts_graph_create", "rts_graph_launch",
           "rts_graph_destroy", "rts_autotune", "rts_solve_host_async", "rts_host_wait", "rts_device_code_version",
           "rts_front_end", "rts_scatter_solve", "rts_wrap_seed_elems", "rts_create_decomposed",
           "rts_solve_decomposed", "rts_decomposed_last_error", "rts_destroy_decomposed")


def library_path() -> str:
    return LIB


def load(build_if_missing: bool = True):
    """Load librts.so (building it first if it is missing and nvcc exists)."""
    global _lib
    if _lib is not None:
        return _lib
    path = LIB
    if not os.path.exists(path):
        if not build_if_missing:
            raise ImportError(f"CUDA library {path} is missing; run python -m paper_2107_08145_b300.build")
        _build()
    L = C.CDLL(path)
    vp, dp = C.c_void_p, C.POINTER(C.c_double)
    L.rts_default_options.argtypes = [C.POINTER(Options)]
    L.rts_default_options.restype = None
    L.rts_create.argtypes = [C.POINTER(C.c_void_p), C.POINTER(Grid), C.c_int, C.POINTER(Quadrature), C.POINTER(Options)]
    L.rts_create.restype = C.c_int
    for f in ("rts_solve", "rts_solve_host", "rts_solve_host_async"):
        getattr(L, f).argtypes = [vp, vp, vp, C.POINTER(Boundary), vp, vp, vp, vp]
        getattr(L, f).restype = C.c_int
    L.rts_adjoint.argtypes = [vp, vp, vp, C.POINTER(Boundary), vp, vp, vp, vp, vp, vp]
    L.rts_adjoint.restype = C.c_int
    L.rts_create_batched.argtypes = [C.POINTER(C.c_void_p), C.c_int, C.POINTER(Grid), C.c_int,
                                     C.POINTER(Quadrature), C.POINTER(Options)]
    L.rts_create_batched.restype = C.c_int
    L.rts_solve_batched.argtypes = [vp, vp, vp, C.POINTER(Boundary), vp, vp, vp, vp]
    L.rts_solve_batched.restype = C.c_int
    ll = C.POINTER(C.c_longlong)
    L.rts_batched_layout.argtypes = [vp, C.c_int, ll, ll, ll, ll]
    L.rts_batched_layout.restype = C.c_int
    L.rts_graph_create.argtypes = [vp, vp, vp, C.POINTER(Boundary), vp, vp, vp, vp, C.POINTER(C.c_void_p)]
    L.rts_graph_create.restype = C.c_int
    L.rts_graph_launch.argtypes = [vp]
    L.rts_graph_launch.restype = C.c_int
    L.rts_graph_destroy.argtypes = [vp]
    L.rts_graph_destroy.restype = None
    L.rts_autotune.argtypes = [C.c_int, C.POINTER(Grid), C.c_int, C.POINTER(Quadrature), C.POINTER(Options), vp, vp,
                               C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int),
                               C.POINTER(C.c_float)]
    L.rts_autotune.restype = C.c_int
    L.rts_check.argtypes = [vp]
    L.rts_check.restype = C.c_int
    L.rts_host_wait.argtypes = [vp]
    L.rts_host_wait.restype = C.c_int
    L.rts_get_stats.argtypes = [vp, C.POINTER(Stats)]
    L.rts_get_stats.restype = C.c_int
    L.rts_last_error.argtypes = [vp]
    L.rts_last_error.restype = C.c_char_p
    L.rts_num_up.argtypes = [vp]
    L.rts_num_up.restype = C.c_int
    L.rts_device_code_version.argtypes = []
    L.rts_device_code_version.restype = C.c_int
    L.rts_front_end.argtypes = [C.POINTER(Grid), C.POINTER(FrontTable), C.c_int, vp, vp, vp, vp, vp, C.c_char_p,
                                C.c_size_t]
    L.rts_front_end.restype = C.c_int
    L.rts_scatter_solve.argtypes = [vp, vp, vp, vp, vp, C.POINTER(Boundary), C.c_int, C.c_double,
                                    C.POINTER(C.c_int), vp, vp, vp, vp]
    L.rts_scatter_solve.restype = C.c_int
    L.rts_wrap_seed_elems.argtypes = [vp]
    L.rts_wrap_seed_elems.restype = C.c_longlong
    L.rts_destroy.argtypes = [vp]
    L.rts_destroy.restype = None
    L.rts_solve_noalloc.argtypes = [C.POINTER(Grid), C.c_int, C.c_int, vp, vp, vp, vp, vp, vp, vp,
                                    C.c_char_p, C.c_size_t]
    L.rts_solve_noalloc.restype = C.c_int
    L.rts_create_decomposed.argtypes = [C.POINTER(C.c_void_p), C.POINTER(Grid), C.c_int, C.c_int,
                                        C.POINTER(Quadrature), C.POINTER(Options)]
    L.rts_create_decomposed.restype = C.c_int
    L.rts_solve_decomposed.argtypes = [vp, vp, vp, C.POINTER(Boundary), C.c_double, C.c_int, C.POINTER(C.c_int),
                                       vp, vp, vp, vp]
    L.rts_solve_decomposed.restype = C.c_int
    L.rts_decomposed_last_error.argtypes = [vp]
    L.rts_decomposed_last_error.restype = C.c_char_p
    L.rts_destroy_decomposed.argtypes = [vp]
    L.rts_destroy_decomposed.restype = None
    _ = dp
    _lib = L
    return L


class RTSError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"rts status {code}: {msg}")
        self.code = code


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _need(name, t, shape, dtype, device, contiguous=False):
    """t unchanged if it is a CUDA tensor of this shape and dtype on this
    device (and contiguous: arrays the library writes through their
    pointer); else ValueError. The library trusts its pointers' extents, so
    a short or misplaced array would be read or written out of bounds."""
    ok = (getattr(t, "is_cuda", False) and t.dtype == dtype and tuple(t.shape) == tuple(shape)
          and t.device == device and (not contiguous or t.is_contiguous()))
    if not ok:
        got = f"{getattr(t, 'dtype', type(t).__name__)} {tuple(getattr(t, 'shape', ()))} on {getattr(t, 'device', 'host')}"
        raise ValueError(f"{name} must be a {'contiguous ' if contiguous else ''}CUDA {dtype} tensor "
                         f"{tuple(shape)} on {device}, got {got}")
    return t


def _need_host(name, a, shape, dtype, writable=False):
    """The host-array form of _need: a C-contiguous numpy array of this shape
    and dtype (writable for outputs)."""
    import numpy as np

    ok = (isinstance(a, np.ndarray) and a.dtype == dtype and a.shape == tuple(shape) and a.flags.c_contiguous
          and (not writable or a.flags.writeable))
    if not ok:
        got = f"{getattr(a, 'dtype', type(a).__name__)} {tuple(getattr(a, 'shape', ()))}"
        raise ValueError(f"{name} must be a C-contiguous{' writable' if writable else ''} {np.dtype(dtype)} array "
                         f"{tuple(shape)}, got {got}")
    return a


class Solver:
    """One grid + band count; owns the device scratch of the CUDA library.

    precision: 'fp64', 'fp32' (FP32 sweep, FP64 accumulation and Q step) or
    'fp32_compensated' (FP32 sweep, double-float accumulation and Q step).
    """

    def __init__(self, nx, ny, nz, nbands=1, dx=1.0, dy=1.0, dz=1.0, precision="fp64", n=None, w=None,
                 tau_switch=0.1, wrap_tol=0.0, max_wrap_iters=64, tile_rows=0, timeout_s=2.0,
                 host_io=False, timing=False, stream=None, adjoint=False, adjoint_chunk_bands=0,
                 host_io_async=False, sweep_kernel="auto", log_chi=False, scatter=False):
        import torch

        L = load()
        self.torch = torch
        self.device = torch.device("cuda", torch.cuda.current_device())  # the device rts_create works on
        self.nx, self.ny, self.nz, self.nbands = nx, ny, nz, nbands
        self.ndir = 24 if n is None else len(w)
        self.precision = precision
        self.prec = _PREC[precision]
        self.dtype = torch.float64 if self.prec == FP64 else torch.float32
        o = Options()
        L.rts_default_options(C.byref(o))
        o.prec = self.prec
        o.tau_switch = tau_switch
        o.wrap_tol = wrap_tol
        o.max_wrap_iters = max_wrap_iters
        o.tile_rows = tile_rows
        o.timeout_s = timeout_s
        o.flags = ((FLAG_HOST_IO if host_io else 0) | (FLAG_TIMING if timing else 0) | (FLAG_ADJOINT if adjoint else 0)
                   | (FLAG_HOST_IO_ASYNC if host_io_async else 0) | (FLAG_LOG_CHI if log_chi else 0)
                   | (FLAG_SCATTER if scatter else 0))
        self.log_chi = log_chi
        o.adjoint_chunk_bands = adjoint_chunk_bands
        o.sweep_kernel = _SWEEP[sweep_kernel]
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        o.stream = C.c_void_p(stream.cuda_stream)
        g = Grid(nx, ny, nz, dx, dy, dz)
        q = None
        if n is not None:
            import numpy as np

            self._n = np.ascontiguousarray(n, dtype=np.float64).reshape(-1, 3)
            self._w = np.ascontiguousarray(w, dtype=np.float64).reshape(-1)
            q = Quadrature(len(self._w), self._n.ctypes.data_as(C.POINTER(C.c_double)),
                           self._w.ctypes.data_as(C.POINTER(C.c_double)))
        h = C.c_void_p()
        rc = L.rts_create(C.byref(h), C.byref(g), nbands, C.byref(q) if q is not None else None, C.byref(o))
        self._h = h
        self._L = L
        if rc != RTS_OK:
            msg = L.rts_last_error(h).decode() if h.value else "rts_create failed"
            L.rts_destroy(h)
            self._h = C.c_void_p()
            raise RTSError(rc, msg)
        self.n_up = L.rts_num_up(h)

    def __del__(self):
        try:
            if self._h and self._h.value:
                self._L.rts_destroy(self._h)
                self._h = C.c_void_p()
        except Exception:
            pass

    def _err(self, rc):
        if rc != RTS_OK:
            raise RTSError(rc, self._L.rts_last_error(self._h).decode())

    def _bc(self, bottom, top):
        b = Boundary()
        keep = []
        for side, v in (("bottom", bottom), ("top", top)):
            if isinstance(v, str):
                setattr(b, side, _BC[v])
            else:
                nr = self.n_up if side == "bottom" else self.ndir - self.n_up
                t = _need(side, v, (self.nbands, nr, self.ny, self.nx), self.dtype, self.device).contiguous()
                keep.append(t)
                setattr(b, side, BC_EXPLICIT)
                setattr(b, side + "_I", t.data_ptr())
        return b, keep

    def _inputs(self, *named):
        """(name, tensor) pairs of [B, nz, ny, nx] inputs -> contiguous tensors."""
        shape = (self.nbands, self.nz, self.ny, self.nx)
        return [_need(n, t, shape, self.dtype, self.device).contiguous() for n, t in named]

    def _out_shapes(self):
        f64 = self.torch.float64
        return dict(I_top=((self.nbands, self.n_up, self.ny, self.nx), self.dtype), J=((self.nz, self.ny, self.nx), f64),
                    F=((3, self.nz, self.ny, self.nx), f64), Q=((self.nz, self.ny, self.nx), f64))

    def _outputs(self, out):
        """The caller's output dict checked (absent or None entries are not
        written), or a new one."""
        shapes = self._out_shapes()
        if out is None:
            return {k: self.torch.empty(shp, dtype=dt, device=self.device) for k, (shp, dt) in shapes.items()}
        for k, v in out.items():
            if k not in shapes:
                raise ValueError(f"unknown output {k!r}; expected some of {sorted(shapes)}")
            if v is not None:
                _need(f"out[{k!r}]", v, shapes[k][0], shapes[k][1], self.device, contiguous=True)
        return out

    def wrap_seed_elems(self):
        """Floats of the warm-start buffer (rts_wrap_seed_elems)."""
        return int(self._L.rts_wrap_seed_elems(self._h))

    def solve(self, chi, S, bottom="equal_s", top="zero", check=True, out=None, wrap_seed=None, seed_in=False,
              seed_tol=0.0):
        """chi, S: CUDA tensors [B, nz, ny, nx] in the solver's dtype.

        wrap_seed: optional float32 CUDA tensor of wrap_seed_elems() elements,
        written with the converged wrap planes; with seed_in=True also read
        as the warm start (rts_boundary.wrap_seed).
        Returns dict(I_top [B,n_up,ny,nx], J [nz,ny,nx], F [3,nz,ny,nx], Q [nz,ny,nx])."""
        torch = self.torch
        chi, S = self._inputs(("chi", chi), ("S", S))
        out = self._outputs(out)
        b, keep = self._bc(bottom, top)
        if wrap_seed is not None:
            if (not wrap_seed.is_cuda or wrap_seed.dtype != torch.float32 or not wrap_seed.is_contiguous()
                    or wrap_seed.numel() != self.wrap_seed_elems() or wrap_seed.device != self.device):
                raise ValueError(f"wrap_seed must be a contiguous CUDA float32 tensor of {self.wrap_seed_elems()}")
            b.wrap_seed = wrap_seed.data_ptr()
            b.seed_in = 1 if seed_in else 0
            b.seed_tol = seed_tol
        rc = self._L.rts_solve(self._h, _ptr(chi), _ptr(S), C.byref(b), _ptr(out.get("I_top")), _ptr(out.get("J")),
                               _ptr(out.get("F")), _ptr(out.get("Q")))
        self._err(rc)
        if check:
            self.check()
        del keep
        return out

    def scatter_solve(self, chi, B, eps, S=None, max_iter=200, tol=None, bottom="equal_s", top="zero", out=None):
        """rts_scatter_solve: the band source functions S = (1 - eps) J + eps B
        (iterated on the GPU from S, default B). chi, B, eps: CUDA tensors
        [B, nz, ny, nx] in the solver dtype. Returns (S, outputs, iterations).
        Needs Solver(..., scatter=True)."""
        chi, B, eps = self._inputs(("chi", chi), ("B", B), ("eps", eps))
        S = (B.clone() if S is None else self._inputs(("S", S))[0].clone()).contiguous()
        if tol is None:
            tol = 1e-12 if self.prec == FP64 else 2e-6
        out = self._outputs(out)
        b, keep = self._bc(bottom, top)
        it = C.c_int(0)
        rc = self._L.rts_scatter_solve(self._h, _ptr(chi), _ptr(B), _ptr(eps),
                                       _ptr(S), C.byref(b), max_iter, tol, C.byref(it), _ptr(out.get("I_top")),
                                       _ptr(out.get("J")), _ptr(out.get("F")), _ptr(out.get("Q")))
        self._err(rc)
        self.check()
        del keep
        return S, out, it.value

    def adjoint(self, chi, S, gI_top=None, gJ=None, gF=None, gQ=None, bottom="equal_s", top="zero", check=True,
                out=None):
        """Gradient of <gI_top,I_top> + <gJ,J> + <gF,F> + <gQ,Q> with respect to
        log chi and S (rts_adjoint). Cotangents may be None (zero); gI_top in
        the solver dtype, gJ/gF/gQ float64. Returns (g_logchi, g_S), each
        [B, nz, ny, nx] in the solver dtype. Needs Solver(..., adjoint=True)."""
        torch = self.torch
        chi, S = self._inputs(("chi", chi), ("S", S))
        shp = self._out_shapes()
        gI_top, gJ, gF, gQ = (None if t is None else _need(n, t, *shp[k], self.device).contiguous()
                              for n, k, t in (("gI_top", "I_top", gI_top), ("gJ", "J", gJ), ("gF", "F", gF),
                                              ("gQ", "Q", gQ)))
        if out is None:
            out = (torch.empty_like(chi), torch.empty_like(S))
        else:
            if len(out) != 2:
                raise ValueError("out must be a pair (g_logchi, g_S)")
            shape = (self.nbands, self.nz, self.ny, self.nx)
            for n, t in zip(("out[0]", "out[1]"), out):
                _need(n, t, shape, self.dtype, self.device, contiguous=True)
        b, keep = self._bc(bottom, top)
        rc = self._L.rts_adjoint(self._h, _ptr(chi), _ptr(S), C.byref(b), _ptr(gI_top), _ptr(gJ), _ptr(gF),
                                 _ptr(gQ), _ptr(out[0]), _ptr(out[1]))
        self._err(rc)
        if check:
            self.check()
        del keep
        return out

    def graph(self, chi, S, bottom="equal_s", top="zero", out=None):
        """Capture one solve with these tensors in a CUDA graph (rts_graph_create).
        The solver's stream must not be the legacy default stream. Returns
        (Graph, out); Graph.launch() replays it."""
        chi, S = self._inputs(("chi", chi), ("S", S))
        out = self._outputs(out)
        b, keep = self._bc(bottom, top)
        return Graph(self, self._L.rts_graph_create, (chi, S), b, out, keep), out

    def solve_host(self, chi, S, bottom="equal_s", top="zero", out=None):
        """Host (numpy) inputs and outputs; the library copies both ways."""
        import numpy as np

        npdt = np.float64 if self.prec == FP64 else np.float32
        shape = (self.nbands, self.nz, self.ny, self.nx)
        chi = _need_host("chi", np.ascontiguousarray(chi, dtype=npdt), shape, npdt)
        S = _need_host("S", np.ascontiguousarray(S, dtype=npdt), shape, npdt)
        out = self._host_outputs(out)
        b = Boundary(_BC[bottom], _BC[top], None, None)
        p = lambda a: None if a is None else C.c_void_p(a.ctypes.data)  # noqa: E731
        rc = self._L.rts_solve_host(self._h, p(chi), p(S), C.byref(b), p(out.get("I_top")), p(out.get("J")),
                                    p(out.get("F")), p(out.get("Q")))
        self._err(rc)
        return out

    def solve_host_async(self, chi, S, out, bottom="equal_s", top="zero"):
        """Enqueue a solve on host (numpy, preferably pinned) buffers and return
        at once (rts_solve_host_async); `out` as returned by solve_host. Call
        host_wait() before reading the outputs."""
        import numpy as np

        npdt = np.float64 if self.prec == FP64 else np.float32
        shape = (self.nbands, self.nz, self.ny, self.nx)
        _need_host("chi", chi, shape, npdt)
        _need_host("S", S, shape, npdt)
        if out is None:
            raise ValueError("solve_host_async needs the output arrays (out)")
        out = self._host_outputs(out)
        p = lambda a: None if a is None else C.c_void_p(a.ctypes.data)  # noqa: E731
        b = Boundary(_BC[bottom], _BC[top], None, None)
        rc = self._L.rts_solve_host_async(self._h, p(chi), p(S), C.byref(b), p(out.get("I_top")), p(out.get("J")),
                                          p(out.get("F")), p(out.get("Q")))
        self._err(rc)
        return out

    def _host_outputs(self, out):
        """The host form of _outputs: numpy arrays (float64 for J, F, Q)."""
        import numpy as np

        shapes = {k: (shp, np.float64 if dt == self.torch.float64 else np.float32)
                  for k, (shp, dt) in self._out_shapes().items()}
        if out is None:
            return {k: np.empty(shp, dtype=dt) for k, (shp, dt) in shapes.items()}
        for k, v in out.items():
            if k not in shapes:
                raise ValueError(f"unknown output {k!r}; expected some of {sorted(shapes)}")
            if v is not None:
                _need_host(f"out[{k!r}]", v, shapes[k][0], shapes[k][1], writable=True)
        return out

    def host_wait(self):
        self._err(self._L.rts_host_wait(self._h))

    def check(self):
        self._err(self._L.rts_check(self._h))

    def stats(self):
        s = Stats()
        rc = self._L.rts_get_stats(self._h, C.byref(s))
        self._err(rc)
        d = {k: getattr(s, k) for k, _ in Stats._fields_ if k not in ("device_status", "ms_adjoint")}
        d["ms_adjoint"] = list(s.ms_adjoint)
        return d


class Graph:
    """A captured solve (rts_graph_*); keeps its tensors alive."""

    def __init__(self, solver, create, inputs, bc, out, keep):
        self.solver = solver
        self._keep = (inputs, out, keep, bc)
        g = C.c_void_p()
        rc = create(solver._h, _ptr(inputs[0]), _ptr(inputs[1]), C.byref(bc), _ptr(out.get("I_top")),
                    _ptr(out.get("J")), _ptr(out.get("F")), _ptr(out.get("Q")), C.byref(g))
        solver._err(rc)
        self._g = g

    def launch(self):
        rc = self.solver._L.rts_graph_launch(self._g)
        self.solver._err(rc)

    def __del__(self):
        try:
            if self._g and self._g.value:
                self.solver._L.rts_graph_destroy(self._g)
                self._g = C.c_void_p()
        except Exception:
            pass


def _grids(shapes, spacing):
    arr = (Grid * len(shapes))()
    for i, (nx, ny, nz) in enumerate(shapes):
        dx, dy, dz = spacing[i] if spacing is not None else (1.0, 1.0, 1.0)
        arr[i] = Grid(nx, ny, nz, dx, dy, dz)
    return arr


class BatchedSolver(Solver):
    """Many grids of uneven size x nbands bands in one persistent launch
    (rts_create_batched / rts_solve_batched).

    shapes: list of (nx, ny, nz); spacing: optional list of (dx, dy, dz).
    Inputs and outputs are packed 1-D tensors (see pack / unpack)."""

    def __init__(self, shapes, nbands=1, spacing=None, precision="fp32", tau_switch=0.1, wrap_tol=0.0,
                 max_wrap_iters=64, tile_rows=0, timeout_s=2.0, timing=False, stream=None, sweep_kernel="auto"):
        import torch

        L = load()
        self.torch = torch
        self.device = torch.device("cuda", torch.cuda.current_device())
        self.shapes = [tuple(int(v) for v in s) for s in shapes]
        self.nbands = nbands
        self.precision = precision
        self.prec = _PREC[precision]
        self.dtype = torch.float64 if self.prec == FP64 else torch.float32
        o = Options()
        L.rts_default_options(C.byref(o))
        o.prec = self.prec
        o.tau_switch = tau_switch
        o.wrap_tol = wrap_tol
        o.max_wrap_iters = max_wrap_iters
        o.tile_rows = tile_rows
        o.timeout_s = timeout_s
        o.flags = FLAG_TIMING if timing else 0
        o.sweep_kernel = _SWEEP[sweep_kernel]
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        o.stream = C.c_void_p(stream.cuda_stream)
        self._opt = o
        self._gr = _grids(self.shapes, spacing)
        h = C.c_void_p()
        rc = L.rts_create_batched(C.byref(h), len(self.shapes), self._gr, nbands, None, C.byref(o))
        self._h = h
        self._L = L
        if rc != RTS_OK:
            msg = L.rts_last_error(h).decode() if h.value else "rts_create_batched failed"
            L.rts_destroy(h)
            self._h = C.c_void_p()
            raise RTSError(rc, msg)
        self.n_up = L.rts_num_up(h)
        self.offsets = []
        tot = (C.c_longlong * 3)()
        for i in range(len(self.shapes)):
            a, b, c = C.c_longlong(), C.c_longlong(), C.c_longlong()
            self._err(L.rts_batched_layout(h, i, C.byref(a), C.byref(b), C.byref(c), tot))
            self.offsets.append((a.value, b.value, c.value))
        self.totals = tuple(tot)

    def pack(self, arrays):
        """List of per-subdomain [B, nz, ny, nx] tensors -> one packed tensor."""
        return self.torch.cat([a.reshape(-1) for a in arrays])

    def unpack(self, out):
        """Packed outputs -> list of per-subdomain dicts of views."""
        res = []
        for (nx, ny, nz), (go, to, po) in zip(self.shapes, self.offsets):
            n = nx * ny * nz
            res.append(dict(I_top=out["I_top"][to:to + self.nbands * self.n_up * nx * ny].view(self.nbands, self.n_up, ny, nx),
                            J=out["J"][po:po + n].view(nz, ny, nx), F=out["F"][3 * po:3 * po + 3 * n].view(3, nz, ny, nx),
                            Q=out["Q"][po:po + n].view(nz, ny, nx)))
        return res

    def empty_outputs(self, device):
        torch = self.torch
        return dict(I_top=torch.empty(self.totals[1], dtype=self.dtype, device=device),
                    J=torch.empty(self.totals[2], dtype=torch.float64, device=device),
                    F=torch.empty(3 * self.totals[2], dtype=torch.float64, device=device),
                    Q=torch.empty(self.totals[2], dtype=torch.float64, device=device))

    def _bc(self, bottom, top):
        # explicit boundary arrays go to the library, which refuses them for
        # batched handles (RTS_EINVAL) without reading them
        b = Boundary()
        keep = []
        for side, v in (("bottom", bottom), ("top", top)):
            if isinstance(v, str):
                setattr(b, side, _BC[v])
            else:
                t = v.contiguous()
                keep.append(t)
                setattr(b, side, BC_EXPLICIT)
                setattr(b, side + "_I", t.data_ptr())
        return b, keep

    def _packed_inputs(self, chi, S):
        n = self.totals[0]
        return [_need(nm, t.reshape(-1) if getattr(t, "numel", lambda: -1)() == n else t, (n,), self.dtype,
                      self.device).contiguous() for nm, t in (("chi", chi), ("S", S))]

    def _packed_outputs(self, out):
        if out is None:
            return self.empty_outputs(self.device)
        f64 = self.torch.float64
        shapes = dict(I_top=(self.totals[1], self.dtype), J=(self.totals[2], f64), F=(3 * self.totals[2], f64),
                      Q=(self.totals[2], f64))
        for k, v in out.items():
            if k not in shapes:
                raise ValueError(f"unknown output {k!r}; expected some of {sorted(shapes)}")
            if v is not None:
                _need(f"out[{k!r}]", v, (shapes[k][0],), shapes[k][1], self.device, contiguous=True)
        return out

    def solve(self, chi, S, bottom="equal_s", top="zero", check=True, out=None):
        """chi, S: packed CUDA tensors of totals[0] elements. Returns packed outputs."""
        chi, S = self._packed_inputs(chi, S)
        out = self._packed_outputs(out)
        b, keep = self._bc(bottom, top)
        rc = self._L.rts_solve_batched(self._h, _ptr(chi), _ptr(S), C.byref(b),
                                       _ptr(out.get("I_top")), _ptr(out.get("J")), _ptr(out.get("F")),
                                       _ptr(out.get("Q")))
        self._err(rc)
        if check:
            self.check()
        del keep
        return out

    def graph(self, chi, S, bottom="equal_s", top="zero", out=None):
        chi, S = self._packed_inputs(chi, S)
        out = self._packed_outputs(out)
        b, keep = self._bc(bottom, top)
        return Graph(self, self._L.rts_graph_create, (chi, S), b, out, keep), out


def autotune(shapes, nbands, chi, S, precision="fp32", spacing=None, repeats=3, stream=None, **opts):
    """rts_autotune: fastest rows per sweep tile for these grids (packed chi,
    S as for BatchedSolver). Returns (best_tile_rows, {rows: ms})."""
    import torch

    L = load()
    o = Options()
    L.rts_default_options(C.byref(o))
    o.prec = _PREC[precision]
    for k, v in opts.items():
        setattr(o, k, v)
    if stream is None:
        stream = torch.cuda.current_stream()
    o.stream = C.c_void_p(stream.cuda_stream)
    # chi, S packed as for BatchedSolver: nbands x the points of every grid
    n = nbands * sum(int(a) * int(b) * int(c) for a, b, c in shapes)
    dt = torch.float64 if o.prec == FP64 else torch.float32
    dev = torch.device("cuda", torch.cuda.current_device())
    chi, S = (_need(nm, t.reshape(-1) if getattr(t, "numel", lambda: -1)() == n else t, (n,), dt, dev).contiguous()
              for nm, t in (("chi", chi), ("S", S)))
    gr = _grids([tuple(s) for s in shapes], spacing)
    best, n = C.c_int(), C.c_int()
    rows = (C.c_int * 8)()
    ms = (C.c_float * 8)()
    rc = L.rts_autotune(len(shapes), gr, nbands, None, C.byref(o), _ptr(chi), _ptr(S), repeats, C.byref(best),
                        C.byref(n), rows, ms)
    if rc != RTS_OK:
        raise RTSError(rc, "autotune found no runnable tile size")
    return best.value, {rows[i]: ms[i] for i in range(n.value)}


def solve_noalloc(chi, S, precision="fp32", dx=1.0, dy=1.0, dz=1.0, out=None, stream=None):
    """Forward solve through rts_solve_noalloc: no device (or host) memory is
    allocated by the library; its scratch is a fixed static device array.
    For callers that must not allocate (an embedding code that owns the
    GPU's memory and gives the solver a fixed budget). The call waits for its
    stream, so it cannot run inside a stream capture. Defaults only: S4
    quadrature, bottom I = S, top I = 0. Outputs may be given (checked for
    shape, dtype and device) or are made here with torch. Returns the outputs
    dict; raises RTSError (with the library's message) on failure, e.g. when
    the grid is too large for the fixed array."""
    import torch

    L = load()
    if chi.dim() != 4:
        raise ValueError(f"chi must be [B, nz, ny, nx], got shape {tuple(chi.shape)}")
    B, nz, ny, nx = chi.shape
    prec = _PREC[precision]
    dt = torch.float64 if prec == FP64 else torch.float32
    for name, t in (("chi", chi), ("S", S)):
        if not t.is_cuda or t.dtype != dt:
            raise ValueError(f"{name} must be a CUDA tensor of {dt}, got {t.dtype} on {t.device}")
    if S.shape != chi.shape or S.device != chi.device:
        raise ValueError(f"S {tuple(S.shape)} on {S.device} must match chi {tuple(chi.shape)} on {chi.device}")
    shapes = dict(I_top=((B, 12, ny, nx), dt), J=((nz, ny, nx), torch.float64), F=((3, nz, ny, nx), torch.float64),
                  Q=((nz, ny, nx), torch.float64))
    with torch.cuda.device(chi.device):  # the library uses the current device's scratch array and stream
        if out is None:
            out = {k: torch.empty(shp, dtype=d, device=chi.device) for k, (shp, d) in shapes.items()}
        for k, v in out.items():
            shp, d = shapes[k]
            if v is not None and (tuple(v.shape) != shp or v.dtype != d or v.device != chi.device
                                  or not v.is_contiguous()):
                raise ValueError(f"out[{k!r}] must be a contiguous {d} tensor {shp} on {chi.device}")
        if stream is None:
            stream = torch.cuda.current_stream(chi.device)
        err = C.create_string_buffer(512)
        g = Grid(nx, ny, nz, dx, dy, dz)
        rc = L.rts_solve_noalloc(C.byref(g), B, prec, _ptr(chi.contiguous()), _ptr(S.contiguous()),
                                 _ptr(out.get("I_top")), _ptr(out.get("J")), _ptr(out.get("F")), _ptr(out.get("Q")),
                                 C.c_void_p(stream.cuda_stream), err, 512)
    if rc != RTS_OK:
        raise RTSError(rc, err.value.decode())
    return out


def device_code_version() -> int:
    """Compute capability the loaded kernels were built for (103 = sm_103a)."""
    return load().rts_device_code_version()


def front_end(T, rho, table, precision="fp32", shift=(-0.5, -0.5, -0.5), out=None, stream=None):
    """rts_front_end: chi_b and S_b [B, nz, ny, nx] on the RTS grid from the
    MHD fields T and rho [nz, ny, nx] (CUDA tensors of the precision's dtype)
    and a band table (dict with ln_kappa [B][nR][nT], ln_B [B][nT], lnT0,
    dlnT, lnR0, dlnR). Enqueued on the current stream; returns (chi, S)."""
    import torch

    L = load()
    prec = _PREC[precision]
    dt = torch.float64 if prec == FP64 else torch.float32
    if T.dim() != 3 or rho.shape != T.shape:
        raise ValueError("T and rho must be [nz, ny, nx] of the same shape")
    for name, t in (("T", T), ("rho", rho)):
        if not t.is_cuda or t.dtype != dt:
            raise ValueError(f"{name} must be a CUDA tensor of {dt}")
    nz, ny, nx = T.shape
    dev = T.device
    if rho.device != dev:
        raise ValueError(f"T and rho must be on the same device, got {T.device} and {rho.device}")
    lnk = torch.as_tensor(table["ln_kappa"], dtype=dt, device=dev).contiguous()
    lnB = torch.as_tensor(table["ln_B"], dtype=dt, device=dev).contiguous()
    nb, nR, nT = lnk.shape
    if tuple(lnB.shape) != (nb, nT):
        raise ValueError("ln_B must be [nbands, nT]")
    tab = FrontTable(nb, nT, nR, table["lnT0"], table["dlnT"], table["lnR0"], table["dlnR"], lnk.data_ptr(),
                     lnB.data_ptr(), (C.c_double * 3)(*shift))
    if out is None:
        out = (torch.empty((nb, nz, ny, nx), dtype=dt, device=dev), torch.empty((nb, nz, ny, nx), dtype=dt, device=dev))
    elif len(out) != 2:
        raise ValueError("out must be a pair (chi, S)")
    else:
        for n, t in zip(("out[0]", "out[1]"), out):
            _need(n, t, (nb, nz, ny, nx), dt, dev, contiguous=True)
    if stream is None:
        stream = torch.cuda.current_stream(dev)
    err = C.create_string_buffer(256)
    g = Grid(nx, ny, nz, 1.0, 1.0, 1.0)
    with torch.cuda.device(dev):
        rc = L.rts_front_end(C.byref(g), C.byref(tab), prec, _ptr(T.contiguous()), _ptr(rho.contiguous()),
                             _ptr(out[0]), _ptr(out[1]), C.c_void_p(stream.cuda_stream), err, 256)
    if rc != RTS_OK:
        raise RTSError(rc, err.value.decode())
    out[0]._rts_keep = (lnk, lnB)  # the tables stay alive until the enqueued kernel has read them
    return out


class DecomposedSolver:
    """The grid cut into nblocks slabs of levels, iterated on their boundary
    intensities until the global J criterion holds (rts_create_decomposed /
    rts_solve_decomposed). FP32 modes only."""

    def __init__(self, nx, ny, nz, nbands=1, nblocks=2, dx=1.0, dy=1.0, dz=1.0, precision="fp32", tau_switch=0.1,
                 wrap_tol=0.0, max_wrap_iters=64, timeout_s=2.0, stream=None):
        import torch

        L = load()
        self.torch = torch
        self._L = L
        self._h = C.c_void_p()
        self.device = torch.device("cuda", torch.cuda.current_device())
        self.nx, self.ny, self.nz, self.nbands, self.nblocks = nx, ny, nz, nbands, nblocks
        self.prec = _PREC[precision]
        self.dtype = torch.float32
        o = Options()
        L.rts_default_options(C.byref(o))
        o.prec = self.prec
        o.tau_switch = tau_switch
        o.wrap_tol = wrap_tol
        o.max_wrap_iters = max_wrap_iters
        o.timeout_s = timeout_s
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        o.stream = C.c_void_p(stream.cuda_stream)
        h = C.c_void_p()
        rc = L.rts_create_decomposed(C.byref(h), C.byref(Grid(nx, ny, nz, dx, dy, dz)), nbands, nblocks, None,
                                     C.byref(o))
        if rc != RTS_OK:
            msg = L.rts_decomposed_last_error(h).decode() if h.value else "rts_create_decomposed failed"
            L.rts_destroy_decomposed(h)
            raise RTSError(rc, msg)
        self._h = h
        self.n_up = 12

    def __del__(self):
        try:
            if self._h and self._h.value:
                self._L.rts_destroy_decomposed(self._h)
                self._h = C.c_void_p()
        except Exception:
            pass

    def solve(self, chi, S, tol=1e-6, max_iter=32, out=None):
        """chi, S: float32 CUDA tensors [B, nz, ny, nx]. Returns (outputs,
        iterations), outputs as Solver.solve."""
        chi, S = self._inputs(("chi", chi), ("S", S))
        out = self._outputs(out)
        it = C.c_int(0)
        rc = self._L.rts_solve_decomposed(self._h, _ptr(chi), _ptr(S), None, tol, max_iter, C.byref(it),
                                          _ptr(out.get("I_top")), _ptr(out.get("J")), _ptr(out.get("F")),
                                          _ptr(out.get("Q")))
        if rc != RTS_OK:
            raise RTSError(rc, self._L.rts_decomposed_last_error(self._h).decode())
        return out, it.value

    _inputs = Solver._inputs
    _out_shapes = Solver._out_shapes
    _outputs = Solver._outputs
