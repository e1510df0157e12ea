"""Helpers for the GPU parity tests: seeded inputs, oracle runs, comparisons."""
from __future__ import annotations

import numpy as np

import oracle
from workloads import stratified_atmosphere, band_stack, workload

OUTPUTS = ("I_top", "J", "F", "Q")


def random_case(nx, ny, nz, B, seed, thin=False):
    """Stratified atmosphere with B bands spread over opacity (and, for
    thin=True, a very transparent top so the periodic wrap works hard)."""
    T, _, chi = stratified_atmosphere(nx, ny, nz, seed)
    cs = [10.0 ** (2.0 * b / max(1, B - 1)) for b in range(B)]
    ss = [0.4 - 0.3 * b / max(1, B - 1) for b in range(B)]
    chib, Sb = band_stack(T, chi, cs, ss)
    if thin:
        chib = chib * 0.05
    return chib, Sb


def norm_err(got, ref):
    """max |got - ref| / max |ref| (normwise relative error)."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    scale = np.abs(ref).max()
    return float(np.abs(got - ref).max() / (scale if scale > 0 else 1.0))


def gpu_solve(solver, chi, S, bottom="equal_s", top="zero"):
    import torch

    dt = solver.dtype
    c = torch.as_tensor(chi, dtype=dt, device="cuda")
    s = torch.as_tensor(S, dtype=dt, device="cuda")
    b = bottom if isinstance(bottom, str) else torch.as_tensor(bottom, dtype=dt, device="cuda")
    t = top if isinstance(top, str) else torch.as_tensor(top, dtype=dt, device="cuda")
    out = solver.solve(c, s, bottom=b, top=t)
    return {k: v.double().cpu().numpy() for k, v in out.items()}


def oracle_solve(chi, S, dx=1.0, dy=1.0, dz=1.0, bottom="equal_s", top="zero", nthreads=None, **kw):
    B, nz, ny, nx = chi.shape
    bk = {"equal_s": oracle.BC_EQUAL_S, "zero": oracle.BC_ZERO}
    args = {}
    if isinstance(bottom, str):
        args["bottom"] = bk[bottom]
    else:
        args.update(bottom=oracle.BC_EXPLICIT, bottom_I=np.asarray(bottom, dtype=np.float64))
    if isinstance(top, str):
        args["top"] = bk[top]
    else:
        args.update(top=oracle.BC_EXPLICIT, top_I=np.asarray(top, dtype=np.float64))
    P = oracle.Problem(nx, ny, nz, B, dx=dx, dy=dy, dz=dz, max_wrap_iters=100000, **args, **kw)
    return P.solve(np.asarray(chi, dtype=np.float64), np.asarray(S, dtype=np.float64),
                   nthreads=nthreads or oracle.default_threads())


def workload_inputs(name, **kw):
    return workload(name, **kw)
