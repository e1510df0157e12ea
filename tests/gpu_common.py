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


FOUR_PI = 4.0 * np.pi


def elementwise_floors(ref, chi, S, h_min=1.0):
    """Per-point scales of the terms each output is formed from, for an
    element-wise bar |got - ref| <= rel * (|ref| + floor):
      I_top, J   0 (sums of non-negative terms: relative to the value)
      F          4 pi J        (every |F_c| <= 4 pi sum_d w_d |n_d| I_d <= 4 pi J)
      Q_rad      4 pi sum_b (chi_b S_b + J_b / h_min), bounded with J for J_b:
                 the sizes of 4 pi chi (J - S) and of div F, which cancel"""
    chi = np.asarray(chi, dtype=np.float64)
    S = np.asarray(S, dtype=np.float64)
    J = np.abs(np.asarray(ref["J"], dtype=np.float64))
    fl = {"I_top": 0.0, "J": 0.0, "F": FOUR_PI * J[None]}
    fl["Q"] = FOUR_PI * ((chi * S).sum(axis=0) + J / h_min)
    return fl


def elementwise_err(got, ref, floor):
    """max over points of |got - ref| / (|ref| + floor) (0/0 counts as 0)."""
    g = np.asarray(got, dtype=np.float64)
    r = np.asarray(ref, dtype=np.float64)
    den = np.abs(r) + floor
    d = np.abs(g - r)
    with np.errstate(invalid="ignore", divide="ignore"):
        q = np.where(den > 0, d / den, np.where(d > 0, np.inf, 0.0))
    return float(q.max())


def error_report(got, ref, chi, S, h_min=1.0):
    """Normwise and element-wise errors per output, and the flux components
    and I_top relative to their own maximum."""
    fl = elementwise_floors(ref, chi, S, h_min)
    rep = {}
    for k in OUTPUTS:
        rep[k] = {"normwise": norm_err(got[k], ref[k]), "elementwise": elementwise_err(got[k], ref[k], fl[k])}
    for c, name in enumerate(("F_x", "F_y", "F_z")):
        rep[name] = {"normwise": norm_err(got["F"][c], ref["F"][c])}
    return rep
