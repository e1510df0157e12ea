"""Brute-force dense solve of one direction's discrete transfer problem.

Used only to pin the oracle's sweep order and its periodic-wrap iteration on
tiny grids: every grid point gets one row of the linear system
    I_p - e_p * sum_c beta_c I(u_c(p)) = w_up,p S_up,p + w_p,p S_p   (integrated)
    I_p = boundary value                                                (set)
which is assembled here from the definitions, independently of the oracle's
code, and solved with dense LU (numpy.linalg.solve). No ordering, no
iteration and no periodic bookkeeping beyond "indices wrap in x and y".
"""
from __future__ import annotations

import math

import numpy as np


def geometry(n, h):
    """Dominant axis, sign, minor axes with signs and fractions, path length."""
    order = [2, 1, 0]
    best, a = None, None
    for ax in order:
        if abs(n[ax]) > 0:
            s = h[ax] / abs(n[ax])
            if best is None or s < best:
                best, a = s, ax
    minors = [ax for ax in (0, 1, 2) if ax != a]
    frac = [best * abs(n[m]) / h[m] for m in minors]
    sg = [(-1 if n[m] < 0 else 1) for m in minors]
    return a, (1 if n[a] > 0 else -1), minors, sg, frac, best


def weights(x):
    e = math.exp(-x)
    if x == 0.0:
        return e, 0.0, 0.0
    ome = -math.expm1(-x)
    return e, ome / x - e, 1.0 - ome / x


def dense_direction(n, h, chi, S, bc_value):
    """I [nz,ny,nx] of one direction; bc_value(i, j) gives the boundary value."""
    nz, ny, nx = chi.shape
    N = nx * ny * nz
    a, sa, minors, sg, frac, ds = geometry(n, h)
    up = n[2] > 0
    kb = 0 if up else nz - 1

    def idx(i, j, k):
        return (k * ny + (j % ny)) * nx + (i % nx)

    A = np.zeros((N, N))
    rhs = np.zeros(N)
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                p = idx(i, j, k)
                A[p, p] = 1.0
                if k == kb:
                    rhs[p] = bc_value(i, j)
                    continue
                corners = []
                for c1 in (0, 1):
                    for c2 in (0, 1):
                        off = [0, 0, 0]
                        off[a] = -sa
                        off[minors[0]] = -sg[0] * c1
                        off[minors[1]] = -sg[1] * c2
                        beta = (frac[0] if c1 else 1 - frac[0]) * (frac[1] if c2 else 1 - frac[1])
                        kk = k + off[2]
                        assert 0 <= kk < nz
                        corners.append((idx(i + off[0], j + off[1], kk), beta))
                chi_up = sum(b * chi.flat[q] for q, b in corners)
                S_up = sum(b * S.flat[q] for q, b in corners)
                dtau = ds * 0.5 * (chi_up + chi.flat[p])
                e, wu, wp = weights(dtau)
                for q, b in corners:
                    A[p, q] -= e * b
                rhs[p] = wu * S_up + wp * S.flat[p]
    return np.linalg.solve(A, rhs).reshape(nz, ny, nx)
