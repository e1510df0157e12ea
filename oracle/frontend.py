"""FP64 oracle of the solver's input step: the paper's RTS "Interpolate"
(Sect. 2: trilinear interpolation of the MHD variables from the MHD grid to
the staggered RTS grid, then the source function and opacities of every
band, from band-integrated tables as in opacity binning, Sect. 1).

TEST INFRASTRUCTURE ONLY: used by tests/ and nothing else; it shares no code
with the CUDA library.

Readings (the paper gives no formulas): the MHD fields T and rho live at the
MHD cell centres; RTS point (i, j, k) sits at MHD cell coordinates
(i, j, k) + shift; ln T and ln rho (not T and rho) are interpolated, because
both vary exponentially with height; x and y are periodic, z is clamped to
the first and last layer; ln kappa_b is bilinear in (ln T, ln rho) on a
regular table, ln B_b linear in ln T, both clamped at the table edges;
chi_b = kappa_b rho, S_b = B_b.

The steps are written one by one with plain loops over the 8 corners and
the 4 table nodes; numpy only vectorises over the grid points.
"""
from __future__ import annotations

import numpy as np


def _cell_and_weight(u, n):
    """Lower node and weight of coordinates u on n nodes 0..n-1, clamped."""
    u = np.asarray(u, dtype=np.float64)
    if n == 1:
        return np.zeros(u.shape, dtype=np.int64), np.zeros(u.shape)
    c = np.floor(u).astype(np.int64)
    w = u - c
    low = u <= 0.0
    high = u >= n - 1
    c = np.where(low, 0, np.where(high, n - 2, c))
    w = np.where(low, 0.0, np.where(high, 1.0, w))
    return c, w


def trilinear_log(field, shift):
    """exp of the trilinear interpolation of ln(field) [nz, ny, nx] at every
    RTS point; returns the interpolated ln(field)."""
    f = np.log(np.asarray(field, dtype=np.float64))
    nz, ny, nx = f.shape
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    ux, uy, uz = i + shift[0], j + shift[1], k + shift[2]
    fx, fy = np.floor(ux), np.floor(uy)
    wx, wy = ux - fx, uy - fy
    x0 = np.mod(fx.astype(np.int64), nx)
    y0 = np.mod(fy.astype(np.int64), ny)
    x1, y1 = np.mod(x0 + 1, nx), np.mod(y0 + 1, ny)
    z0, wz = _cell_and_weight(uz, nz)
    z1 = np.minimum(z0 + 1, nz - 1)
    out = np.zeros(f.shape)
    for cz, wzc in ((z0, 1.0 - wz), (z1, wz)):
        for cy, wyc in ((y0, 1.0 - wy), (y1, wy)):
            for cx, wxc in ((x0, 1.0 - wx), (x1, wx)):
                out += wzc * wyc * wxc * f[cz, cy, cx]
    return out


def table_lookup(lnT, lnR, table):
    """ln kappa_b (bilinear) and ln B_b (linear) at every point, per band."""
    lnk = np.asarray(table["ln_kappa"], dtype=np.float64)   # [B][nR][nT]
    lnB = np.asarray(table["ln_B"], dtype=np.float64)       # [B][nT]
    nb, nR, nT = lnk.shape
    it, at = _cell_and_weight((lnT - table["lnT0"]) / table["dlnT"], nT)
    ir, ar = _cell_and_weight((lnR - table["lnR0"]) / table["dlnR"], nR)
    it1 = np.minimum(it + 1, nT - 1)
    ir1 = np.minimum(ir + 1, nR - 1)
    k = np.empty((nb,) + lnT.shape)
    b = np.empty((nb,) + lnT.shape)
    for band in range(nb):
        t = lnk[band]
        k[band] = ((1 - ar) * ((1 - at) * t[ir, it] + at * t[ir, it1]) +
                   ar * ((1 - at) * t[ir1, it] + at * t[ir1, it1]))
        b[band] = (1 - at) * lnB[band][it] + at * lnB[band][it1]
    return k, b


def front_end(T, rho, table, shift=(-0.5, -0.5, -0.5)):
    """chi_b, S_b [B, nz, ny, nx] on the RTS grid from T, rho on the MHD grid."""
    lnT = trilinear_log(T, shift)
    lnR = trilinear_log(rho, shift)
    lnk, lnb = table_lookup(lnT, lnR, table)
    chi = np.exp(lnk) * np.exp(lnR)[None]
    S = np.exp(lnb)
    return chi, S
