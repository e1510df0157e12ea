"""Synthetic MHD fields and a synthetic band-opacity table for the solver's
input step (no MURaM snapshot, EOS or opacity table is available).

mhd_fields(nx, ny, nz, seed): T from the stratified atmosphere generator and
rho = rho0 exp(-z / (4L)) exp(0.3 g) with g ~ N(0, 1) (the opacity profile
of that generator, read as a density), on the MHD cell centres.

synthetic_table(nb, nT, nR): ln kappa_b on a regular (ln T, ln rho) grid,
ln kappa_b = ln(10^(b - 1)) + 3 ln T + 0.5 ln rho + 0.2 sin(2 ln T) cos(ln rho)
(a smooth function that bilinear interpolation does not reproduce exactly),
and ln B_b = 4 ln T + ln(w_b) with band weights w_b summing to 1.
"""
from __future__ import annotations

import numpy as np

from .atmosphere import stratified_atmosphere


def mhd_fields(nx: int, ny: int, nz: int, seed: int = 0):
    T, _, chi = stratified_atmosphere(nx, ny, nz, seed)
    return T, chi  # the generator's opacity field stands in for the density


def synthetic_table(nb: int = 4, nT: int = 64, nR: int = 96, lnT_range=(-1.0, 1.0), lnR_range=(-14.0, 6.0)):
    lnT = np.linspace(lnT_range[0], lnT_range[1], nT)
    lnR = np.linspace(lnR_range[0], lnR_range[1], nR)
    w = np.arange(nb, 0, -1, dtype=np.float64)
    w = w / w.sum()
    lnk = np.empty((nb, nR, nT))
    lnB = np.empty((nb, nT))
    for b in range(nb):
        lnk[b] = (np.log(10.0 ** (b - 1)) + 3.0 * lnT[None, :] + 0.5 * lnR[:, None]
                  + 0.2 * np.sin(2.0 * lnT[None, :]) * np.cos(lnR[:, None]))
        lnB[b] = 4.0 * lnT + np.log(w[b])
    return {"ln_kappa": lnk, "ln_B": lnB, "lnT0": float(lnT[0]), "dlnT": float(lnT[1] - lnT[0]),
            "lnR0": float(lnR[0]), "dlnR": float(lnR[1] - lnR[0])}
