"""Synthetic stratified solar-like atmospheres on the RTS grid.

The paper's test problem is a 288^3 MURaM snapshot (Sect. 6, "Results"); no
snapshot, opacity table or equation-of-state table is available, so these
generators stand in for it with the same grid sizes and band counts.

Recipe (all arrays C-contiguous [Nz][Ny][Nx], x fastest, k=0 at the bottom):
  z = k * dz with dz = 1 and L = Nz / 32 (the profile is stretched with Nz);
  T = 1 + 0.5 tanh((16 L - z) / (8 L)) + 0.05 n, where n ~ N(0,1) is smoothed
      by a 3-point box [1,1,1]/3 along x, then y (periodic), then z
      (edge-replicated);
  S = T^4;
  chi = chi0 exp(-z / (4 L)) exp(0.3 g), g ~ N(0,1) independent of n
      (lognormal sigma 0.3, median 1);
  chi0 = 1 / (4 L (exp(-z_mid/(4L)) - exp(-z_top/(4L)))), z_mid=(Nz-1)/2,
      z_top = Nz - 1, so that the smooth profile has optical depth 1 at
      mid-height.
Random numbers: numpy default_rng(seed); the T noise is drawn first, then g.
"""
from __future__ import annotations

import numpy as np

def _box3(a: np.ndarray, axis: int, periodic: bool) -> np.ndarray:
    if periodic:
        return (np.roll(a, 1, axis) + a + np.roll(a, -1, axis)) / 3.0
    lo = np.concatenate([np.take(a, [0], axis), np.take(a, range(a.shape[axis] - 1), axis)], axis)
    hi = np.concatenate([np.take(a, range(1, a.shape[axis]), axis), np.take(a, [a.shape[axis] - 1], axis)], axis)
    return (lo + a + hi) / 3.0


def stratified_atmosphere(nx: int, ny: int, nz: int, seed: int = 0):
    """Return (T, S, chi) float64 arrays of shape [nz, ny, nx]."""
    rng = np.random.default_rng(seed)
    noise = rng.standard_normal((nz, ny, nx))
    g = rng.standard_normal((nz, ny, nx))
    noise = _box3(noise, 2, True)
    noise = _box3(noise, 1, True)
    noise = _box3(noise, 0, False)
    L = nz / 32.0
    z = np.arange(nz, dtype=np.float64)[:, None, None]
    T = 1.0 + 0.5 * np.tanh((16.0 * L - z) / (8.0 * L)) + 0.05 * noise
    S = T ** 4
    z_mid = (nz - 1) / 2.0
    z_top = float(nz - 1)
    denom = np.exp(-z_mid / (4.0 * L)) - np.exp(-z_top / (4.0 * L))
    chi0 = 1.0 / (4.0 * L * denom) if denom > 0 else 1.0
    chi = chi0 * np.exp(-z / (4.0 * L)) * np.exp(0.3 * g)
    return T, S, chi


def band_stack(T: np.ndarray, chi: np.ndarray, chi_scale, s_scale):
    """Per-band inputs chi_b = chi * chi_scale[b], S_b = T^4 * s_scale[b].

    Returns (chi_b, S_b) of shape [B, nz, ny, nx] float64."""
    chi_scale = np.asarray(chi_scale, dtype=np.float64)
    s_scale = np.asarray(s_scale, dtype=np.float64)
    S4 = T ** 4
    chib = chi[None] * chi_scale[:, None, None, None]
    Sb = S4[None] * s_scale[:, None, None, None]
    return np.ascontiguousarray(chib), np.ascontiguousarray(Sb)


def _bands(name: str, nb: int):
    if name == "gray":
        return [1.0], [1.0]
    if name == "four":  # chi x {1,10,100,1000}, S x {0.4,0.3,0.2,0.1}
        return [1.0, 10.0, 100.0, 1000.0], [0.4, 0.3, 0.2, 0.1]
    if name == "twelve":  # chi x 10^(3b/11), S x (12-b)/78
        return [10.0 ** (3.0 * b / 11.0) for b in range(12)], [(12 - b) / 78.0 for b in range(12)]
    if name == "sixteen":  # chi x 10^(4b/15), S x 1/16
        return [10.0 ** (4.0 * b / 15.0) for b in range(16)], [1.0 / 16.0] * 16
    raise KeyError(name)


# Named workloads: grid, band set and default boundary conditions.
WORKLOADS = {
    # gray 32^3, FP64 reference case
    "gray32": dict(nx=32, ny=32, nz=32, bands="gray", seed=0),
    # the paper's 288^3 test size with 4 opacity bands
    "rts288x4": dict(nx=288, ny=288, nz=288, bands="four", seed=0),
    # adjoint case and its finite-difference sub-case
    "adj96x4": dict(nx=96, ny=96, nz=96, bands="four", seed=0),
    "adj16x4": dict(nx=16, ny=16, nz=16, bands="four", seed=0),
    # large anisotropic grid, 16 bands
    "large512x256x16": dict(nx=512, ny=512, nz=256, bands="sixteen", seed=0),
}


def workload(name: str, dtype=np.float64, nx=None, ny=None, nz=None, seed=None):
    """Build (chi_b, S_b) [B,nz,ny,nx] for a named workload (sizes overridable)."""
    w = dict(WORKLOADS[name])
    nx = w["nx"] if nx is None else nx
    ny = w["ny"] if ny is None else ny
    nz = w["nz"] if nz is None else nz
    seed = w["seed"] if seed is None else seed
    T, _, chi = stratified_atmosphere(nx, ny, nz, seed)
    cs, ss = _bands(w["bands"], 0)
    chib, Sb = band_stack(T, chi, cs, ss)
    return chib.astype(dtype), Sb.astype(dtype)


def batched_subdomain_shapes(count: int = 64, seed: int = 0):
    """Uneven subdomain sizes: Nx=Ny from {48,64,96,128}, Nz from {96,128,192}."""
    rng = np.random.default_rng(seed)
    nxy = rng.choice([48, 64, 96, 128], size=count)
    nzs = rng.choice([96, 128, 192], size=count)
    return [(int(a), int(a), int(c)) for a, c in zip(nxy, nzs)]


def batched_bands():
    return _bands("twelve", 12)
