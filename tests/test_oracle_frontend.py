"""Pins of the input-step oracle (oracle/frontend.py) against what the
mathematics fixes: trilinear interpolation is exact for a field whose log is
linear in the cell coordinates, the half-cell stagger of an interior point
averages its 8 cells, a z position below the first layer takes that layer,
bilinear table interpolation is exact for a bilinear function and returns
the node values at the nodes, lookups outside the table take its edge, and
shifting the MHD fields by one cell shifts the result by one point."""
import numpy as np

from oracle.frontend import front_end, table_lookup, trilinear_log
from workloads.opacity import mhd_fields, synthetic_table


def test_trilinear_exact_for_log_linear_fields():
    nz, ny, nx = 7, 6, 9
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    a, b, c, d = 0.3, -0.11, 0.07, 0.23
    f = np.exp(a + b * i + c * j + d * k)
    for shift in ((-0.5, -0.5, -0.5), (0.25, -0.75, 0.4)):
        got = trilinear_log(f, shift)
        want = a + b * (i + shift[0]) + c * (j + shift[1]) + d * (k + shift[2])
        # interior: no periodic seam in x, y and no clamping in z
        sx = slice(1, nx - 1)
        sy = slice(1, ny - 1)
        sz = slice(1, nz - 1)
        assert np.allclose(got[sz, sy, sx], want[sz, sy, sx], rtol=0, atol=1e-14)


def test_half_cell_stagger_is_the_mean_of_eight_cells():
    rng = np.random.default_rng(4)
    f = np.exp(rng.standard_normal((5, 6, 7)))
    got = trilinear_log(f, (-0.5, -0.5, -0.5))
    lf = np.log(f)
    kk, jj, ii = 3, 2, 4
    cells = [lf[kk - dz, (jj - dy) % 6, (ii - dx) % 7] for dz in (0, 1) for dy in (0, 1) for dx in (0, 1)]
    assert abs(got[kk, jj, ii] - sum(cells) / 8.0) < 1e-15
    # the periodic seam: point (i = 0) averages cells nx-1 and 0
    cells0 = [lf[kk - dz, (jj - dy) % 6, (0 - dx) % 7] for dz in (0, 1) for dy in (0, 1) for dx in (0, 1)]
    assert abs(got[kk, jj, 0] - sum(cells0) / 8.0) < 1e-15
    # z below the first layer: that layer alone (x, y still interpolated)
    cz = [lf[0, (jj - dy) % 6, (ii - dx) % 7] for dy in (0, 1) for dx in (0, 1)]
    assert abs(got[0, jj, ii] - sum(cz) / 4.0) < 1e-15


def _bilinear_table(nb=2, nT=5, nR=4):
    lnT = np.linspace(-0.5, 0.7, nT)
    lnR = np.linspace(-3.0, 2.0, nR)
    lnk = np.empty((nb, nR, nT))
    for b in range(nb):
        lnk[b] = 0.1 * b + 1.5 * lnT[None] - 0.4 * lnR[:, None] + 0.3 * lnT[None] * lnR[:, None]
    lnB = np.stack([4 * lnT + b for b in range(nb)])
    return {"ln_kappa": lnk, "ln_B": lnB, "lnT0": lnT[0], "dlnT": lnT[1] - lnT[0], "lnR0": lnR[0],
            "dlnR": lnR[1] - lnR[0]}, lnT, lnR


def test_table_exact_for_bilinear_functions_and_at_nodes():
    tab, lnT, lnR = _bilinear_table()
    rng = np.random.default_rng(1)
    qT = rng.uniform(lnT[0], lnT[-1], 200)
    qR = rng.uniform(lnR[0], lnR[-1], 200)
    k, b = table_lookup(qT, qR, tab)
    for band in range(2):
        want = 0.1 * band + 1.5 * qT - 0.4 * qR + 0.3 * qT * qR
        assert np.allclose(k[band], want, rtol=0, atol=1e-13)
        assert np.allclose(b[band], 4 * qT + band, rtol=0, atol=1e-13)
    # the nodes themselves
    TT, RR = np.meshgrid(lnT, lnR)
    k, _ = table_lookup(TT, RR, tab)
    assert np.allclose(k, tab["ln_kappa"], rtol=0, atol=1e-14)
    # outside the table: the edge
    k_lo, _ = table_lookup(np.array([lnT[0] - 5.0]), np.array([lnR[0] - 5.0]), tab)
    k_hi, _ = table_lookup(np.array([lnT[-1] + 5.0]), np.array([lnR[-1] + 5.0]), tab)
    assert np.allclose(k_lo[:, 0], tab["ln_kappa"][:, 0, 0]) and np.allclose(k_hi[:, 0], tab["ln_kappa"][:, -1, -1])


def test_front_end_shifts_with_the_fields():
    T, rho = mhd_fields(10, 8, 6, 3)
    tab = synthetic_table(nb=3)
    chi, S = front_end(T, rho, tab)
    chi2, S2 = front_end(np.roll(T, 1, axis=2), np.roll(rho, 1, axis=2), tab)
    assert np.allclose(chi2, np.roll(chi, 1, axis=3), rtol=1e-14, atol=0)
    assert np.allclose(S2, np.roll(S, 1, axis=3), rtol=1e-14, atol=0)
    # chi = kappa rho and S = B at a point whose T, rho are constant around it
    Tc, rc = np.full((4, 4, 4), 1.3), np.full((4, 4, 4), 0.02)
    chi, S = front_end(Tc, rc, tab)
    k, b = table_lookup(np.array([np.log(1.3)]), np.array([np.log(0.02)]), tab)
    assert np.allclose(chi[:, 2, 2, 2], np.exp(k[:, 0]) * 0.02, rtol=1e-14)
    assert np.allclose(S[:, 2, 2, 2], np.exp(b[:, 0]), rtol=1e-14)
