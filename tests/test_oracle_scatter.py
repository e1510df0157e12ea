"""Pins of the scattering oracle (oracle/scatter.py) by what fixes the
solution exactly: eps = 1 gives S = B after one step; an isothermal medium
whose boundaries radiate B (bottom I = S, explicit top I = B) has J = B, so
S = B is the fixed point for every eps and every opacity field; S is linear
in B; the converged S satisfies its defining equation."""
import numpy as np

import oracle
from oracle.scatter import scatter_solve


def _case(nx=6, ny=5, nz=7, nb=2, seed=0):
    rng = np.random.default_rng(seed)
    chi = np.exp(rng.normal(0.0, 0.5, (nb, nz, ny, nx))) * np.array([0.5, 3.0][:nb])[:, None, None, None]
    B = 1.0 + 0.3 * rng.random((nb, nz, ny, nx))
    return chi, B


def test_eps_one_is_thermal():
    chi, B = _case()
    P = oracle.Problem(6, 5, 7, 2, max_wrap_iters=100000)
    S, out, it = scatter_solve(P, chi, B, np.ones_like(B))
    assert np.array_equal(S, B) and it == 1


def test_isothermal_box_is_a_fixed_point():
    chi, _ = _case(seed=2)
    B = np.full_like(chi, 1.7)
    top = np.full((2, 12, 5, 6), 1.7)
    P = oracle.Problem(6, 5, 7, 2, max_wrap_iters=100000, top=oracle.BC_EXPLICIT, top_I=top)
    for e in (0.05, 0.5):
        S, out, it = scatter_solve(P, chi, B, np.full_like(B, e))
        assert np.abs(S - 1.7).max() < 1e-12
        assert np.abs(out["J"] - 2 * 1.7).max() < 1e-12  # two bands


def test_linear_in_the_thermal_source_and_satisfies_its_equation():
    chi, B = _case(seed=3)
    eps = np.full_like(B, 0.2)
    P = oracle.Problem(6, 5, 7, 2, max_wrap_iters=100000, bottom=oracle.BC_ZERO)
    S1, _, _ = scatter_solve(P, chi, B, eps)
    S2, _, _ = scatter_solve(P, chi, 3.0 * B, eps)
    assert np.abs(S2 - 3.0 * S1).max() < 1e-11 * np.abs(S2).max()
    Jb = P.solve(chi, S1, debug=True)["Jb"]
    assert np.abs(S1 - (0.8 * Jb + 0.2 * B)).max() < 1e-12 * np.abs(S1).max()
    assert np.abs(S1 - B).max() > 1e-3  # scattering changes S
