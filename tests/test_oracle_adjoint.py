"""Pins of the oracle's adjoint: central finite differences of the oracle's
own forward solve (in FP64), and properties the exact gradient must have."""
import numpy as np
import pytest

import oracle


def _loss(P, chi, S, c):
    out = P.solve(chi, S)
    return (np.sum(c["I_top"] * out["I_top"]) + np.sum(c["J"] * out["J"]) + np.sum(c["F"] * out["F"])
            + np.sum(c["Q"] * out["Q"]))


def _cot(P, rng):
    B = P.nbands
    return dict(I_top=rng.normal(size=(B, P.nup, P.ny, P.nx)), J=rng.normal(size=P.shape),
                F=rng.normal(size=(3,) + P.shape), Q=rng.normal(size=P.shape))


@pytest.mark.parametrize("shape,bottom,top", [((5, 4, 6), oracle.BC_EQUAL_S, oracle.BC_ZERO),
                                              ((4, 5, 7), oracle.BC_EQUAL_S, oracle.BC_EQUAL_S)])
def test_adjoint_directional_fd(oracle_mod, shape, bottom, top):
    nx, ny, nz = shape
    rng = np.random.default_rng(nx * 100 + nz)
    B = 2
    chi = np.exp(rng.normal(-0.5, 1.0, (B, nz, ny, nx)))
    S = 0.5 + rng.random((B, nz, ny, nx))
    P = oracle.Problem(nx, ny, nz, B, bottom=bottom, top=top, max_wrap_iters=100000)
    c = _cot(P, rng)
    glc, gS = P.adjoint(chi, S, c["I_top"], c["J"], c["F"], c["Q"])
    for trial in range(3):
        v1 = rng.normal(size=chi.shape)
        v2 = rng.normal(size=S.shape)
        eps = 1e-6
        lp = _loss(P, chi * np.exp(eps * v1), S + eps * v2, c)
        lm = _loss(P, chi * np.exp(-eps * v1), S - eps * v2, c)
        fd = (lp - lm) / (2 * eps)
        an = np.sum(glc * v1) + np.sum(gS * v2)
        assert abs(fd - an) <= 1e-7 * max(1.0, abs(an)), (fd, an)


def test_adjoint_elementwise_fd(oracle_mod):
    """A few single entries, including boundary layers and a periodic edge."""
    from workloads import stratified_atmosphere

    nx, ny, nz = 6, 5, 8
    T, S0, chi0 = stratified_atmosphere(nx, ny, nz, 1)
    chi = chi0[None].copy()
    S = S0[None].copy()
    rng = np.random.default_rng(2)
    P = oracle.Problem(nx, ny, nz, 1, max_wrap_iters=100000)
    c = _cot(P, rng)
    glc, gS = P.adjoint(chi, S, c["I_top"], c["J"], c["F"], c["Q"])
    for (k, j, i) in [(0, 0, 0), (nz - 1, 2, 5), (3, 4, 0), (5, 0, 3), (nz - 2, 1, 1)]:
        for which in ("chi", "S"):
            eps = 1e-6
            a, b = chi.copy(), S.copy()
            a2, b2 = chi.copy(), S.copy()
            if which == "chi":
                a[0, k, j, i] *= np.exp(eps)
                a2[0, k, j, i] *= np.exp(-eps)
                ref = glc[0, k, j, i]
            else:
                b[0, k, j, i] += eps
                b2[0, k, j, i] -= eps
                ref = gS[0, k, j, i]
            fd = (_loss(P, a, b, c) - _loss(P, a2, b2, c)) / (2 * eps)
            assert abs(fd - ref) <= 1e-7 * max(1.0, abs(ref)), (which, k, j, i, fd, ref)


def test_adjoint_linear_in_cotangent(oracle_mod):
    rng = np.random.default_rng(9)
    nx, ny, nz = 4, 4, 5
    chi = np.exp(rng.normal(0, 1, (1, nz, ny, nx)))
    S = 1 + rng.random((1, nz, ny, nx))
    P = oracle.Problem(nx, ny, nz, 1, max_wrap_iters=100000)
    c1, c2 = _cot(P, rng), _cot(P, rng)
    g1 = P.adjoint(chi, S, c1["I_top"], c1["J"], c1["F"], c1["Q"])
    g2 = P.adjoint(chi, S, c2["I_top"], c2["J"], c2["F"], c2["Q"])
    c3 = {k: 2 * c1[k] - 0.5 * c2[k] for k in c1}
    g3 = P.adjoint(chi, S, c3["I_top"], c3["J"], c3["F"], c3["Q"])
    for a, b, c in zip(g1, g2, g3):
        assert np.allclose(c, 2 * a - 0.5 * b, rtol=1e-10, atol=1e-12)


def test_adjoint_isothermal_opacity_gradient_vanishes(oracle_mod):
    """In an isothermal box with incident I = S0 the intensity is S0 for any
    opacity, so J, F and Q do not depend on chi: d/d log chi must be 0."""
    rng = np.random.default_rng(4)
    nx, ny, nz, S0 = 5, 4, 6, 1.9
    chi = np.exp(rng.normal(0, 1, (1, nz, ny, nx)))
    S = np.full_like(chi, S0)
    top = np.full((1, 12, ny, nx), S0)
    P = oracle.Problem(nx, ny, nz, 1, bottom=oracle.BC_EQUAL_S, top=oracle.BC_EXPLICIT, top_I=top)
    c = _cot(P, rng)
    glc, gS = P.adjoint(chi, S, c["I_top"], c["J"], c["F"], c["Q"])
    assert np.abs(glc).max() < 1e-10 * max(1.0, np.abs(gS).max())
    assert np.abs(gS).max() > 1e-3


def test_adjoint_source_gradient_of_mean_intensity(oracle_mod):
    """sum_p dJ(p)/dS(q) over all q equals the fraction of J that comes from
    sources: with zero incident intensity at the top and I = S at the bottom
    and S scaled uniformly, J is linear and homogeneous in S, so
    <dL/dS, S> = L for L = <gJ, J> (Euler's theorem)."""
    rng = np.random.default_rng(6)
    nx, ny, nz = 5, 5, 7
    chi = np.exp(rng.normal(0, 1, (1, nz, ny, nx)))
    S = 1 + rng.random((1, nz, ny, nx))
    P = oracle.Problem(nx, ny, nz, 1, bottom=oracle.BC_EQUAL_S, top=oracle.BC_ZERO, max_wrap_iters=100000)
    gJ = rng.normal(size=P.shape)
    gQ = rng.normal(size=P.shape)
    _, gS = P.adjoint(chi, S, None, gJ, None, gQ)
    out = P.solve(chi, S)
    L = np.sum(gJ * out["J"]) + np.sum(gQ * out["Q"])
    assert abs(np.sum(gS * S) - L) < 1e-11 * max(1.0, abs(L))
