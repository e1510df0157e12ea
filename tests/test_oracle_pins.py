"""Pins of the FP64 oracle against facts it does not compute itself.

Each test fixes a part of the oracle by something independent of its code:
published table values, closed-form solutions of the transfer equation,
invariants of the discrete scheme, a brute-force dense solve and exact
arithmetic (mpmath). A plausible slip anywhere in the oracle (a dropped term,
a wrong sign or index, a transposed operand) fails at least one of them.
"""
import math
import os

import mpmath
import numpy as np
import pytest

import oracle
from tests.dense_reference import dense_direction

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    vals = {}
    for line in open(os.path.join(GOLD, name)):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        k, v = line.split()
        vals[k] = float(v)
    return vals


# --------------------------------------------------------------------------
# Quadrature (Sect. 2 and 5.1: 3 rays per octant, 24 rays, Carlson set)
# --------------------------------------------------------------------------

def test_quadrature_matches_published_table(oracle_mod):
    n, w = oracle.a4_quadrature()
    g = _golden("carlson_s4.txt")
    comps = np.sort(np.abs(n), axis=1)
    assert np.allclose(comps[:, 0], g["mu1"], atol=5e-8)
    assert np.allclose(comps[:, 1], g["mu1"], atol=5e-8)
    assert np.allclose(comps[:, 2], g["mu2"], atol=5e-8)
    assert np.allclose(w * 8, g["weight_per_octant_direction"], atol=5e-8)


def test_quadrature_moments(oracle_mod):
    n, w = oracle.a4_quadrature()
    assert n.shape == (24, 3)
    assert abs(w.sum() - 1) < 1e-15
    assert np.allclose(np.linalg.norm(n, axis=1), 1, atol=1e-15)
    assert np.allclose((w[:, None] * n).sum(0), 0, atol=1e-16)
    M2 = np.einsum("d,da,db->ab", w, n, n)
    assert np.allclose(M2, np.eye(3) / 3, atol=1e-15)
    # level-symmetric S4: the 4th moment of each axis is exact (1/5)
    for a in range(3):
        assert abs((w * n[:, a] ** 4).sum() - 0.2) < 1e-15
    # each octant holds exactly 3 directions
    oct_ = ((n > 0) * np.array([1, 2, 4])).sum(1)
    assert sorted(np.bincount(oct_, minlength=8)) == [3] * 8


def test_quadrature_closed_under_rotation_and_mirror(oracle_mod):
    n, _ = oracle.a4_quadrature()
    key = lambda v: tuple(np.round(v, 12))  # noqa: E731
    s = {key(v) for v in n}
    rot = n[:, [1, 0, 2]] * np.array([-1, 1, 1])  # 90 deg about z: (x,y)->(-y,x)
    assert {key(v) for v in rot} == s
    for a in range(3):
        m = n.copy()
        m[:, a] *= -1
        assert {key(v) for v in m} == s


def test_quadrature_grouping(oracle_mod):
    """6 sweep groups of 4, each group sharing dominant axis and its sign."""
    P = oracle.Problem(8, 8, 8)
    for grp in range(6):
        gs = [P.geometry(4 * grp + m) for m in range(4)]
        assert len({(g.axis, g.sa) for g in gs}) == 1
    assert [P.geometry(4 * g).axis for g in range(6)] == [2, 2, 0, 0, 1, 1]


# --------------------------------------------------------------------------
# Geometry of a short characteristic
# --------------------------------------------------------------------------

def test_geometry_cube(oracle_mod):
    P = oracle.Problem(8, 8, 8)
    n, _ = oracle.a4_quadrature()
    mu1, mu2 = np.sort(np.abs(n[0]))[[0, 2]]
    for d in range(24):
        g = P.geometry(d)
        assert abs(g.ds - 1 / mu2) < 1e-15
        assert abs(g.d1 - mu1 / mu2) < 1e-15 and abs(g.d2 - mu1 / mu2) < 1e-15
        assert abs(sum(g.beta) - 1) < 1e-15
        # the upwind point r - ds*n equals the bilinear combination of corners
        c = np.zeros(3)
        c[g.axis] -= g.sa
        pt = -g.ds * n[d]
        corners = []
        for q in range(4):
            u = c.copy()
            if q & 1:
                u[g.b1] -= g.s1
            if q & 2:
                u[g.b2] -= g.s2
            corners.append(u)
        assert np.allclose(sum(b * u for b, u in zip(g.beta, corners)), pt, atol=1e-15)


def test_geometry_anisotropic_spacing(oracle_mod):
    # tall cells: a 'z-type' direction becomes x- or y-dominant
    P = oracle.Problem(8, 8, 8, dz=4.0)
    n, _ = oracle.a4_quadrature()
    for d in range(24):
        g = P.geometry(d)
        h = np.array([1.0, 1.0, 4.0])
        s = h / np.maximum(np.abs(n[d]), 1e-300)
        assert g.axis == int(np.argmin(s)) or abs(s[g.axis] - s.min()) < 1e-15
        assert 0 <= g.d1 <= 1 and 0 <= g.d2 <= 1


# --------------------------------------------------------------------------
# Segment weights: exact arithmetic
# --------------------------------------------------------------------------

@pytest.mark.parametrize("x", [0.0, 1e-9, 1e-5, 3e-3, 0.00999, 0.01, 0.01001, 0.05, 0.3, 1.0, 3.0, 20.0, 200.0])
def test_segment_weights_exact(oracle_mod, x):
    mpmath.mp.dps = 50
    e, wu, wp = oracle.segment_weights(x)
    X = mpmath.mpf(x)
    E = mpmath.e ** (-X)
    if x == 0:
        WU = WP = mpmath.mpf(0)
    else:
        WU = (1 - E) / X - E
        WP = 1 - (1 - E) / X
    # e to a few ulp; the weights to ~1e-16 absolute: they multiply S values
    # of the same scale as I (e + w_up + w_p = 1), so an absolute bound is the
    # one that reaches the intensity. Just above the series switch the direct
    # formula 1 - (1-e)/x cancels two digits, which this bound allows.
    assert abs(e - float(E)) <= 4e-16 * float(E) + 1e-300
    for got, ref in ((wu, WU), (wp, WP)):
        ref = float(ref)
        assert abs(got - ref) <= 1e-16 + 4e-16 * abs(ref)
    assert abs(e + wu + wp - 1) < 4e-16


def test_segment_weights_integral(oracle_mod):
    """w_up, w_p are the integral of a linear source against e^{-(x-t)}."""
    mpmath.mp.dps = 40
    for x in (0.004, 0.7, 5.0):
        e, wu, wp = oracle.segment_weights(x)
        # S(t) = 1 at the upwind end, 0 at the point -> integral = w_up
        ref_u = mpmath.quad(lambda t: (1 - t / x) * mpmath.e ** (-(x - t)), [0, x])
        ref_p = mpmath.quad(lambda t: (t / x) * mpmath.e ** (-(x - t)), [0, x])
        assert abs(wu - float(ref_u)) < 1e-15 * max(1.0, float(ref_u))
        assert abs(wp - float(ref_p)) < 1e-15 * max(1.0, float(ref_p))


# --------------------------------------------------------------------------
# Closed-form solutions (horizontally uniform atmosphere)
# --------------------------------------------------------------------------

def _uniform(nx, ny, nz, c, a, b, dz=1.0):
    z = np.arange(nz) * dz
    tau = c * (z[-1] - z)
    chi = np.full((1, nz, ny, nx), c)
    S = np.broadcast_to((a + b * tau)[None, :, None, None], (1, nz, ny, nx)).copy()
    return chi, S, tau


@pytest.mark.parametrize("c", [0.05, 0.4, 2.0])
def test_closed_form_up_rays(oracle_mod, c):
    """S = a + b tau, chi = c: the upward intensity is a + b (tau + mu) at every
    level, so I_top(mu) = a + b mu (exact for the linear-in-tau scheme)."""
    nx, ny, nz, a, b = 6, 5, 24, 1.3, 0.7
    chi, S, tau = _uniform(nx, ny, nz, c, a, b)
    n, w = oracle.a4_quadrature()
    up = np.where(n[:, 2] > 0)[0]
    bot = np.zeros((1, len(up), ny, nx))
    for u, d in enumerate(up):
        bot[0, u] = a + b * (tau[0] + n[d, 2])
    P = oracle.Problem(nx, ny, nz, 1, bottom=oracle.BC_EXPLICIT, bottom_I=bot, top=oracle.BC_ZERO,
                       max_wrap_iters=2000)
    out = P.solve(chi, S)
    for u, d in enumerate(up):
        assert np.allclose(out["I_top"][0, u], a + b * n[d, 2], rtol=0, atol=1e-13)
        I, _ = P.sweep(0, d, chi[0], S[0])
        ref = a + b * (tau[:, None, None] + n[d, 2])
        assert np.allclose(I, ref, rtol=0, atol=1e-13)


@pytest.mark.parametrize("c", [0.1, 1.0])
def test_closed_form_down_z_rays(oracle_mod, c):
    """z-dominant down rays with zero incident intensity match the exact
    I(tau, mu) = a(1 - e^{-tau/mu}) + b[tau - mu(1 - e^{-tau/mu})]."""
    nx, ny, nz, a, b = 4, 4, 20, 0.8, 1.5
    chi, S, tau = _uniform(nx, ny, nz, c, a, b)
    P = oracle.Problem(nx, ny, nz, 1, bottom=oracle.BC_EQUAL_S, top=oracle.BC_ZERO)
    n, _ = oracle.a4_quadrature()
    for d in range(24):
        g = P.geometry(d)
        if g.axis != 2 or g.up:
            continue
        mu = abs(n[d, 2])
        I, _ = P.sweep(0, d, chi[0], S[0])
        E = np.exp(-tau / mu)
        ref = a * (1 - E) + b * (tau - mu * (1 - E))
        assert np.allclose(I, ref[:, None, None], rtol=0, atol=2e-14)


def test_down_xy_rays_converge_first_order(oracle_mod):
    """x/y-dominant down rays interpolate a curved intensity profile between
    levels. Each step commits an O(h^2) interpolation error and crossing a
    fixed optical depth takes O(1/h) steps, so at fixed total optical depth
    the largest error must halve with the grid spacing (first order
    globally). A wrong corner, weight or sign would not converge at all."""
    n, _ = oracle.a4_quadrature()
    d = 8 + 2  # +x group, (+y, -z) minor signs: a down ray
    mu = abs(n[d, 2])
    errs = []
    for nz in (16, 32, 64, 128):
        c = 4.0 / (nz - 1)  # total optical depth 4 along z
        chi, S, tau = _uniform(3, 3, nz, c, 1.0, 1.0)
        P = oracle.Problem(3, 3, nz, 1, top=oracle.BC_ZERO, max_wrap_iters=5000)
        assert P.geometry(d).axis == 0 and not P.geometry(d).up
        I, _ = P.sweep(0, d, chi[0], S[0])
        E = np.exp(-tau / mu)
        ref = (1 - E) + (tau - mu * (1 - E))
        errs.append(np.abs(I[:, 0, 0] - ref).max())
    ratios = [errs[i] / errs[i + 1] for i in range(3)]
    assert all(1.6 < r < 2.3 for r in ratios), (errs, ratios)
    assert errs[-1] < 1e-2


# --------------------------------------------------------------------------
# Invariants of the discrete scheme
# --------------------------------------------------------------------------

def test_isothermal_box_any_opacity(oracle_mod):
    """S = S0 everywhere and incident I = S0 on both boundaries: I = S0 for
    any opacity field, so J = S0, F = 0 and Q_rad = 0."""
    rng = np.random.default_rng(3)
    nx, ny, nz, S0 = 7, 6, 9, 2.5
    chi = np.exp(rng.normal(0, 1.5, (2, nz, ny, nx)))
    S = np.full_like(chi, S0)
    nup = 12
    top = np.full((2, 24 - nup, ny, nx), S0)
    P = oracle.Problem(nx, ny, nz, 2, bottom=oracle.BC_EQUAL_S, top=oracle.BC_EXPLICIT, top_I=top)
    out = P.solve(chi, S, debug=True)
    assert np.allclose(out["I_top"], S0, atol=1e-13)
    assert np.allclose(out["J"], 2 * S0, atol=1e-13)
    assert np.allclose(out["F"], 0, atol=1e-12)
    assert np.allclose(out["Q"], 0, atol=1e-10)


def test_isothermal_thick_box_top_zero(oracle_mod):
    """With zero incident intensity at the top, deep inside an optically
    thick isothermal box I ~ S and Q_rad ~ 0."""
    nx, ny, nz, S0 = 4, 4, 40, 1.7
    chi = np.full((1, nz, ny, nx), 5.0)
    S = np.full_like(chi, S0)
    P = oracle.Problem(nx, ny, nz, 1, top=oracle.BC_ZERO)
    out = P.solve(chi, S, debug=True)
    deep = slice(0, nz - 8)  # > 30 optical depths below the top
    assert np.allclose(out["J"][deep], S0, rtol=1e-12)
    assert np.abs(out["Q"][deep]).max() <= 1e-10 * 4 * np.pi * 5.0 * S0


def test_transparent_medium(oracle_mod):
    """chi = 0: intensity is constant along rays. Up rays carry the bottom
    value s0, down rays carry 0: J = s0/2, F_z = 4 pi s0 sum_up w n_z, Q = 0."""
    nx, ny, nz, s0 = 5, 4, 12, 1.25
    chi = np.zeros((1, nz, ny, nx))
    S = np.full_like(chi, s0)
    P = oracle.Problem(nx, ny, nz, 1, bottom=oracle.BC_EQUAL_S, top=oracle.BC_ZERO, max_wrap_iters=5000)
    out = P.solve(chi, S, debug=True)
    n, w = oracle.a4_quadrature()
    fz = 4 * np.pi * s0 * (w * n[:, 2] * (n[:, 2] > 0)).sum()
    assert abs(fz / (4 * np.pi * s0) - 0.2614888) < 1e-7
    assert np.allclose(out["J"], s0 / 2, atol=1e-14)
    assert np.allclose(out["F"][2], fz, atol=1e-13)
    assert np.allclose(out["F"][:2], 0, atol=1e-14)
    assert np.allclose(out["I_top"], s0, atol=1e-14)
    assert np.allclose(out["Q"], 0, atol=1e-12)


def test_horizontal_symmetry_uniform(oracle_mod):
    """Horizontally uniform input: directions related by 90-degree rotation
    about z give the same intensity at every level."""
    rng = np.random.default_rng(5)
    nx = ny = 5
    nz = 14
    prof_c = np.exp(rng.normal(0, 0.7, nz))
    prof_s = 1 + rng.random(nz)
    chi = np.broadcast_to(prof_c[:, None, None], (nz, ny, nx)).copy()
    S = np.broadcast_to(prof_s[:, None, None], (nz, ny, nx)).copy()
    P = oracle.Problem(nx, ny, nz, 1, max_wrap_iters=5000)
    n, _ = oracle.a4_quadrature()
    Is = [P.sweep(0, d, chi, S)[0] for d in range(24)]
    for d in range(24):
        r = np.array([-n[d, 1], n[d, 0], n[d, 2]])
        e = int(np.argmin(np.linalg.norm(n - r, axis=1)))
        assert np.allclose(n[e], r, atol=1e-14)
        assert np.allclose(Is[d], Is[e], rtol=1e-13, atol=1e-14)


def test_rotation_covariance(oracle_mod):
    """Rotating chi and S by 90 degrees about z rotates J and Q and turns F as
    a vector; mirroring x flips F_x."""
    rng = np.random.default_rng(11)
    nx = ny = 6
    nz = 8
    chi = np.exp(rng.normal(0, 0.8, (1, nz, ny, nx)))
    S = 1 + rng.random((1, nz, ny, nx))
    P = oracle.Problem(nx, ny, nz, 1, max_wrap_iters=5000)
    base = P.solve(chi, S)
    # rotation (x, y) -> (-y, x): new[j', i'] with i' = -j, j' = i
    rot = lambda a: np.rot90(a, k=1, axes=(-1, -2))  # noqa: E731
    out = P.solve(np.ascontiguousarray(rot(chi)), np.ascontiguousarray(rot(S)))
    assert np.allclose(out["J"], rot(base["J"]), rtol=1e-12, atol=1e-13)
    assert np.allclose(out["Q"], rot(base["Q"]), rtol=1e-11, atol=1e-12)
    Fx, Fy, Fz = (rot(base["F"][a]) for a in range(3))
    assert np.allclose(out["F"][0], -Fy, rtol=1e-11, atol=1e-12)
    assert np.allclose(out["F"][1], Fx, rtol=1e-11, atol=1e-12)
    assert np.allclose(out["F"][2], Fz, rtol=1e-11, atol=1e-12)
    mir = lambda a: a[..., ::-1]  # noqa: E731  i -> -i  (periodic: index nx-1-i)
    out = P.solve(np.ascontiguousarray(mir(chi)), np.ascontiguousarray(mir(S)))
    assert np.allclose(out["J"], mir(base["J"]), rtol=1e-12, atol=1e-13)
    assert np.allclose(out["F"][0], -mir(base["F"][0]), rtol=1e-11, atol=1e-12)
    assert np.allclose(out["F"][1], mir(base["F"][1]), rtol=1e-11, atol=1e-12)


# --------------------------------------------------------------------------
# Brute force: dense solve of the periodic linear system
# --------------------------------------------------------------------------

@pytest.mark.parametrize("shape", [(2, 3, 4), (3, 3, 3), (4, 2, 5)])
def test_sweep_equals_dense_solve(oracle_mod, shape):
    nx, ny, nz = shape
    rng = np.random.default_rng(sum(shape))
    chi = np.exp(rng.normal(0, 0.8, (nz, ny, nx))) * 0.5
    S = 0.5 + rng.random((nz, ny, nx))
    bot = rng.random((1, 12, ny, nx))
    top = rng.random((1, 12, ny, nx))
    P = oracle.Problem(nx, ny, nz, 1, dx=1.0, dy=1.3, dz=0.9, bottom=oracle.BC_EXPLICIT, bottom_I=bot,
                       top=oracle.BC_EXPLICIT, top_I=top, max_wrap_iters=100000)
    n, _ = oracle.a4_quadrature()
    up = [d for d in range(24) if n[d, 2] > 0]
    dn = [d for d in range(24) if n[d, 2] < 0]
    for d in range(24):
        I, _ = P.sweep(0, d, chi, S)
        if n[d, 2] > 0:
            bv = lambda i, j, u=up.index(d): bot[0, u, j, i]  # noqa: E731
        else:
            bv = lambda i, j, u=dn.index(d): top[0, u, j, i]  # noqa: E731
        ref = dense_direction(n[d], (1.0, 1.3, 0.9), chi, S, bv)
        assert np.allclose(I, ref, rtol=1e-14, atol=1e-14), (d, np.abs(I - ref).max())


def test_solve_outputs_from_dense(oracle_mod):
    """J, F, I_top and Q of the full solve, rebuilt from dense per-direction
    solutions with the definitions J = sum w I, F = 4 pi sum w n I and the
    Q blend."""
    nx, ny, nz = 3, 4, 5
    rng = np.random.default_rng(7)
    chi = np.exp(rng.normal(0, 1.0, (1, nz, ny, nx)))
    S = 0.5 + rng.random((1, nz, ny, nx))
    P = oracle.Problem(nx, ny, nz, 1, bottom=oracle.BC_EQUAL_S, top=oracle.BC_ZERO, max_wrap_iters=100000)
    out = P.solve(chi, S, debug=True)
    n, w = oracle.a4_quadrature()
    J = np.zeros((nz, ny, nx))
    F = np.zeros((3, nz, ny, nx))
    Itop = []
    for d in range(24):
        bv = (lambda i, j: S[0, 0, j, i]) if n[d, 2] > 0 else (lambda i, j: 0.0)
        I = dense_direction(n[d], (1.0, 1.0, 1.0), chi[0], S[0], bv)
        J += w[d] * I
        F += 4 * np.pi * w[d] * n[d][:, None, None, None] * I
        if n[d, 2] > 0:
            Itop.append(I[-1])
    assert np.allclose(out["J"], J, rtol=1e-13)
    assert np.allclose(out["F"], F, rtol=1e-12, atol=1e-13)
    assert np.allclose(out["I_top"][0], np.array(Itop), rtol=1e-13)
    # Q: thin/thick blend of 4 pi chi (J - S) and -div F (own stencil here)
    Fx, Fy, Fz = F
    div = (np.roll(Fx, -1, 2) - np.roll(Fx, 1, 2)) / 2 + (np.roll(Fy, -1, 1) - np.roll(Fy, 1, 1)) / 2
    dz = np.empty_like(Fz)
    dz[1:-1] = (Fz[2:] - Fz[:-2]) / 2
    dz[0] = Fz[1] - Fz[0]
    dz[-1] = Fz[-1] - Fz[-2]
    om = np.exp(-chi[0] * 1.0 / 0.1)
    Q = om * 4 * np.pi * chi[0] * (J - S[0]) + (1 - om) * (-(div + dz))
    assert np.allclose(out["Q"], Q, rtol=1e-11, atol=1e-12)


# --------------------------------------------------------------------------
# Q step stencil
# --------------------------------------------------------------------------

def test_divergence_exact_on_polynomials(oracle_mod):
    """Central differences are exact on quadratics (interior and periodic
    trigonometric fields); the one-sided ends are exact on linear fields."""
    nx, ny, nz = 8, 6, 7
    dx, dy, dz = 0.5, 2.0, 1.5
    k = np.arange(nz)[:, None, None] * dz
    j = np.arange(ny)[None, :, None] * dy
    i = np.arange(nx)[None, None, :] * dx
    Lx, Ly = nx * dx, ny * dy
    F = np.zeros((3, nz, ny, nx))
    F[0] = np.sin(2 * np.pi * i / Lx) + 0 * j + 0 * k
    F[1] = np.cos(2 * np.pi * j / Ly) * (1 + 0 * i) + 0 * k
    F[2] = 3.0 + 2.0 * k + 0.25 * k ** 2 + 0 * i + 0 * j
    nd = oracle.neg_divergence(F, dx, dy, dz)
    dFx = (np.sin(2 * np.pi * (i + dx) / Lx) - np.sin(2 * np.pi * (i - dx) / Lx)) / (2 * dx)
    dFy = (np.cos(2 * np.pi * (j + dy) / Ly) - np.cos(2 * np.pi * (j - dy) / Ly)) / (2 * dy)
    dFz = 2.0 + 0.5 * k  # exact derivative of the quadratic (interior)
    ref = -(dFx + dFy + dFz)
    assert np.allclose(nd[1:-1], np.broadcast_to(ref, nd.shape)[1:-1], atol=1e-12)
    # ends: first-order one-sided differences
    kk = np.arange(nz) * dz
    fz = 3.0 + 2.0 * kk + 0.25 * kk ** 2
    bot = -(dFx + dFy)[0] - (fz[1] - fz[0]) / dz
    topv = -(dFx + dFy)[0] - (fz[-1] - fz[-2]) / dz
    assert np.allclose(nd[0], bot, atol=1e-12)
    assert np.allclose(nd[-1], topv, atol=1e-12)


# --------------------------------------------------------------------------
# Periodic wrap: result independent of the tolerance / thread count
# --------------------------------------------------------------------------

def test_threads_do_not_change_result(oracle_mod):
    from workloads import workload

    chi, S = workload("adj16x4")
    P = oracle.Problem(16, 16, 16, 4)
    a = P.solve(chi, S, nthreads=1)
    b = P.solve(chi, S, nthreads=5)
    for k in ("J", "F", "Q", "I_top"):
        assert np.array_equal(a[k], b[k])


def test_wrap_iteration_converged(oracle_mod):
    from workloads import workload

    chi, S = workload("gray32")
    P1 = oracle.Problem(32, 32, 32, 1, wrap_tol=1e-15)
    P2 = oracle.Problem(32, 32, 32, 1, wrap_tol=1e-9)
    a = P1.solve(chi, S)
    b = P2.solve(chi, S)
    assert (a["wrap_iters"][0, 8:] >= b["wrap_iters"][0, 8:]).all()
    assert np.allclose(a["J"], b["J"], rtol=1e-8)
    assert (a["wrap_iters"][0, :8] == 1).all()


def test_nonconvergence_reported(oracle_mod):
    chi = np.zeros((1, 30, 4, 4))
    S = np.ones_like(chi)
    P = oracle.Problem(4, 4, 30, 1, max_wrap_iters=2)
    with pytest.raises(oracle.OracleError) as ei:
        P.solve(chi, S)
    assert ei.value.code == oracle.ENOCONV


def test_invalid_problem_rejected(oracle_mod):
    n = np.array([[1.0, 0.0, 0.0]])  # horizontal ray: neither up nor down
    P = oracle.Problem(4, 4, 4, 1, n=n, w=np.array([1.0]))
    with pytest.raises(oracle.OracleError):
        P.solve(np.ones((1, 4, 4, 4)), np.ones((1, 4, 4, 4)))


def test_exact_value_from_math(oracle_mod):
    """one cell column, one z ray: hand-derived single-step formula."""
    n = np.array([[0.0, 0.0, 1.0]])
    P = oracle.Problem(1, 1, 2, 1, n=n, w=np.array([1.0]), bottom=oracle.BC_EXPLICIT,
                       bottom_I=np.array([[[[3.0]]]]))
    chi = np.array([[[[2.0]], [[4.0]]]])
    S = np.array([[[[1.0]], [[5.0]]]])
    I, _ = P.sweep(0, 0, chi[0], S[0])
    x = 1.0 * (2.0 + 4.0) / 2
    e = math.exp(-x)
    wu = (1 - e) / x - e
    wp = 1 - (1 - e) / x
    assert abs(I[1, 0, 0] - (e * 3.0 + wu * 1.0 + wp * 5.0)) < 1e-15
