"""GPU adjoint (rts_adjoint, reverse sweep) against the FP64 oracle's adjoint
and against central finite differences of the GPU forward solve.

Bars: FP64 path max|gpu - oracle| <= 1e-10 max|oracle| per gradient; FP32
paths <= 1e-4 max|oracle|."""
import numpy as np
import pytest

import oracle
from tests.gpu_common import norm_err, random_case, workload_inputs

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-10
FP32_TOL = 1e-4


@pytest.fixture(scope="module")
def rts():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2107_08145_b300 as m

    m.load(build_if_missing=False)
    return m


def _cotangents(B, nup, nx, ny, nz, seed, which=("I_top", "J", "F", "Q")):
    rng = np.random.default_rng(seed)
    c = dict(gI_top=rng.standard_normal((B, nup, ny, nx)), gJ=rng.standard_normal((nz, ny, nx)),
             gF=rng.standard_normal((3, nz, ny, nx)), gQ=rng.standard_normal((nz, ny, nx)))
    keep = {"I_top": "gI_top", "J": "gJ", "F": "gF", "Q": "gQ"}
    return {keep[k]: c[keep[k]] for k in which}


def _gpu_adjoint(solver, chi, S, cot, bottom="equal_s", top="zero"):
    import torch

    dt = solver.dtype
    t = lambda a, d=dt: torch.as_tensor(a, dtype=d, device="cuda")  # noqa: E731
    kw = {}
    if "gI_top" in cot:
        kw["gI_top"] = t(cot["gI_top"])
    for k in ("gJ", "gF", "gQ"):
        if k in cot:
            kw[k] = t(cot[k], torch.float64)
    b = bottom if isinstance(bottom, str) else t(bottom)
    tp = top if isinstance(top, str) else t(top)
    gl, gs = solver.adjoint(t(chi), t(S), bottom=b, top=tp, **kw)
    return gl.double().cpu().numpy(), gs.double().cpu().numpy()


def _oracle_adjoint(chi, S, cot, dx=1.0, dy=1.0, dz=1.0, bottom="equal_s", top="zero"):
    B, nz, ny, nx = chi.shape
    bk = {"equal_s": oracle.BC_EQUAL_S, "zero": oracle.BC_ZERO}
    args = {}
    if isinstance(bottom, str):
        args["bottom"] = bk[bottom]
    else:
        args.update(bottom=oracle.BC_EXPLICIT, bottom_I=bottom)
    if isinstance(top, str):
        args["top"] = bk[top]
    else:
        args.update(top=oracle.BC_EXPLICIT, top_I=top)
    P = oracle.Problem(nx, ny, nz, B, dx=dx, dy=dy, dz=dz, max_wrap_iters=100000, **args)
    return P.adjoint(chi, S, nthreads=oracle.default_threads(), **cot)


def _check(got, ref, tol, what):
    e = (norm_err(got[0], ref[0]), norm_err(got[1], ref[1]))
    assert e[0] <= tol and e[1] <= tol, (what, e)
    return e


@pytest.mark.parametrize("shape,B,spacing,chunk", [((13, 11, 9), 2, (1.0, 1.0, 1.0), 0),
                                                   ((13, 11, 9), 2, (1.0, 1.0, 1.0), 2),
                                                   ((20, 18, 16), 3, (1.0, 1.3, 0.8), 1),
                                                   ((33, 17, 12), 1, (0.7, 0.7, 1.0), 0)])
def test_adjoint_fp64_vs_oracle(rts, shape, B, spacing, chunk):
    """All four cotangents at once; ragged tiles; per-band and whole-problem checkpoints."""
    nx, ny, nz = shape
    chi, S = random_case(nx, ny, nz, B, seed=nx * 7 + ny)
    s = rts.Solver(nx, ny, nz, B, *spacing, precision="fp64", adjoint=True, adjoint_chunk_bands=chunk)
    # automatic (0): a small problem fits in one checkpoint of all bands
    assert s.stats()["adjoint_chunk_bands"] == (chunk if chunk else B)
    cot = _cotangents(B, s.n_up, nx, ny, nz, seed=5)
    got = _gpu_adjoint(s, chi, S, cot)
    ref = _oracle_adjoint(chi, S, cot, *spacing)
    _check(got, ref, FP64_TOL, shape)


@pytest.mark.parametrize("which", [("I_top",), ("J",), ("F",), ("Q",)])
def test_adjoint_fp64_each_output(rts, which):
    """One cotangent at a time (the others NULL): each transposed path alone."""
    nx, ny, nz, B = 12, 10, 14, 2
    chi, S = random_case(nx, ny, nz, B, seed=11)
    s = rts.Solver(nx, ny, nz, B, precision="fp64", adjoint=True)
    cot = _cotangents(B, s.n_up, nx, ny, nz, seed=9, which=which)
    got = _gpu_adjoint(s, chi, S, cot)
    ref = _oracle_adjoint(chi, S, cot)
    _check(got, ref, FP64_TOL, which)


def test_adjoint_fp64_thin_wrap(rts):
    """Transparent medium: the reverse periodic wrap has to work hard."""
    nx, ny, nz, B = 16, 12, 10, 1
    chi, S = random_case(nx, ny, nz, B, seed=2, thin=True)
    s = rts.Solver(nx, ny, nz, B, precision="fp64", adjoint=True)
    cot = _cotangents(B, s.n_up, nx, ny, nz, seed=3)
    got = _gpu_adjoint(s, chi, S, cot)
    ref = _oracle_adjoint(chi, S, cot)
    _check(got, ref, FP64_TOL, "thin")


def test_adjoint_fp64_explicit_boundaries(rts):
    """Explicit boundary intensities are constants; zero top and bottom."""
    nx, ny, nz, B = 12, 10, 14, 2
    chi, S = random_case(nx, ny, nz, B, seed=3)
    rng = np.random.default_rng(4)
    s = rts.Solver(nx, ny, nz, B, precision="fp64", adjoint=True)
    bot = rng.uniform(0.5, 1.5, (B, s.n_up, ny, nx))
    top = rng.uniform(0.0, 0.2, (B, 24 - s.n_up, ny, nx))
    cot = _cotangents(B, s.n_up, nx, ny, nz, seed=6)
    _check(_gpu_adjoint(s, chi, S, cot, bot, top), _oracle_adjoint(chi, S, cot, bottom=bot, top=top), FP64_TOL,
           "explicit")
    _check(_gpu_adjoint(s, chi, S, cot, "zero", "zero"), _oracle_adjoint(chi, S, cot, bottom="zero", top="zero"),
           FP64_TOL, "zero")


@pytest.mark.parametrize("precision", ["fp32", "fp32_compensated"])
@pytest.mark.parametrize("sweep,chunk", [("auto", 0), ("auto", 1), ("shared", 0)])
def test_adjoint_fp32_vs_oracle(rts, precision, sweep, chunk):
    """Both FP32 adjoint paths: on the register sweep (its checkpoint
    instantiation, the double-float reduction and Q-step transpose; with one
    band per checkpoint also the general reduction over a chunk's units) and
    on the shared-memory sweep."""
    nx, ny, nz, B = 24, 20, 18, 2
    chi, S = random_case(nx, ny, nz, B, seed=8)
    s = rts.Solver(nx, ny, nz, B, precision=precision, adjoint=True, adjoint_chunk_bands=chunk, sweep_kernel=sweep)
    st = s.stats()
    assert st["sweep_kernel"] == (rts.SWEEP_SHARED if sweep == "shared" else rts.SWEEP_REGISTER)
    if chunk:
        assert st["adjoint_chunk_bands"] == chunk
    cot = _cotangents(B, s.n_up, nx, ny, nz, seed=12)
    got = _gpu_adjoint(s, chi, S, cot)
    ref = _oracle_adjoint(chi, S, cot)
    _check(got, ref, FP32_TOL, (precision, sweep, chunk))


def test_adjoint_null_gq_equals_zero_gq(rts):
    """With gQ NULL the first forward solve is skipped; the result must be
    the same as with gQ = 0."""
    import torch

    nx, ny, nz, B = 14, 12, 10, 2
    chi, S = random_case(nx, ny, nz, B, seed=21)
    s = rts.Solver(nx, ny, nz, B, precision="fp64", adjoint=True)
    cot = _cotangents(B, s.n_up, nx, ny, nz, seed=1, which=("I_top", "J", "F"))
    a = _gpu_adjoint(s, chi, S, cot)
    cot0 = dict(cot, gQ=np.zeros((nz, ny, nx)))
    b = _gpu_adjoint(s, chi, S, cot0)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    del torch


def test_adjoint_dot_product(rts):
    """<J_F v, w> = <v, J_F^T w>: directional derivative of the GPU forward
    solve (central differences, FP64) against the GPU adjoint."""
    import torch

    nx, ny, nz, B = 10, 9, 8, 2
    chi, S = random_case(nx, ny, nz, B, seed=31)
    s = rts.Solver(nx, ny, nz, B, precision="fp64", adjoint=True)
    cot = _cotangents(B, s.n_up, nx, ny, nz, seed=2)
    gl, gs = _gpu_adjoint(s, chi, S, cot)
    rng = np.random.default_rng(7)
    vl = rng.standard_normal(chi.shape)
    vs = rng.standard_normal(S.shape)
    t = lambda a: torch.as_tensor(a, dtype=torch.float64, device="cuda")  # noqa: E731

    def L(h):
        out = s.solve(t(chi * np.exp(h * vl)), t(S + h * vs))
        o = {k: v.cpu().numpy() for k, v in out.items()}
        return (np.sum(o["I_top"] * cot["gI_top"]) + np.sum(o["J"] * cot["gJ"]) + np.sum(o["F"] * cot["gF"])
                + np.sum(o["Q"] * cot["gQ"]))

    h = 1e-5
    fd = (L(h) - L(-h)) / (2 * h)
    ad = np.sum(gl * vl) + np.sum(gs * vs)
    assert abs(fd - ad) <= 1e-7 * max(abs(ad), 1.0), (fd, ad)


def test_autograd_function_matches_adjoint(rts):
    """RTSFunction's backward is rts_adjoint: a torch loss on its outputs
    gives the gradients of the direct call."""
    import torch
    from paper_2107_08145_b300.autograd import rts_apply

    nx, ny, nz, B = 12, 12, 10, 2
    chi, S = random_case(nx, ny, nz, B, seed=41)
    s = rts.Solver(nx, ny, nz, B, precision="fp64", adjoint=True, log_chi=True)
    lc = torch.tensor(np.log(chi), device="cuda", requires_grad=True)
    St = torch.tensor(S, device="cuda", requires_grad=True)
    I_top, J, F, Q = rts_apply(s, lc, St)
    target = I_top.detach() * 1.05
    loss = ((I_top - target) ** 2).sum() + 1e-3 * (Q ** 2).sum()
    loss.backward()
    cot = dict(gI_top=(2 * (I_top - target)).detach().cpu().numpy(), gQ=(2e-3 * Q).detach().cpu().numpy())
    ref = _oracle_adjoint(chi, S, cot)
    _check((lc.grad.cpu().numpy(), St.grad.cpu().numpy()), ref, FP64_TOL, "autograd")


def _fd_case(rts, precision):
    """adj16x4: loss = sum (I_top - I_target)^2 + 1e-3 sum Q^2, I_target from
    the same atmosphere 5% hotter; central differences of the GPU forward
    solve at sampled points against the GPU adjoint."""
    import torch
    from paper_2107_08145_b300.autograd import rts_apply

    chi, S = workload_inputs("adj16x4")
    B, nz, ny, nx = chi.shape
    s = rts.Solver(nx, ny, nz, B, precision=precision, adjoint=True, log_chi=True)
    dt = s.dtype
    S_hot = S * 1.05 ** 4
    with torch.no_grad():  # the solver takes log chi
        tgt = s.solve(torch.tensor(np.log(chi), dtype=dt, device="cuda"), torch.tensor(S_hot, dtype=dt, device="cuda"))
    I_target = tgt["I_top"].clone()

    def loss_of(lc, St):
        I_top, J, F, Q = rts_apply(s, lc, St)
        return ((I_top.double() - I_target.double()) ** 2).sum() + 1e-3 * (Q ** 2).sum()

    lc = torch.tensor(np.log(chi), dtype=dt, device="cuda", requires_grad=True)
    St = torch.tensor(S, dtype=dt, device="cuda", requires_grad=True)
    loss_of(lc, St).backward()
    g_lc = lc.grad.double().cpu().numpy()
    g_S = St.grad.double().cpu().numpy()
    rng = np.random.default_rng(0)
    pts = [tuple(int(rng.integers(0, n)) for n in (B, nz, ny, nx)) for _ in range(6)]
    pts += [(1, nz - 1, 3, 4), (2, 0, 5, 5), (0, nz // 2, 0, 0)]
    errs = []
    with torch.no_grad():
        for which, g, base in (("logchi", g_lc, np.log(chi)), ("S", g_S, S)):
            for p in pts:
                h = 1e-6 * max(1.0, abs(base[p]))
                vals = []
                for sgn in (1, -1):
                    a = base.copy()
                    a[p] += sgn * h
                    lc2 = torch.tensor(a if which == "logchi" else np.log(chi), dtype=dt, device="cuda")
                    S2 = torch.tensor(a if which == "S" else S, dtype=dt, device="cuda")
                    vals.append(float(loss_of(lc2, S2)))
                fd = (vals[0] - vals[1]) / (2 * h)
                errs.append((which, p, fd, g[p]))
    return errs, g_lc, g_S


def test_adjoint_finite_differences_16(rts):
    errs, g_lc, g_S = _fd_case(rts, "fp64")
    scale = {"logchi": np.abs(g_lc).max(), "S": np.abs(g_S).max()}
    for which, p, fd, ad in errs:
        assert abs(fd - ad) <= 1e-6 * scale[which] + 1e-6 * abs(ad), (which, p, fd, ad)


@pytest.mark.slow
def test_adjoint_96x4_fp32_vs_oracle(rts):
    """The 96^3 x 4-band adjoint configuration, FP32 forward + reverse sweep,
    against the FP64 oracle adjoint (loss on I_top and Q_rad)."""
    chi, S = workload_inputs("adj96x4")
    B, nz, ny, nx = chi.shape
    s = rts.Solver(nx, ny, nz, B, precision="fp32", adjoint=True)
    rng = np.random.default_rng(3)
    cot = dict(gI_top=rng.standard_normal((B, s.n_up, ny, nx)), gQ=1e-3 * rng.standard_normal((nz, ny, nx)))
    got = _gpu_adjoint(s, chi, S, cot)
    ref = _oracle_adjoint(chi, S, cot)
    _check(got, ref, FP32_TOL, "adj96x4")
