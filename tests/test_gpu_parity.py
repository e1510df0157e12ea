"""GPU parity: the CUDA library (through its C ABI) against the FP64 oracle.

Bars: FP64 path element-wise, |gpu - oracle| <= 1e-12 (|oracle| + floor) at
every point of every output, the floor being the size of the terms the
output is formed from (tests.gpu_common.elementwise_floors); FP32 paths
max|gpu - oracle| <= 1e-5 max|oracle| per output (I_top, J, F, Q_rad)."""
import numpy as np
import pytest

from tests.gpu_common import (OUTPUTS, elementwise_err, elementwise_floors, gpu_solve, norm_err, oracle_solve,
                               random_case, workload_inputs)

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12
FP32_TOL = 1e-5


@pytest.fixture(scope="module")
def rts():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2107_08145_b300 as m

    m.load(build_if_missing=False)
    return m


def _compare(got, ref, tol, what=""):
    errs = {k: norm_err(got[k], ref[k]) for k in OUTPUTS}
    assert all(e <= tol for e in errs.values()), (what, errs)
    return errs


def _compare64(got, ref, chi, S, what="", spacing=(1.0, 1.0, 1.0)):
    """The FP64 bar, element-wise (see the module docstring)."""
    fl = elementwise_floors(ref, chi, S, min(spacing))
    errs = {k: elementwise_err(got[k], ref[k], fl[k]) for k in OUTPUTS}
    assert all(e <= FP64_TOL for e in errs.values()), (what, errs)
    return errs


def test_gray32_fp64(rts):
    """32^3, one band, FP64, bottom I = S, top I = 0, periodic."""
    chi, S = workload_inputs("gray32")
    s = rts.Solver(32, 32, 32, 1, precision="fp64")
    got = gpu_solve(s, chi, S)
    ref = oracle_solve(chi, S)
    _compare64(got, ref, chi, S, "gray32")


@pytest.mark.parametrize("shape,B,spacing", [((5, 7, 9), 2, (1.0, 1.0, 1.0)),
                                             ((13, 11, 6), 3, (1.0, 1.3, 0.8)),
                                             ((33, 17, 20), 2, (1.0, 1.0, 1.0)),
                                             ((40, 40, 35), 1, (0.7, 0.7, 1.0))])
def test_ragged_fp64(rts, shape, B, spacing):
    """Odd sizes that leave ragged last tiles, anisotropic spacing."""
    nx, ny, nz = shape
    chi, S = random_case(nx, ny, nz, B, seed=nx + ny)
    s = rts.Solver(nx, ny, nz, B, *spacing, precision="fp64")
    got = gpu_solve(s, chi, S)
    ref = oracle_solve(chi, S, *spacing)
    _compare64(got, ref, chi, S, shape, spacing)


@pytest.mark.parametrize("prec,tol", [("fp64", FP64_TOL), ("fp32", FP32_TOL)])
def test_quadrature_with_empty_slots(rts, prec, tol):
    """A 19-ray subset of the default set: five direction groups keep only 3
    of their 4 sign slots, so those sweep units run with an empty slot."""
    import oracle

    n, w = oracle.a4_quadrature()
    keep = [d for d in range(24) if d not in (1, 6, 11, 12, 21)]
    n, w = np.ascontiguousarray(n[keep]), np.ascontiguousarray(w[keep] / w[keep].sum())
    nx, ny, nz, B = 20, 18, 16, 2
    chi, S = random_case(nx, ny, nz, B, seed=11)
    s = rts.Solver(nx, ny, nz, B, precision=prec, n=n, w=w)
    got = gpu_solve(s, chi, S)
    ref = oracle_solve(chi, S, n=n, w=w)
    if prec == "fp64":
        _compare64(got, ref, chi, S, "19 rays")
    else:
        _compare(got, ref, tol, "19 rays")


def test_explicit_boundaries_fp64(rts):
    nx, ny, nz, B = 12, 10, 14, 2
    chi, S = random_case(nx, ny, nz, B, seed=3)
    rng = np.random.default_rng(1)
    bot = 1 + rng.random((B, 12, ny, nx))
    top = 0.1 * rng.random((B, 12, ny, nx))
    s = rts.Solver(nx, ny, nz, B, precision="fp64")
    got = gpu_solve(s, chi, S, bottom=bot, top=top)
    ref = oracle_solve(chi, S, bottom=bot, top=top)
    _compare64(got, ref, chi, S, "explicit")


def test_thin_atmosphere_wrap_fp64(rts):
    """Optically thin medium: many periods of warm-up for the x/y groups."""
    nx, ny, nz, B = 16, 16, 24, 1
    chi, S = random_case(nx, ny, nz, B, seed=5, thin=True)
    s = rts.Solver(nx, ny, nz, B, precision="fp64", max_wrap_iters=256)
    got = gpu_solve(s, chi, S)
    st = s.stats()
    assert st["max_warmup_steps"] > nx  # really went around the period
    ref = oracle_solve(chi, S)
    _compare64(got, ref, chi, S, "thin")


@pytest.mark.parametrize("prec", ["fp32", "fp32_compensated"])
def test_gray32_fp32(rts, prec):
    chi, S = workload_inputs("gray32")
    s = rts.Solver(32, 32, 32, 1, precision=prec)
    got = gpu_solve(s, chi.astype(np.float32), S.astype(np.float32))
    ref = oracle_solve(chi.astype(np.float32), S.astype(np.float32))
    _compare(got, ref, FP32_TOL, prec)


@pytest.mark.parametrize("prec", ["fp32", "fp32_compensated"])
def test_four_band_fp32(rts, prec):
    """The 4-band opacity set of the 288^3 case on a 48^3 grid."""
    chi, S = workload_inputs("rts288x4", nx=48, ny=48, nz=48)
    chi32, S32 = chi.astype(np.float32), S.astype(np.float32)
    s = rts.Solver(48, 48, 48, 4, precision=prec)
    got = gpu_solve(s, chi32, S32)
    ref = oracle_solve(chi32, S32)
    _compare(got, ref, FP32_TOL, prec)


def test_isothermal_box_any_size(rts):
    """I = S0 everywhere for any opacity when S = S0 and both boundaries
    carry S0: holds at any size, checked on the full 288^3 x 4 workload."""
    import torch

    chi, _ = workload_inputs("rts288x4")
    B, nz, ny, nx = chi.shape
    S0 = 1.7
    s = rts.Solver(nx, ny, nz, B, precision="fp32")
    c = torch.as_tensor(chi, dtype=torch.float32, device="cuda")
    S = torch.full_like(c, S0)
    top = torch.full((B, 12, ny, nx), S0, dtype=torch.float32, device="cuda")
    out = s.solve(c, S, bottom="equal_s", top=top)
    assert torch.allclose(out["I_top"], torch.tensor(S0, device="cuda"), rtol=1e-6, atol=0)
    assert torch.allclose(out["J"], torch.tensor(B * S0, dtype=torch.float64, device="cuda"), rtol=1e-6, atol=0)
    assert out["F"].abs().max().item() <= 1e-5 * B * S0
    # 4 pi chi (J - S) with chi up to ~1e3 per band: relative to 4 pi chi S
    assert out["Q"].abs().max().item() <= 1e-4 * 4 * np.pi * 1.5e3 * S0


@pytest.mark.slow
def test_full_288x4_fp32_vs_oracle(rts):
    """The full 288^3 x 4-band workload in the configuration the benchmark
    times, against the FP64 oracle (OpenMP over directions)."""
    chi, S = workload_inputs("rts288x4")
    chi32, S32 = chi.astype(np.float32), S.astype(np.float32)
    s = rts.Solver(288, 288, 288, 4, precision="fp32")
    got = gpu_solve(s, chi32, S32)
    ref = oracle_solve(chi32, S32)
    _compare(got, ref, FP32_TOL, "288x4")


def test_host_io_matches_device(rts):
    chi, S = workload_inputs("gray32")
    s = rts.Solver(32, 32, 32, 1, precision="fp64", host_io=True)
    dev = gpu_solve(s, chi, S)
    host = s.solve_host(chi, S)
    for k in OUTPUTS:
        assert np.array_equal(dev[k], host[k]), k


def test_host_io_async_pipeline(rts):
    """rts_solve_host_async: four solves in flight on two staging sets, each
    with its own inputs and output buffers, equal the device solves."""
    import torch

    nx, ny, nz, B = 24, 20, 18, 2
    chi, S = random_case(nx, ny, nz, B, seed=4)
    s = rts.Solver(nx, ny, nz, B, precision="fp32", host_io_async=True)
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()  # noqa: E731
    ins, outs, refs = [], [], []
    for i in range(4):
        c = pin(chi.astype(np.float32) * (1.0 + 0.1 * i))
        sv = pin(S.astype(np.float32))
        ins.append((c, sv))
        outs.append(dict(I_top=pin(np.zeros((B, s.n_up, ny, nx), np.float32)), J=pin(np.zeros((nz, ny, nx))),
                         F=pin(np.zeros((3, nz, ny, nx))), Q=pin(np.zeros((nz, ny, nx)))))
        refs.append(gpu_solve(s, c, sv))
    for (c, sv), o in zip(ins, outs):
        s.solve_host_async(c, sv, o)
    s.host_wait()
    for o, r in zip(outs, refs):
        for k in OUTPUTS:
            assert np.array_equal(o[k], r[k]), k


def test_repeat_solves_identical(rts):
    """The schedule is dynamic (atomic tickets) but the arithmetic of each
    point is fixed: repeated solves are bitwise identical."""
    chi, S = random_case(24, 20, 18, 2, seed=9)
    s = rts.Solver(24, 20, 18, 2, precision="fp32")
    a = gpu_solve(s, chi.astype(np.float32), S.astype(np.float32))
    b = gpu_solve(s, chi.astype(np.float32), S.astype(np.float32))
    for k in OUTPUTS:
        assert np.array_equal(a[k], b[k]), k


def test_nonconvergence_reported(rts):
    """Transparent medium with a warm-up cap of one period: RTS_ENOCONV."""
    import torch

    s = rts.Solver(8, 8, 40, 1, precision="fp64", max_wrap_iters=1)
    c = torch.zeros((1, 40, 8, 8), dtype=torch.float64, device="cuda")
    S = torch.ones_like(c)
    with pytest.raises(rts.RTSError) as ei:
        s.solve(c, S)
    assert ei.value.code == rts.RTS_ENOCONV
    # the handle stays usable: an optically thick medium converges at once
    out = s.solve(c + 20.0, S)
    assert torch.isfinite(out["J"]).all()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_nonfinite_input_is_reported(rts, prec):
    """A NaN or an infinity in chi or S is found on the device and reported
    as RTS_ENONFINITE (with and without x-dominant rays, whose transposed
    copy otherwise does the check); the handle stays usable."""
    import oracle

    nx, ny, nz, B = 12, 10, 9, 2
    chi, S = random_case(nx, ny, nz, B, seed=9)
    n, w = oracle.a4_quadrature()
    zonly = [d for d in range(24) if abs(n[d][2]) > 0.8]  # the z-dominant rays only: no transposed copy
    for quad in (None, (np.ascontiguousarray(n[zonly]), np.ascontiguousarray(w[zonly] / w[zonly].sum()))):
        kw = {} if quad is None else dict(n=quad[0], w=quad[1])
        s = rts.Solver(nx, ny, nz, B, precision=prec, **kw)
        for arr, bad in ((0, np.nan), (1, np.inf)):
            c, S2 = chi.copy(), S.copy()
            (c if arr == 0 else S2)[1, 3, 4, 5] = bad
            with pytest.raises(rts.RTSError) as e:
                gpu_solve(s, c, S2)
            assert e.value.code == rts.RTS_ENONFINITE, e.value
        got = gpu_solve(s, chi, S)  # a clean solve afterwards
        assert all(np.isfinite(got[k]).all() for k in OUTPUTS)


def test_log_chi_flag_matches_chi(rts):
    """RTS_FLAG_LOG_CHI: the library forms chi = exp(log chi) itself; the
    solve equals the one on chi to the rounding of exp."""
    import torch

    nx, ny, nz, B = 14, 12, 10, 2
    chi, S = random_case(nx, ny, nz, B, seed=13)
    for prec, tol in (("fp64", 1e-13), ("fp32", 2e-6)):
        a = rts.Solver(nx, ny, nz, B, precision=prec)
        b = rts.Solver(nx, ny, nz, B, precision=prec, log_chi=True)
        dt = a.dtype
        ga = a.solve(torch.tensor(chi, dtype=dt, device="cuda"), torch.tensor(S, dtype=dt, device="cuda"))
        gb = b.solve(torch.log(torch.tensor(chi, dtype=dt, device="cuda")), torch.tensor(S, dtype=dt, device="cuda"))
        for k in OUTPUTS:
            assert norm_err(gb[k].double().cpu().numpy(), ga[k].double().cpu().numpy()) <= tol, (prec, k)


def test_device_code_version(rts):
    assert rts.device_code_version() == 103
