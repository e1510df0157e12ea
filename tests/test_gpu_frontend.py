"""GPU parity of the input step (rts_front_end: trilinear MHD -> RTS
interpolation and the band-table lookup) against the FP64 oracle, element
by element: FP64 to 1e-12 relative; FP32 to 16 eps (1 + |ln v| + |ln rho| +
4 |ln T|) relative with eps = 2^-24 and rho, T the interpolated fields:
v = exp(ln v) is formed from FP32 logarithms, each rounded relative to its
own size, and the table's ln kappa carries ln T with slope up to ~3 (chi and
S are positive).
Grids with a ragged last CTA, several staggers, a table that the
atmosphere overruns (clamping), and the 288^3 x 4 band case; for the tiled
FP32 kernel also a single level, a 1 x 1 plane and shifts of several
periods (the footprint wraps more than once)."""
import numpy as np
import pytest

from oracle.frontend import front_end as oracle_front_end
from oracle.frontend import trilinear_log
from workloads.opacity import mhd_fields, synthetic_table

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rts():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2107_08145_b300 as m

    m.load(build_if_missing=False)
    return m


def _rel(got, ref):
    return float(np.max(np.abs(got - ref) / np.abs(ref)))


def _fp32_ok(got, ref, lnT, lnR):
    bound = 16 * 2.0 ** -24 * (1 + np.abs(np.log(ref)) + np.abs(lnR)[None] + 4 * np.abs(lnT)[None])
    return bool(np.all(np.abs(got - ref) <= bound * np.abs(ref)))


@pytest.mark.parametrize("shape,shift,nb", [((13, 11, 9), (-0.5, -0.5, -0.5), 3), ((32, 24, 20), (0.25, -0.75, 0.4), 4),
                                            ((7, 5, 3), (-1.5, 2.5, -0.5), 1)])
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", None)])
def test_front_end_matches_oracle(rts, shape, shift, nb, prec, tol):
    import torch

    nx, ny, nz = shape
    T, rho = mhd_fields(nx, ny, nz, seed=nx)
    tab = synthetic_table(nb=nb, nT=40, nR=30, lnR_range=(-4.0, 2.0))  # the densest/thinnest points clamp
    dt = torch.float64 if prec == "fp64" else torch.float32
    chi, S = rts.front_end(torch.tensor(T, dtype=dt, device="cuda"), torch.tensor(rho, dtype=dt, device="cuda"),
                           tab, precision=prec, shift=shift)
    T_in, r_in = (T, rho) if prec == "fp64" else (T.astype(np.float32), rho.astype(np.float32))
    tab_in = dict(tab)
    if prec != "fp64":
        tab_in["ln_kappa"] = tab["ln_kappa"].astype(np.float32)
        tab_in["ln_B"] = tab["ln_B"].astype(np.float32)
    rchi, rS = oracle_front_end(T_in, r_in, tab_in, shift)
    lnT, lnR = trilinear_log(T_in, shift), trilinear_log(r_in, shift)
    for got, ref in ((chi, rchi), (S, rS)):
        g = got.double().cpu().numpy()
        assert (_rel(g, ref) <= tol) if tol else _fp32_ok(g, ref, lnT, lnR), _rel(g, ref)


@pytest.mark.parametrize("shape,shift", [((100, 9, 1), (-0.5, -0.5, -0.5)), ((1, 1, 2), (3.5, -7.25, 1.5)),
                                         ((97, 17, 4), (-200.5, 33.75, 2.0))])
def test_front_end_fp32_edges(rts, shape, shift):
    import torch

    nx, ny, nz = shape
    rng = np.random.default_rng(nx + ny)
    T = (0.5 + rng.random((nz, ny, nx))).astype(np.float32)
    rho = np.exp(rng.normal(size=(nz, ny, nx))).astype(np.float32)
    tab = synthetic_table(nb=2, nT=40, nR=30, lnR_range=(-4.0, 2.0))
    tab32 = dict(tab, ln_kappa=tab["ln_kappa"].astype(np.float32), ln_B=tab["ln_B"].astype(np.float32))
    chi, S = rts.front_end(torch.tensor(T, device="cuda"), torch.tensor(rho, device="cuda"), tab, precision="fp32",
                           shift=shift)
    rchi, rS = oracle_front_end(T, rho, tab32, shift)
    lnT, lnR = trilinear_log(T, shift), trilinear_log(rho, shift)
    for got, ref in ((chi, rchi), (S, rS)):
        g = got.double().cpu().numpy()
        assert _fp32_ok(g, ref, lnT, lnR), _rel(g, ref)


def test_front_end_288x4(rts):
    import torch

    T, rho = mhd_fields(288, 288, 288, 0)
    tab = synthetic_table(nb=4)
    chi, S = rts.front_end(torch.tensor(T, dtype=torch.float32, device="cuda"),
                           torch.tensor(rho, dtype=torch.float32, device="cuda"), tab, precision="fp32")
    T32, r32 = T.astype(np.float32), rho.astype(np.float32)
    rchi, rS = oracle_front_end(T32, r32, dict(tab, ln_kappa=tab["ln_kappa"].astype(np.float32),
                                               ln_B=tab["ln_B"].astype(np.float32)))
    lnT, lnR = trilinear_log(T32, (-0.5, -0.5, -0.5)), trilinear_log(r32, (-0.5, -0.5, -0.5))
    for got, ref in ((chi, rchi), (S, rS)):
        g = got.double().cpu().numpy()
        assert _fp32_ok(g, ref, lnT, lnR), _rel(g, ref)
