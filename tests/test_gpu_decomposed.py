"""Spatial decomposition (rts_create_decomposed / rts_solve_decomposed): the
grid cut into slabs of levels, each slab solved from the previous
iteration's boundary intensities of its neighbours, iterated until the
largest change of J is below tol times max J (the paper's decomposition and
its global J criterion). The converged result must be the undecomposed
solution: checked against the FP64 oracle (FP32 bar, 1e-5 of max) and
against the undecomposed GPU solve."""
import numpy as np
import pytest

from tests.gpu_common import OUTPUTS, norm_err, oracle_solve, random_case
from workloads import band_stack, stratified_atmosphere

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rts():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2107_08145_b300 as m

    m.load(build_if_missing=False)
    return m


def _t(a):
    import torch

    return torch.tensor(a, dtype=torch.float32, device="cuda")


def _np(out):
    return {k: v.double().cpu().numpy() for k, v in out.items()}


@pytest.mark.parametrize("nblocks", [2, 3, 5])
@pytest.mark.parametrize("prec", ["fp32", "fp32_compensated"])
def test_decomposed_matches_oracle_and_whole_solve(rts, nblocks, prec):
    nx, ny, nz, B = 24, 20, 30, 2
    chi, S = random_case(nx, ny, nz, B, seed=11)
    chi32, S32 = chi.astype(np.float32), S.astype(np.float32)
    ref = oracle_solve(chi32, S32)
    d = rts.DecomposedSolver(nx, ny, nz, B, nblocks=nblocks, precision=prec)
    out, iters = d.solve(_t(chi32), _t(S32), tol=1e-7, max_iter=4 * nblocks)
    got = _np(out)
    whole = _np(rts.Solver(nx, ny, nz, B, precision=prec, sweep_kernel="register").solve(_t(chi32), _t(S32)))
    for k in OUTPUTS:
        assert norm_err(got[k], ref[k]) <= 1e-5, (k, norm_err(got[k], ref[k]))
        assert norm_err(got[k], whole[k]) <= 2e-6, (k, norm_err(got[k], whole[k]))
    # boundary values cross one slab per iteration; one more shows no change
    assert 2 <= iters <= nblocks + 1, iters


def test_decomposed_stratified_atmosphere(rts):
    """A solar-like stratification (optically thick below, thin above) cut
    into 4 slabs of uneven optical depth."""
    nx, ny, nz, B = 32, 32, 40, 2
    T, _, chi = stratified_atmosphere(nx, ny, nz, 3)
    chib, Sb = band_stack(T, chi, [1.0, 30.0], [0.5, 0.2])
    chi32, S32 = chib.astype(np.float32), Sb.astype(np.float32)
    ref = oracle_solve(chi32, S32)
    d = rts.DecomposedSolver(nx, ny, nz, B, nblocks=4)
    out, iters = d.solve(_t(chi32), _t(S32), tol=1e-6, max_iter=16)
    got = _np(out)
    for k in OUTPUTS:
        assert norm_err(got[k], ref[k]) <= 1e-5, (k, norm_err(got[k], ref[k]))
    assert iters <= 5


def test_decomposed_reports_no_convergence(rts):
    nx, ny, nz, B = 16, 16, 12, 1
    chi, S = random_case(nx, ny, nz, B, seed=3, thin=True)
    d = rts.DecomposedSolver(nx, ny, nz, B, nblocks=3)
    with pytest.raises(rts.RTSError) as ei:
        d.solve(_t(chi), _t(S), tol=1e-7, max_iter=1)
    assert ei.value.code == rts.RTS_ENOCONV
    out, iters = d.solve(_t(chi), _t(S), tol=1e-7, max_iter=8)  # usable afterwards
    assert iters <= 4


def test_decomposed_rejects(rts):
    with pytest.raises(rts.RTSError) as ei:
        rts.DecomposedSolver(16, 16, 12, 1, nblocks=2, precision="fp64")
    assert ei.value.code == rts.RTS_EINVAL
    with pytest.raises(rts.RTSError) as ei:
        rts.DecomposedSolver(16, 16, 7, 1, nblocks=4)
    assert ei.value.code == rts.RTS_EINVAL
