"""GPU parity of the register-resident FP32 sweep (sweep_reg_kernel) against
the FP64 oracle, on grids chosen to reach every path of that kernel: tile
heights 2, 4 and 8; x/y-group tiles whose last tile is short (padding rows);
plane extents narrower than the CTA (idle warps) and a single column pair;
explicit boundary intensities; a very transparent top (long periodic
warm-up); both FP32 modes. Bar: 1e-5 max|oracle| per output, as for every
FP32 path."""
import numpy as np
import pytest

from tests.gpu_common import OUTPUTS, gpu_solve, norm_err, oracle_solve, random_case

pytestmark = pytest.mark.gpu

FP32_TOL = 1e-5


@pytest.fixture(scope="module")
def rts():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2107_08145_b300 as m

    m.load(build_if_missing=False)
    return m


def _solver(rts, nx, ny, nz, B, **kw):
    s = rts.Solver(nx, ny, nz, B, sweep_kernel="register", **kw)
    return s


def _check(rts, s, chi, S, ref, what, **solve_kw):
    got = gpu_solve(s, chi, S, **solve_kw)
    st = s.stats()
    assert st["sweep_kernel"] == rts.SWEEP_REGISTER, st
    errs = {k: norm_err(got[k], ref[k]) for k in OUTPUTS}
    assert all(e <= FP32_TOL for e in errs.values()), (what, st["tile_rows"], errs)
    return got


@pytest.mark.parametrize("tile_rows", [4, 8])
def test_tile_heights(rts, tile_rows):
    """z groups 16 rows (every tile height divides), x/y groups 13 rows: the
    last x/y tile is short for heights 4 and 8."""
    nx, ny, nz, B = 24, 16, 13, 2
    chi, S = random_case(nx, ny, nz, B, seed=5)
    ref = oracle_solve(chi, S)
    s = _solver(rts, nx, ny, nz, B, precision="fp32", tile_rows=tile_rows)
    assert s.stats()["tile_rows"] == tile_rows
    _check(rts, s, chi, S, ref, ("tile", tile_rows))


@pytest.mark.parametrize("shape", [(64, 200, 9), (2, 8, 7), (96, 36, 20), (290, 8, 5)])
def test_plane_widths(rts, shape):
    """Units narrower than the CTA (idle warps), one column pair, a partial
    last warp, and a plane of 145 column pairs (5 warps)."""
    nx, ny, nz = shape
    B = 2
    chi, S = random_case(nx, ny, nz, B, seed=nx + 3 * ny)
    ref = oracle_solve(chi, S)
    s = _solver(rts, nx, ny, nz, B, precision="fp32")
    _check(rts, s, chi, S, ref, shape)


@pytest.mark.parametrize("prec", ["fp32", "fp32_compensated"])
def test_thin_top_and_spacing(rts, prec):
    """A very transparent top (the periodic wrap warms up for several
    periods) on an anisotropic grid."""
    nx, ny, nz, B = 32, 24, 30, 3
    spacing = (1.0, 1.3, 0.8)
    chi, S = random_case(nx, ny, nz, B, seed=17, thin=True)
    ref = oracle_solve(chi, S, *spacing)
    s = _solver(rts, nx, ny, nz, B, dx=spacing[0], dy=spacing[1], dz=spacing[2], precision=prec)
    _check(rts, s, chi, S, ref, prec)
    assert s.stats()["max_warmup_steps"] > 0


def test_two_row_tiles(rts):
    """ny even but not a multiple of 4: the register sweep runs with 2-row
    tiles (the periodic z-group rows must be a multiple of the tile height);
    x/y groups of 13 rows end with a short tile."""
    nx, ny, nz, B = 28, 18, 13, 2
    chi, S = random_case(nx, ny, nz, B, seed=29)
    ref = oracle_solve(chi, S)
    s = _solver(rts, nx, ny, nz, B, precision="fp32")
    assert s.stats()["tile_rows"] == 2
    _check(rts, s, chi, S, ref, "two-row tiles")


def test_explicit_boundaries(rts):
    nx, ny, nz, B = 12, 12, 14, 2
    chi, S = random_case(nx, ny, nz, B, seed=3)
    rng = np.random.default_rng(1)
    bot = (1 + rng.random((B, 12, ny, nx))).astype(np.float32)
    top = (0.1 * rng.random((B, 12, ny, nx))).astype(np.float32)
    ref = oracle_solve(chi, S, bottom=bot, top=top)
    s = _solver(rts, nx, ny, nz, B, precision="fp32")
    _check(rts, s, chi, S, ref, "explicit", bottom=bot, top=top)


def test_zero_bottom_and_gray32(rts):
    from tests.gpu_common import workload_inputs

    chi, S = workload_inputs("gray32")
    ref = oracle_solve(chi, S, bottom="zero")
    s = _solver(rts, 32, 32, 32, 1, precision="fp32")
    _check(rts, s, chi, S, ref, "gray32 zero bottom", bottom="zero")


def test_register_matches_shared_sweep(rts):
    """Both FP32 sweeps solve the same discrete problem and the register sweep
    runs by default where it applies; against the oracle its error is of the
    same FP32-rounding size as the shared sweep's."""
    nx, ny, nz, B = 40, 36, 24, 3
    chi, S = random_case(nx, ny, nz, B, seed=23)
    ref = oracle_solve(chi, S)
    a = rts.Solver(nx, ny, nz, B, precision="fp32")
    assert a.stats()["sweep_kernel"] == rts.SWEEP_REGISTER
    b = rts.Solver(nx, ny, nz, B, precision="fp32", sweep_kernel="shared")
    assert b.stats()["sweep_kernel"] == rts.SWEEP_SHARED
    ga, gb = gpu_solve(a, chi, S), gpu_solve(b, chi, S)
    for k in OUTPUTS:
        ea, eb = norm_err(ga[k], ref[k]), norm_err(gb[k], ref[k])
        assert ea <= FP32_TOL and eb <= FP32_TOL, (k, ea, eb)
        assert ea <= 3 * eb + 1e-6, (k, ea, eb)


def test_register_sweep_refuses_what_it_cannot_run(rts):
    """Odd plane extents, an odd ny (no register tile height, 2 or 4 rows,
    divides the z groups' periodic rows) and FP64 have no register sweep:
    asking for it fails at create time with RTS_EINVAL; 'auto' falls back to
    the shared sweep. An even ny that is not a multiple of 4 takes 2-row
    tiles."""
    with pytest.raises(rts.RTSError) as e:
        rts.Solver(13, 10, 8, 1, precision="fp32", sweep_kernel="register")
    assert e.value.code == rts.RTS_EINVAL
    s = rts.Solver(13, 10, 8, 1, precision="fp32")
    assert s.stats()["sweep_kernel"] == rts.SWEEP_SHARED
    with pytest.raises(rts.RTSError):
        rts.Solver(12, 10, 8, 1, precision="fp64", sweep_kernel="register")
    with pytest.raises(rts.RTSError) as e:
        rts.Solver(12, 9, 8, 1, precision="fp32", sweep_kernel="register")
    assert e.value.code == rts.RTS_EINVAL
    assert rts.Solver(12, 9, 8, 1, precision="fp32").stats()["sweep_kernel"] == rts.SWEEP_SHARED
    st = rts.Solver(12, 10, 8, 1, precision="fp32").stats()
    assert st["sweep_kernel"] == rts.SWEEP_REGISTER and st["tile_rows"] == 2
