"""The Python binding refuses, before any library call, arrays that the
library would read or write out of bounds or on the wrong device: inputs of
the wrong shape, dtype or placement, caller-supplied outputs that are short,
strided or of the wrong dtype, explicit boundaries of the wrong ray count,
batched arrays of the wrong length (explicit boundaries on a batched handle
are refused by the library itself). Valid arrays are still accepted after
the refusals (the handle is unchanged by them)."""
import numpy as np
import pytest

from workloads.opacity import synthetic_table

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rts():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2107_08145_b300 as m

    m.load(build_if_missing=False)
    return m


def test_solve_arguments(rts):
    import torch

    nx, ny, nz, B = 8, 8, 8, 2
    s = rts.Solver(nx, ny, nz, B, precision="fp32")
    chi = torch.ones((B, nz, ny, nx), device="cuda")
    S = torch.ones_like(chi)
    for bad in (torch.ones((B, nz, ny, nx - 1), device="cuda"),
                torch.ones((B, nz, ny, nx), dtype=torch.float64, device="cuda"),
                torch.ones((B, nz, ny, nx))):  # host memory
        with pytest.raises(ValueError):
            s.solve(chi, bad)
    out = s.solve(chi, S)
    f64 = dict(dtype=torch.float64, device="cuda")
    for bad in (dict(out, J=torch.empty(nz * ny * nx - 1, **f64)),
                dict(out, F=torch.empty((3, nz, ny, 2 * nx), **f64)[..., ::2]),  # strided
                dict(out, Q=torch.empty((nz, ny, nx), device="cuda")),  # float32
                dict(out, I_top=torch.empty((B, s.n_up - 1, ny, nx), device="cuda")),
                dict(out, Jx=out["J"])):
        with pytest.raises(ValueError):
            s.solve(chi, S, out=bad)
    with pytest.raises(ValueError):
        s.solve(chi, S, bottom=torch.ones((B, s.n_up - 1, ny, nx), device="cuda"))
    assert s.solve(chi, S, out=out) is out
    top = torch.zeros((B, s.ndir - s.n_up, ny, nx), device="cuda")
    J = s.solve(chi, S, top=top)["J"]  # an explicit zero top is the zero kind
    assert torch.allclose(J, out["J"], rtol=1e-5, atol=0)


def test_adjoint_arguments(rts):
    import torch

    n = 8
    s = rts.Solver(n, n, n, 1, precision="fp64", adjoint=True)
    chi = torch.ones((1, n, n, n), dtype=torch.float64, device="cuda")
    S = torch.ones_like(chi)
    gQ = torch.ones((n, n, n), dtype=torch.float64, device="cuda")
    with pytest.raises(ValueError):
        s.adjoint(chi, S, gJ=torch.ones((n, n, n - 1), dtype=torch.float64, device="cuda"))
    with pytest.raises(ValueError):
        s.adjoint(chi, S, gQ=gQ.float())
    with pytest.raises(ValueError):
        s.adjoint(chi, S, gQ=gQ, out=(torch.empty_like(chi)[:, : n // 2], torch.empty_like(S)))
    g = s.adjoint(chi, S, gQ=gQ)
    assert g[0].shape == chi.shape and bool(torch.isfinite(g[0]).all())


def test_batched_arguments(rts):
    import torch

    bs = rts.BatchedSolver([(12, 10, 9), (16, 16, 12)], 1, precision="fp32")
    n = bs.totals[0]
    chi = torch.ones(n, device="cuda")
    S = torch.ones(n, device="cuda")
    with pytest.raises(ValueError):
        bs.solve(chi[:-1], S)
    with pytest.raises(rts.RTSError):  # the library refuses explicit boundaries on batched handles
        bs.solve(chi, S, bottom=torch.ones(10, device="cuda"))
    out = bs.solve(chi, S)
    with pytest.raises(ValueError):
        bs.solve(chi, S, out=dict(out, Q=out["Q"][:-1]))
    assert bs.solve(chi, S, out=out) is out
    with pytest.raises(ValueError):
        rts.autotune([(12, 10, 9), (16, 16, 12)], 1, chi[:-1], S, precision="fp32")


def test_host_arguments(rts):
    n = 8
    s = rts.Solver(n, n, n, 1, precision="fp64", host_io=True)
    chi = np.ones((1, n, n, n))
    S = np.ones_like(chi)
    with pytest.raises(ValueError):
        s.solve_host(chi, S[:, : n // 2])
    with pytest.raises(ValueError):
        s.solve_host(chi, S, out=dict(J=np.empty((n, n, n), np.float32)))
    with pytest.raises(ValueError):
        s.solve_host(chi, S, out=dict(F=np.empty((3, n, n, 2 * n))[..., ::2]))
    out = s.solve_host(chi, S)
    assert np.isfinite(out["Q"]).all()


def test_front_end_arguments(rts):
    import torch

    T = torch.ones((4, 6, 8), device="cuda")
    rho = torch.ones_like(T)
    tab = synthetic_table(nb=2, nT=8, nR=8)
    good = torch.empty((2, 4, 6, 8), device="cuda")
    with pytest.raises(ValueError):
        rts.front_end(T, rho, tab, out=(torch.empty((2, 4, 6, 7), device="cuda"), good))
    with pytest.raises(ValueError):
        rts.front_end(T, rho.cpu(), tab)
    chi, S = rts.front_end(T, rho, tab, out=(good, torch.empty_like(good)))
    assert chi is good and bool((S > 0).all())
