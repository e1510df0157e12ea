"""rts_solve_noalloc: the forward solve for callers that cannot allocate
device memory (code running inside someone else's CUDA graph capture, or an
application that gives the solver a fixed memory budget). Its scratch is one
fixed static device array, so this test checks that two calls in a row, with
different inputs, give what the regular rts_solve gives, and that a problem
too large for the array is refused with a clear message. It sits in its own
file so that it runs after every other test."""
import numpy as np
import pytest

from tests.gpu_common import OUTPUTS, norm_err, random_case

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 1e-5, "fp32_compensated": 1e-5}


@pytest.fixture(scope="module")
def rts():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2107_08145_b300 as m

    m.load(build_if_missing=False)
    return m


@pytest.mark.parametrize("prec", ["fp32", "fp64", "fp32_compensated"])
def test_noalloc_matches_regular_solve_twice(rts, prec):
    import torch

    nx, ny, nz, B = 24, 20, 18, 2
    dt = torch.float64 if prec == "fp64" else torch.float32
    solver = rts.Solver(nx, ny, nz, B, precision=prec)
    for seed in (1, 2):  # two calls in a row; the array keeps the first call's contents
        chi, S = random_case(nx, ny, nz, B, seed=seed)
        c = torch.as_tensor(chi, dtype=dt, device="cuda")
        s = torch.as_tensor(S, dtype=dt, device="cuda")
        ref = solver.solve(c, s)
        got = rts.solve_noalloc(c, s, precision=prec)
        for k in OUTPUTS:
            e = norm_err(got[k].double().cpu().numpy(), ref[k].double().cpu().numpy())
            assert e <= TOL[prec], (prec, seed, k, e)


def test_noalloc_rejects_too_large(rts):
    import torch

    c = torch.ones((4, 160, 160, 160), dtype=torch.float32, device="cuda")
    with pytest.raises(rts.RTSError) as ei:
        rts.solve_noalloc(c, c, precision="fp32")
    assert ei.value.code == rts.RTS_EINVAL
    assert "scratch" in str(ei.value)


def test_noalloc_smaller_grid_after_larger(rts):
    """The shared array keeps a larger earlier call's contents (partials,
    reductions, transposes at other offsets): a smaller, differently shaped
    call afterwards still matches rts_solve."""
    import torch

    for (nx, ny, nz, B) in ((40, 36, 30, 2), (18, 22, 11, 1), (26, 14, 17, 3)):
        chi, S = random_case(nx, ny, nz, B, seed=nx)
        c = torch.as_tensor(chi, dtype=torch.float32, device="cuda")
        s = torch.as_tensor(S, dtype=torch.float32, device="cuda")
        ref = rts.Solver(nx, ny, nz, B, precision="fp32").solve(c, s)
        got = rts.solve_noalloc(c, s, precision="fp32")
        for k in OUTPUTS:
            e = norm_err(got[k].double().cpu().numpy(), ref[k].double().cpu().numpy())
            assert e <= TOL["fp32"], ((nx, ny, nz, B), k, e)


def test_noalloc_refuses_stream_capture(rts):
    """The call waits for its stream, so inside a capture it must refuse
    (RTS_EINVAL) and leave the capture intact."""
    import torch

    nx, ny, nz, B = 16, 16, 8, 1
    chi, S = random_case(nx, ny, nz, B, seed=2)
    c = torch.as_tensor(chi, dtype=torch.float32, device="cuda")
    s = torch.as_tensor(S, dtype=torch.float32, device="cuda")
    out = rts.solve_noalloc(c, s, precision="fp32")  # outputs made outside the capture
    side = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    refused = None
    with torch.cuda.stream(side):
        with torch.cuda.graph(g, stream=side):
            try:
                rts.solve_noalloc(c, s, precision="fp32", out=out, stream=side)
            except rts.RTSError as e:
                refused = e
            c.add_(0.0)  # the capture is still usable
    assert refused is not None and refused.code == rts.RTS_EINVAL and "capture" in str(refused)
    g.replay()
    torch.cuda.synchronize()
