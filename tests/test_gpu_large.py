"""The large anisotropic configuration: 512 x 512 x 256, 16 bands
(chi x 10^(4b/15), S = T^4 / 16), FP32 sweep with compensated accumulation.

The full 16-band oracle solve takes too long for a test, so the forward
solve is checked on sampled outputs the oracle computes one direction at a
time (I_top of chosen bands and upward rays, including periodic x- and
y-dominant ones), and the adjoint on the full grid with one band (bar 1e-4
of max|oracle| per gradient)."""
import numpy as np
import pytest

import oracle
from tests.gpu_common import norm_err
from workloads import stratified_atmosphere
from workloads.atmosphere import _bands

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

NX, NY, NZ, B = 512, 512, 256, 16


@pytest.fixture(scope="module")
def rts():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2107_08145_b300 as m

    m.load(build_if_missing=False)
    return m


@pytest.fixture(scope="module")
def atmosphere():
    T, _, chi = stratified_atmosphere(NX, NY, NZ, 0)
    cs, ss = _bands("sixteen", B)
    return T ** 4, chi, cs, ss


def test_large_forward_sampled_itop(rts, atmosphere):
    import torch

    S4, chi, cs, ss = atmosphere
    s = rts.Solver(NX, NY, NZ, B, precision="fp32_compensated")
    c = torch.empty((B, NZ, NY, NX), dtype=torch.float32, device="cuda")
    Sd = torch.empty_like(c)
    for b in range(B):
        c[b] = torch.as_tensor(chi * cs[b], dtype=torch.float32)
        Sd[b] = torch.as_tensor(S4 * ss[b], dtype=torch.float32)
    out = s.solve(c, Sd)
    itop = out["I_top"].cpu().numpy()
    del out, c, Sd
    P = oracle.Problem(NX, NY, NZ, B, max_wrap_iters=100000)
    n, _ = oracle.a4_quadrature()
    ups = [d for d in range(24) if n[d][2] > 0]
    # a z-dominant, an x-dominant and a y-dominant upward ray, thin to thick bands
    for b, d in ((0, ups[0]), (15, ups[5]), (7, ups[9])):
        I, _ = P.sweep(b, d, chi * cs[b], S4 * ss[b])
        err = norm_err(itop[b, ups.index(d)], I[NZ - 1])
        assert err <= 1e-5, (b, d, err)


def test_large_adjoint_one_band(rts, atmosphere):
    import torch

    S4, chi, cs, ss = atmosphere
    b = 7
    chi1 = (chi * cs[b])[None]
    S1 = (S4 * ss[b])[None]
    s = rts.Solver(NX, NY, NZ, 1, precision="fp32_compensated", adjoint=True)
    rng = np.random.default_rng(5)
    gI = rng.standard_normal((1, s.n_up, NY, NX))
    gQ = 1e-3 * rng.standard_normal((NZ, NY, NX))
    gl, gs = s.adjoint(torch.as_tensor(chi1, dtype=torch.float32, device="cuda"),
                       torch.as_tensor(S1, dtype=torch.float32, device="cuda"),
                       gI_top=torch.as_tensor(gI, dtype=torch.float32, device="cuda"),
                       gQ=torch.as_tensor(gQ, device="cuda"))
    P = oracle.Problem(NX, NY, NZ, 1, max_wrap_iters=100000)
    rl, rs = P.adjoint(chi1, S1, gI_top=gI, gQ=gQ, nthreads=oracle.default_threads())
    e = (norm_err(gl.double().cpu().numpy(), rl), norm_err(gs.double().cpu().numpy(), rs))
    assert e[0] <= 1e-4 and e[1] <= 1e-4, e
