"""Warm start of the periodic wrap (rts_boundary.wrap_seed, register sweep):
a solve writes its converged wrap planes; a later solve started from them
(seed_in) iterates periods until the wrap plane changes by at most seed_tol
(the paper's test on boundary intensities). Checked against the FP64 oracle
(FP32 bar, 1e-5 of max): the same atmosphere again, and a sequence of
slowly changing atmospheres each started from the previous solution."""
import numpy as np
import pytest

from tests.gpu_common import OUTPUTS, gpu_solve, norm_err, oracle_solve, random_case
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


def _solve(s, chi, S, **kw):
    import torch

    out = s.solve(torch.tensor(chi, dtype=torch.float32, device="cuda"),
                  torch.tensor(S, dtype=torch.float32, device="cuda"), **kw)
    return {k: v.double().cpu().numpy() for k, v in out.items()}


def test_seed_written_and_reused(rts):
    import torch

    nx, ny, nz, B = 24, 20, 18, 2
    chi, S = random_case(nx, ny, nz, B, seed=4, thin=True)
    chi32, S32 = chi.astype(np.float32), S.astype(np.float32)
    ref = oracle_solve(chi32, S32)
    s = rts.Solver(nx, ny, nz, B, precision="fp32")
    seed = torch.zeros(s.wrap_seed_elems(), dtype=torch.float32, device="cuda")
    # per band two x-dominant groups (plane ny x nz) and two y-dominant (nx x nz), 4 slots each
    assert seed.numel() == B * 2 * 4 * nz * (nx + ny)
    cold = _solve(s, chi32, S32, wrap_seed=seed)
    st_cold = s.stats()
    assert torch.count_nonzero(seed) > 0
    warm = _solve(s, chi32, S32, wrap_seed=seed, seed_in=True)
    st_warm = s.stats()
    for got in (cold, warm):
        for k in OUTPUTS:
            assert norm_err(got[k], ref[k]) <= 1e-5, k
    # started from its own converged planes: one period and the decision lag
    assert st_warm["max_warmup_steps"] <= 8 < st_cold["max_warmup_steps"]


def test_sequence_of_changing_atmospheres(rts):
    import torch

    nx, ny, nz, B = 32, 32, 24, 2
    T, _, chi = stratified_atmosphere(nx, ny, nz, 1)
    s = rts.Solver(nx, ny, nz, B, precision="fp32")
    seed = torch.zeros(s.wrap_seed_elems(), dtype=torch.float32, device="cuda")
    for step in range(4):
        Ts = T * (1.0 + 2e-3 * step)
        chib, Sb = band_stack(Ts, chi * (1.0 - 1e-3 * step), [1.0, 30.0], [0.5, 0.2])
        c32, S32 = chib.astype(np.float32), Sb.astype(np.float32)
        got = _solve(s, c32, S32, wrap_seed=seed, seed_in=step > 0)
        ref = oracle_solve(c32, S32)
        for k in OUTPUTS:
            assert norm_err(got[k], ref[k]) <= 1e-5, (step, k)


def test_warm_start_needs_the_register_sweep(rts):
    import torch

    s = rts.Solver(12, 10, 8, 1, precision="fp64")
    assert s.wrap_seed_elems() == 0
    s2 = rts.Solver(13, 10, 8, 1, precision="fp32")  # odd nx: the shared sweep
    b, _ = s2._bc("equal_s", "zero")
    x = torch.ones((1, 8, 10, 13), dtype=torch.float32, device="cuda")
    b.wrap_seed = x.data_ptr()
    rc = s2._L.rts_solve(s2._h, x.data_ptr(), x.data_ptr(), b, None, None, None, None)
    assert rc == rts.RTS_EINVAL
