"""Measured error of every GPU precision mode against the FP64 oracle on the
full workloads, element-wise where the FP64 path is concerned.

Bars (the FP64 path is the plain solve, the FP32 paths carry FP32 intensities):
  FP64:  |gpu - oracle| <= 1e-12 (|oracle| + floor) at every point and
         output, the floor being the size of the terms that output is formed
         from (tests.gpu_common.elementwise_floors): 0 for I_top and J,
         4 pi J for F, 4 pi sum_b (chi_b S_b + J_b / h) for Q_rad;
  FP32 (sweep in FP32, FP64 or double-float accumulation and Q step):
         max |gpu - oracle| <= 1e-5 max |oracle| per output.
Each test prints its per-output table (pytest -s).

Configurations: the 288^3 x 4-band workload (FP64 and both FP32 modes,
one oracle solve), one full band of the 512 x 512 x 256 x 16-band workload in
the compensated mode (the thinnest band: the longest periodic warm-up), and
one 128 x 128 x 192 subdomain of the batched workload with its 12 bands."""
import json

import numpy as np
import pytest

from tests.gpu_common import OUTPUTS, error_report, gpu_solve, oracle_solve, workload_inputs
from workloads import band_stack, stratified_atmosphere
from workloads.atmosphere import _bands

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

FP64_REL = 1e-12
FP32_TOL = 1e-5


@pytest.fixture(scope="module")
def rts():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2107_08145_b300 as m

    m.load(build_if_missing=False)
    return m


def _table(name, reps):
    print(f"\n== {name}")
    print(json.dumps(reps, indent=1, sort_keys=True))


def test_rts288x4_all_precisions(rts):
    chi, S = workload_inputs("rts288x4")
    chi32, S32 = chi.astype(np.float32), S.astype(np.float32)
    ref = oracle_solve(chi, S)
    reps = {}
    s = rts.Solver(288, 288, 288, 4, precision="fp64")
    got = gpu_solve(s, chi, S)
    del s
    reps["fp64"] = error_report(got, ref, chi, S)
    for k in OUTPUTS:
        assert reps["fp64"][k]["elementwise"] <= FP64_REL, (k, reps["fp64"][k])
    # the FP32 modes see the inputs rounded to FP32: compare with the oracle on those
    ref32 = oracle_solve(chi32, S32)
    for prec in ("fp32", "fp32_compensated"):
        s = rts.Solver(288, 288, 288, 4, precision=prec)
        got = gpu_solve(s, chi32, S32)
        del s
        reps[prec] = error_report(got, ref32, chi32, S32)
        for k in OUTPUTS:
            assert reps[prec][k]["normwise"] <= FP32_TOL, (prec, k, reps[prec][k])
    _table("rts288x4", reps)


def test_large512_thinnest_band_compensated(rts):
    """Band 0 of the 512 x 512 x 256 x 16 workload (chi x 1, S = T^4/16) as a
    one-band solve: J, F, Q_rad and I_top on the full grid."""
    nx, ny, nz = 512, 512, 256
    T, _, chi = stratified_atmosphere(nx, ny, nz, 0)
    cs, ss = _bands("sixteen", 16)
    chib, Sb = band_stack(T, chi, cs[:1], ss[:1])
    chi32, S32 = chib.astype(np.float32), Sb.astype(np.float32)
    ref = oracle_solve(chi32, S32)
    s = rts.Solver(nx, ny, nz, 1, precision="fp32_compensated")
    got = gpu_solve(s, chi32, S32)
    rep = error_report(got, ref, chi32, S32)
    for k in OUTPUTS:
        assert rep[k]["normwise"] <= FP32_TOL, (k, rep[k])
    _table("large512 band 0, fp32_compensated", rep)


def test_batched_size_subdomain_12_bands(rts):
    """A 128 x 128 x 192 subdomain with the batched workload's 12 bands
    (chi x 10^(3b/11), S x (12-b)/78), FP32 sweep with the FP64 Q step,
    directly against the oracle."""
    nx, ny, nz = 128, 128, 192
    T, _, chi = stratified_atmosphere(nx, ny, nz, 7)
    cs, ss = _bands("twelve", 12)
    chib, Sb = band_stack(T, chi, cs, ss)
    chi32, S32 = chib.astype(np.float32), Sb.astype(np.float32)
    ref = oracle_solve(chi32, S32)
    s = rts.Solver(nx, ny, nz, 12, precision="fp32")
    got = gpu_solve(s, chi32, S32)
    rep = error_report(got, ref, chi32, S32)
    for k in OUTPUTS:
        assert rep[k]["normwise"] <= FP32_TOL, (k, rep[k])
    _table("128x128x192 x 12 bands, fp32", rep)
