"""Batched solves (rts_create_batched / rts_solve_batched): many grids of
uneven size x bands in one persistent launch, its CUDA graph, and the tile
autotuner. On the shared-memory tile sweep (FP64, and FP32 batches with an
odd plane width) a batched solve must give exactly (bit for bit) what
rts_solve gives on each grid alone; FP32 batches of even widths run the
register sweep in one launch and must match the register-sweep single solves
to the rounding of the band reduction and the FP32 oracle bar; the FP64 path
must match the oracle element-wise."""
import numpy as np
import pytest

from tests.gpu_common import elementwise_err, elementwise_floors, OUTPUTS, norm_err, oracle_solve, random_case
from workloads import batched_bands, batched_subdomain_shapes, band_stack, stratified_atmosphere

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rts():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2107_08145_b300 as m

    m.load(build_if_missing=False)
    return m


def _inputs(shapes, B, seed0=0):
    chis, Ss = [], []
    for i, (nx, ny, nz) in enumerate(shapes):
        c, s = random_case(nx, ny, nz, B, seed=seed0 + i)
        chis.append(c)
        Ss.append(s)
    return chis, Ss


def _batched(rts, shapes, B, chis, Ss, precision, **kw):
    import torch

    bs = rts.BatchedSolver(shapes, B, precision=precision, **kw)
    dt = bs.dtype
    chi = bs.pack([torch.as_tensor(c, dtype=dt, device="cuda") for c in chis])
    S = bs.pack([torch.as_tensor(s, dtype=dt, device="cuda") for s in Ss])
    out = bs.solve(chi, S)
    return bs, chi, S, out


def _singles(rts, shapes, B, chis, Ss, precision, tile_rows=0, sweep_kernel="shared"):
    """rts_solve on each grid with the sweep the batched handle runs."""
    import torch

    res = []
    for (nx, ny, nz), c, s in zip(shapes, chis, Ss):
        so = rts.Solver(nx, ny, nz, B, precision=precision, tile_rows=tile_rows, sweep_kernel=sweep_kernel)
        o = so.solve(torch.as_tensor(c, dtype=so.dtype, device="cuda"), torch.as_tensor(s, dtype=so.dtype, device="cuda"))
        res.append({k: v.cpu().numpy() for k, v in o.items()})
    return res


SHAPES = [(12, 10, 9), (16, 16, 12), (9, 13, 8), (20, 8, 10), (33, 17, 6)]


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp32_compensated"])
def test_batched_equals_single_solves(rts, precision):
    B = 3
    chis, Ss = _inputs(SHAPES, B)
    bs, _, _, out = _batched(rts, SHAPES, B, chis, Ss, precision)
    assert bs.stats()["sweep_kernel"] == rts.SWEEP_SHARED  # odd plane widths: the shared-memory sweep
    got = bs.unpack(out)
    ref = _singles(rts, SHAPES, B, chis, Ss, precision)
    for i, (g, r) in enumerate(zip(got, ref)):
        for k in OUTPUTS:
            assert np.array_equal(g[k].cpu().numpy(), r[k]), (precision, i, k)


def test_batched_fp64_vs_oracle(rts):
    B = 2
    shapes = SHAPES[:3]
    chis, Ss = _inputs(shapes, B, seed0=10)
    bs, _, _, out = _batched(rts, shapes, B, chis, Ss, "fp64")
    for g, c, s in zip(bs.unpack(out), chis, Ss):
        ref = oracle_solve(c, s)
        fl = elementwise_floors(ref, c, s)
        for k in OUTPUTS:
            assert elementwise_err(g[k].cpu().numpy(), ref[k], fl[k]) <= 1e-12, k


@pytest.mark.parametrize("tile_rows", [1, 2, 3, 4, 8, 12, 16])
def test_batched_tile_rows_do_not_change_results(rts, tile_rows):
    B = 2
    chis, Ss = _inputs(SHAPES, B, seed0=20)
    bs, _, _, out = _batched(rts, SHAPES, B, chis, Ss, "fp32", tile_rows=tile_rows)
    ref = _singles(rts, SHAPES, B, chis, Ss, "fp32", tile_rows=4)
    for g, r in zip(bs.unpack(out), ref):
        for k in OUTPUTS:
            assert np.array_equal(g[k].cpu().numpy(), r[k]), (tile_rows, k)


def test_batched_graph_replay(rts):
    """A captured batched solve replays to the same results, twice."""
    import torch

    B = 2
    chis, Ss = _inputs(SHAPES, B, seed0=30)
    stream = torch.cuda.Stream()
    bs, chi, S, out = _batched(rts, SHAPES, B, chis, Ss, "fp32", stream=stream)
    ref = {k: v.clone() for k, v in out.items()}
    g, gout = bs.graph(chi, S)
    for _ in range(2):
        for v in gout.values():
            v.fill_(-1)
        g.launch()
        bs.check()
        for k in OUTPUTS:
            assert torch.equal(gout[k], ref[k]), k


def test_single_graph_replay(rts):
    import torch

    nx, ny, nz, B = 16, 14, 12, 2
    c, s = random_case(nx, ny, nz, B, seed=5)
    stream = torch.cuda.Stream()
    so = rts.Solver(nx, ny, nz, B, precision="fp64", stream=stream)
    chi = torch.as_tensor(c, device="cuda")
    S = torch.as_tensor(s, device="cuda")
    with torch.cuda.stream(stream):
        ref = so.solve(chi, S)
    g, gout = so.graph(chi, S)
    g.launch()
    so.check()
    for k in OUTPUTS:
        assert torch.equal(gout[k], ref[k]), k


def test_autotune(rts):
    import torch

    B = 2
    chis, Ss = _inputs(SHAPES, B, seed0=40)
    bs = rts.BatchedSolver(SHAPES, B, precision="fp32")
    chi = bs.pack([torch.as_tensor(x, dtype=torch.float32, device="cuda") for x in chis])
    S = bs.pack([torch.as_tensor(x, dtype=torch.float32, device="cuda") for x in Ss])
    best, ms = rts.autotune(SHAPES, B, chi, S, precision="fp32", repeats=2)
    assert best in (1, 2, 3, 4) and best in ms and all(v > 0 for v in ms.values()), (best, ms)


def test_batched_rejects_explicit_boundaries(rts):
    import torch

    B = 1
    chis, Ss = _inputs(SHAPES[:2], B)
    bs, chi, S, _ = _batched(rts, SHAPES[:2], B, chis, Ss, "fp32")
    with pytest.raises(rts.RTSError):
        bs.solve(chi, S, bottom=torch.zeros(10, device="cuda"))


def test_batched_uneven_subdomains_12_bands(rts):
    """Eight subdomains of the batched workload's size mix x 12 bands, FP32,
    on the register sweep in one launch: the same as solving each grid alone
    with the register sweep, to the rounding of the band reduction."""
    shapes = batched_subdomain_shapes(8, seed=0)
    cs, ss = batched_bands()
    chis, Ss = [], []
    for i, (nx, ny, nz) in enumerate(shapes):
        T, _, chi = stratified_atmosphere(nx, ny, nz, seed=i)
        c, s = band_stack(T, chi, cs, ss)
        chis.append(c)
        Ss.append(s)
    bs, _, _, out = _batched(rts, shapes, 12, chis, Ss, "fp32")
    assert bs.stats()["sweep_kernel"] == rts.SWEEP_REGISTER
    ref = _singles(rts, shapes, 12, chis, Ss, "fp32", sweep_kernel="register")
    for g, r in zip(bs.unpack(out), ref):
        assert np.array_equal(g["I_top"].cpu().numpy(), r["I_top"])  # the same sweep arithmetic per point
        for k in ("J", "F", "Q"):
            e = norm_err(g[k].cpu().numpy(), r[k])
            assert e <= 1e-6, (k, e)


EVEN = [(16, 16, 12), (24, 20, 10), (12, 28, 14), (20, 24, 8)]  # ny multiples of 4


@pytest.mark.parametrize("precision", ["fp32", "fp32_compensated"])
def test_batched_register_sweep_vs_oracle(rts, precision):
    """Even plane widths: one register-sweep launch for all subdomains,
    against the FP64 oracle (FP32 bar, 1e-5 of max)."""
    B = 3
    chis, Ss = _inputs(EVEN, B, seed0=40)
    bs, _, _, out = _batched(rts, EVEN, B, chis, Ss, precision)
    assert bs.stats()["sweep_kernel"] == rts.SWEEP_REGISTER
    for g, c, s in zip(bs.unpack(out), chis, Ss):
        ref = oracle_solve(c.astype(np.float32), s.astype(np.float32))
        for k in OUTPUTS:
            e = norm_err(g[k].double().cpu().numpy(), ref[k])
            assert e <= 1e-5, (precision, k, e)


def test_batched_register_sweep_graph_and_shared_option(rts):
    """The register-sweep batch replays in a CUDA graph; sweep_kernel='shared'
    keeps the per-width launches and agrees to the FP32 bar."""
    import torch

    B = 2
    chis, Ss = _inputs(EVEN, B, seed0=50)
    stream = torch.cuda.Stream()
    bs, chi, S, out = _batched(rts, EVEN, B, chis, Ss, "fp32", stream=stream)
    assert bs.stats()["sweep_kernel"] == rts.SWEEP_REGISTER
    ref = {k: v.clone() for k, v in out.items()}
    g, gout = bs.graph(chi, S)
    for _ in range(2):
        for v in gout.values():
            v.fill_(-1)
        g.launch()
        bs.check()
        for k in OUTPUTS:
            assert torch.equal(gout[k], ref[k]), k
    sh = rts.BatchedSolver(EVEN, B, precision="fp32", sweep_kernel="shared")
    assert sh.stats()["sweep_kernel"] == rts.SWEEP_SHARED
    o2 = sh.solve(chi, S)
    for k in OUTPUTS:
        e = norm_err(o2[k].double().cpu().numpy(), out[k].double().cpu().numpy())
        assert e <= 1e-5, (k, e)
