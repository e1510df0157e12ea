#!/usr/bin/env python3
"""Benchmark of the B300 RTS solve on the paper's 288^3 test size, 4 bands.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

A step is one forward solve (rts_solve: transpose, persistent sweep over all
bands and direction groups, per-band reduction, Q step) of the synthetic
288^3 x 4-band stratified atmosphere with the FP32 sweep and FP64 Q step,
inputs resident in HBM (764 MB of chi/S, larger than L2, so no flush is
needed between steps). The metric is point x direction x band updates per
second (Gupd/s = 288^3 * 24 * 4 / t). One JSON line is printed by rank 0.

Extra keys: roofline of the sweep kernel (timed live with CUDA events on its
own stream through the library's phase timer), the FP64 solve, the end-to-end
number through rts_solve_host (host buffers, copies inside the timed region),
the CPU oracle timed on this host, and SM clocks sampled during the timed
region. Under torchrun (N > 1) every rank solves its own replica (no data-path
collective); timing is the max over ranks.

--impl reference times the CPU oracle (the paper has no code to run) on a
bounded sample of the same workload and prints the same kind of line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Gupd/s (pts×dirs×bands) 288³×4 bands FP32 vs FP64, %HBM; adjoint/fwd ratio"
WORKLOAD = "rts288x4"
NX = NY = NZ = 288
NB = 4
NDIR = 24
TILE_ROWS = None


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


def _config(prec, ws=1, sweep_kernel=2):
    """The workload as the JSON line names it. sweep_kernel: 2 for the register
    sweep (both FP32 modes then reduce and form Q_rad in double-float), 1 for
    the shared sweep (FP32 mixed: FP64 for the cancelling parts)."""
    if prec == "fp64":
        q_step = "FP64"
    elif sweep_kernel == 2 or prec == "fp32_compensated":
        q_step = "double-float (2xFP32)"
    else:
        q_step = "FP64 for the cancelling parts"
    return {
        "grid": [NX, NY, NZ],
        "parallelism": ("single GPU" if ws == 1 else
                        f"band-sharded over {ws} GPUs: {NB} bands per GPU ({NB * ws}-band atmosphere), "
                        "one NCCL all-reduce of J, F, Q_rad (FP64) per solve inside the timed region"),
        "workload": f"rts288x4: {NX}x{NY}x{NZ} periodic grid, 4 opacity bands (chi x {{1,10,100,1000}}, "
                    "S = T^4 x {0.4,0.3,0.2,0.1}), 24 rays (S4 Carlson), bottom I=S, top I=0",
        "precision": prec,
        "sweep": "FP32 sweep" if prec != "fp64" else "FP64 sweep",
        "q_step": q_step,
        "l2": "inputs (764 MB chi+S FP32) larger than the 126 MB L2; no flush between steps",
        "step": "one rts_solve over all 4 bands and 24 rays",
        "tile_rows": TILE_ROWS,
    }


# ----------------------------------------------------------------------------
# SM clocks and throttle reasons during the timed region (NVML, read only)
# ----------------------------------------------------------------------------
class ClockSampler:
    """Samples SM clock and clock-event reasons while the timed region runs:
    NVML when its library loads, else `nvidia-smi -lms` (both read only)."""
    REASONS = {0x1: "gpu_idle", 0x2: "applications_clocks_setting", 0x4: "sw_power_cap",
               0x8: "hw_slowdown", 0x10: "sync_boost", 0x20: "sw_thermal_slowdown",
               0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown",
               0x100: "display_clock_setting"}

    def __init__(self, index):
        self.index = index
        self.samples = []
        self.reasons = 0
        self.max_mhz = None
        self._stop = threading.Event()
        self.mode = None
        self.err = None
        try:
            import pynvml

            pynvml.nvmlInit()
            self.nv = pynvml
            self.h = pynvml.nvmlDeviceGetHandleByIndex(index)
            self.max_mhz = pynvml.nvmlDeviceGetMaxClockInfo(self.h, pynvml.NVML_CLOCK_SM)
            self.mode = "nvml"
        except Exception as e:
            self.err = f"nvml: {e}"
            self.mode = "nvidia-smi"

    def _reason_bits(self):
        for name in ("nvmlDeviceGetCurrentClocksEventReasons", "nvmlDeviceGetCurrentClocksThrottleReasons"):
            f = getattr(self.nv, name, None)
            if f is not None:
                try:
                    return f(self.h)
                except Exception:
                    continue
        return 0

    def _run_nvml(self):
        while not self._stop.is_set():
            try:
                self.samples.append(self.nv.nvmlDeviceGetClockInfo(self.h, self.nv.NVML_CLOCK_SM))
                self.reasons |= self._reason_bits()
            except Exception as e:
                self.err = f"nvml sample: {e}"
            time.sleep(0.005)

    def __enter__(self):
        if self.mode == "nvml":
            self.t = threading.Thread(target=self._run_nvml, daemon=True)
            self.t.start()
        else:
            import subprocess

            q = ("clocks.sm,clocks.max.sm,clocks_event_reasons.active")
            try:
                self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + q,
                                              "--format=csv,noheader,nounits", "-lms", "20"],
                                             stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            except Exception as e:
                self.proc = None
                self.err = (self.err or "") + f"; nvidia-smi: {e}"
        return self

    def __exit__(self, *a):
        if self.mode == "nvml":
            self._stop.set()
            self.t.join()
        elif self.proc is not None:
            self.proc.terminate()
            out, _ = self.proc.communicate()
            for line in out.splitlines():
                f = [x.strip() for x in line.split(",")]
                try:
                    self.samples.append(float(f[0]))
                    self.max_mhz = float(f[1])
                    self.reasons |= int(f[2], 16)
                except Exception:
                    continue

    def summary(self):
        names = [n for b, n in self.REASONS.items() if self.reasons & b and n != "gpu_idle"]
        out = {"sm_mhz": statistics.median(self.samples) if self.samples else None, "sm_max_mhz": self.max_mhz,
               "reasons": names, "samples": len(self.samples), "source": self.mode}
        if not self.samples:  # why the clocks are missing (an NVML miss with nvidia-smi samples is no error)
            out["error"] = self.err
        return out


# ----------------------------------------------------------------------------
def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


SWEEP_PROFILES = {  # sweep kernel -> (committed DRAM summary, the source its counters were taken from)
    2: ("sweep_reg_rts288x4_dram.md", "sweep_reg.cuh"),
    1: ("sweep_rts288x4_dram.md", "sweep.cuh"),
}


def _traffic_from_profile(prec, grid, tile_rows, kernel):
    """DRAM bytes per sweep launch from the committed ncu summary of the
    sweep kernel that ran ("- key: value" lines), or None if that kernel's
    source changed since the counters were taken or the run is not the
    summary's workload (grid, precision, tile height)."""
    if kernel not in SWEEP_PROFILES:
        return None
    name, src_name = SWEEP_PROFILES[kernel]
    path = os.path.join(ROOT, "profiles", name)
    rec = {}
    try:
        for line in open(path):
            if line.startswith("- ") and ":" in line:
                k, v = line[2:].split(":", 1)
                rec[k.strip()] = v.strip()
    except OSError:
        return None
    src = os.path.join(ROOT, "paper_2107_08145_b300", "csrc", src_name)
    digest = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    if rec.get("sweep_source_sha256_16") != digest or rec.get("precision") != prec:
        return None
    if rec.get("grid") != "x".join(str(v) for v in grid) or rec.get("tile_rows") != str(tile_rows):
        return None
    try:
        return int(rec["dram_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


def _solve_bytes(prec, ms_step, sweep_traffic):
    """Bytes of one whole FP32 solve of the bench workload (register path):
    the compulsory floor (chi, S read once, J, F, Q written once: 72 B per
    point at 4 bands), the streaming model of the method (744 B per point at
    4 bands: each of the 6 groups streams every band's chi and S, its J/F
    partials leave and return once, and the Q step reads chi, S and writes
    J, F, Q), the
    algorithmic bytes of the four kernels as built (x transpose, sweep,
    reduction, Q step), and the DRAM bytes ncu measured for the sweep, the
    reduction and the Q step (profiles/sweep_reg_rts288x4_dram.md, only while
    their sources are unchanged) plus the transpose's algorithmic bytes."""
    if prec == "fp64":
        return None
    n = NX * NY * NZ
    alg = {"transpose": 4 * NB * n * 4,             # chi, S read and written once
           "sweep": sweep_algorithmic_bytes(prec),
           "reduction": NB * (NDIR // 4) * n * 16 + NB * 4 * n * 8,  # raw slots in, double-float J_b, F_b out
           "q_step": NB * 4 * n * 8 + 2 * NB * n * 4 + 5 * n * 8}    # J_b, F_b and chi, S in; J, F, Q out
    out = {"floor_bytes": (8 * NB + 40) * n, "streaming_model_bytes": (6 * 8 * NB + 6 * 2 * 40 + 8 * NB + 40) * n,
           "algorithmic_bytes": sum(alg.values()), "algorithmic_by_kernel": alg}
    rec = {}
    try:
        for line in open(os.path.join(ROOT, "profiles", "sweep_reg_rts288x4_dram.md")):
            if line.startswith("- ") and ":" in line:
                k, v = line[2:].split(":", 1)
                rec[k.strip()] = v.strip()
    except OSError:
        rec = {}
    q = os.path.join(ROOT, "paper_2107_08145_b300", "csrc", "qfused.cuh")
    if sweep_traffic and rec.get("qfused_source_sha256_16") == hashlib.sha256(open(q, "rb").read()).hexdigest()[:16]:
        try:
            dram = sweep_traffic + int(rec["qf_reduce_dram_bytes"]) + int(rec["qstep_df2_dram_bytes"]) + alg["transpose"]
            out["dram_bytes"] = dram
            out["dram_gbs"] = round(dram / (ms_step * 1e-3) / 1e9, 1)
        except (KeyError, ValueError):
            pass
    return out


FP64_PEAK_GFLOPS = 1250.0  # nominal B300 FP64 rate; no measured FP64 peak is on record


def _performed_updates(st, nx, ny, nz, nb):
    """Ray-point updates the sweep executed: every unit's planes, the x/y
    groups' warm-up planes included (mean over units from the stats), 4 rays
    per unit (24-ray set: 2 z, 2 y, 2 x groups per band)."""
    warm = st.get("mean_warmup_steps", 0.0)
    z = 2 * nz * nx * ny
    xy = 2 * (nx + warm) * ny * nz + 2 * (ny + warm) * nx * nz
    return 4 * nb * (z + xy)


def _fp64_roofline(st):
    """The FP64 sweep against the FP64 rate: FP64 flops executed per launch
    (the per-update count of profiles/sweep_fp64_ops.md, measured by ncu on a
    smaller grid, times the updates this launch performed) over its time.
    None when that record is missing or the sweep source changed since."""
    path = os.path.join(ROOT, "profiles", "sweep_fp64_ops.md")
    rec = {}
    try:
        for line in open(path):
            if line.startswith("- ") and ":" in line:
                k, v = line[2:].split(":", 1)
                rec[k.strip()] = v.strip()
    except OSError:
        return None
    src = os.path.join(ROOT, "paper_2107_08145_b300", "csrc", "sweep.cuh")
    digest = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    if rec.get("sweep_source_sha256_16") != digest:
        return None
    try:
        per_upd = float(rec["fp64_flops_per_update"])
    except (KeyError, ValueError):
        return None
    flops = per_upd * _performed_updates(st, NX, NY, NZ, NB)
    ach = flops / (st["ms_sweep"] * 1e-3) / 1e9
    return {"kernel": "sweep_kernel<double> (FP64 persistent tile-DAG sweep)", "bound": "fp64",
            "achieved": round(ach, 2), "peak": FP64_PEAK_GFLOPS, "unit": "GFLOP/s",
            "frac": round(ach / FP64_PEAK_GFLOPS, 4), "peak_source": "nominal (1.25 TFLOP/s FP64), not measured",
            "fp64_flops_per_update": per_upd, "tile_rows": st["tile_rows"]}


def sweep_algorithmic_bytes(prec, nb=NB, ndir=NDIR):
    """Per launch: every sweep unit (band x group of 4 rays) reads its band's
    chi and S once and writes 4 values per point once (its raw slot
    intensities, or its partial sums J, Fx, Fy, Fz); plus the upward
    intensities at the top."""
    es = 8 if prec == "fp64" else 4
    n = NX * NY * NZ
    units = nb * (ndir // 4)
    return units * n * (2 * es + 4 * es) + nb * (ndir // 2) * NX * NY * es


def _adjoint_timing(rts, torch, workload, name, grid, prec, stream, steps, chunk=0):
    """Mean ms of rts_solve and of rts_adjoint (loss on I_top and Q_rad;
    `chunk` bands per checkpoint, 0 = the library's automatic choice) on one
    workload, CUDA events on the solver's stream."""
    import numpy as np

    nx, ny, nz = grid
    chi64, S64 = workload(name, nx=nx, ny=ny, nz=nz)
    nb = chi64.shape[0]
    s = rts.Solver(nx, ny, nz, nb, precision=prec, stream=stream, adjoint=True, adjoint_chunk_bands=chunk)
    dev = torch.device("cuda", torch.cuda.current_device())
    chi = torch.as_tensor(chi64, dtype=s.dtype, device=dev)
    S = torch.as_tensor(S64, dtype=s.dtype, device=dev)
    out = s.solve(chi, S)
    rng = np.random.default_rng(0)
    gI = torch.as_tensor(rng.standard_normal(tuple(out["I_top"].shape)), dtype=s.dtype, device=dev)
    gQ = 2e-3 * out["Q"]
    grads = s.adjoint(chi, S, gI_top=gI, gQ=gQ)

    def timed(fn):
        for _ in range(2):
            fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(steps):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / steps

    fwd = timed(lambda: s.solve(chi, S, out=out, check=False))
    bwd = timed(lambda: s.adjoint(chi, S, gI_top=gI, gQ=gQ, out=grads, check=False))
    s.check()
    chunk = s.stats()["adjoint_chunk_bands"]
    upd = nx * ny * nz * NDIR * nb
    r = {"forward_ms": round(fwd, 3), "adjoint_ms": round(bwd, 3), "adjoint_over_forward": round(bwd / fwd, 3),
         "adjoint_gupd_s": round(upd / (bwd * 1e-3) / 1e9, 3),
         "checkpoint": f"{chunk} bands" if chunk > 1 else "1 band", "steps": steps,
         "loss": "sum gI*I_top + 1e-3 sum Q^2 cotangents"}
    del s, chi, S, out, grads
    torch.cuda.empty_cache()
    return r


def _batched_timing(rts, torch, steps):
    """The batched workload: 64 uneven subdomains x 12 bands, FP32 sweep with
    FP64 Q step, one persistent launch inside a CUDA graph, tile height from
    rts_autotune; against 768 separate rts_solve calls (one per subdomain and
    band) on the same data. CUDA events on the solvers' stream."""
    from workloads import band_stack, batched_bands, batched_subdomain_shapes, stratified_atmosphere

    shapes = batched_subdomain_shapes(64, seed=0)
    cs, ss = batched_bands()
    nb = len(cs)
    dev = torch.device("cuda", torch.cuda.current_device())
    chis, Ss = [], []
    for i, (nx, ny, nz) in enumerate(shapes):
        T, _, chi = stratified_atmosphere(nx, ny, nz, seed=i)
        c, s_ = band_stack(T, chi, cs, ss)
        chis.append(torch.as_tensor(c, dtype=torch.float32, device=dev).reshape(-1))
        Ss.append(torch.as_tensor(s_, dtype=torch.float32, device=dev).reshape(-1))
        del T, chi, c, s_
    chi = torch.cat(chis)
    S = torch.cat(Ss)
    del chis, Ss
    side = torch.cuda.Stream()
    best, tune_ms = rts.autotune(shapes, nb, chi, S, precision="fp32", repeats=1, stream=side)
    bs = rts.BatchedSolver(shapes, nb, precision="fp32", tile_rows=best, stream=side)
    g, out = bs.graph(chi, S)

    def timed(fn, n, stream):
        for _ in range(2):
            fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(n):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / n

    ms_b = timed(g.launch, steps, side)
    bs.check()
    st = bs.stats()
    offs = bs.offsets
    del g, bs, out
    torch.cuda.empty_cache()
    # the sweep alone (phase timer of uncaptured solves) against HBM: every
    # unit reads chi, S and writes its 4 slot intensities once per point
    bt = rts.BatchedSolver(shapes, nb, precision="fp32", tile_rows=best, stream=side, timing=True)
    ot = bt.solve(chi, S)
    bt.stats()
    for _ in range(3):
        bt.solve(chi, S, out=ot, check=False)
    torch.cuda.synchronize()
    bt.check()
    stt = bt.stats()
    kernel = stt["sweep_kernel"]
    del bt, ot
    torch.cuda.empty_cache()
    npts = sum(nx * ny * nz for nx, ny, nz in shapes)
    alg = nb * (NDIR // 4) * npts * 24 + nb * (NDIR // 2) * sum(nx * ny for nx, ny, _ in shapes) * 4
    hbm = _peaks().get("hbm_gbs") or 6400.0
    ach = alg / (stt["ms_sweep"] * 1e-3) / 1e9
    roof = {"kernel": "sweep_reg_kernel, one launch for all subdomains" if kernel == 2 else
            "sweep_kernel, one launch per CTA-width class", "bound": "hbm", "achieved": round(ach, 2), "peak": hbm,
            "unit": "GB/s", "frac": round(ach / hbm, 5), "algorithmic_bytes_per_launch": alg,
            "sweep_ms_mean": round(stt["ms_sweep"], 3), "phases_ms": {k: round(stt[k], 3) for k in
                                                                     ("ms_transpose", "ms_sweep", "ms_reduce",
                                                                      "ms_qstep")}}
    # plain FP64 solves, one per subdomain and band: a sample of one band per
    # subdomain (64 solves, band 0's data), scaled to the 768 solves
    ms64 = 0.0
    for (nx, ny, nz), (go, _, _) in zip(shapes, offs):
        n = nx * ny * nz
        so = rts.Solver(nx, ny, nz, 1, precision="fp64", stream=side)
        c64 = chi[go:go + n].double().view(1, nz, ny, nx)
        s64 = S[go:go + n].double().view(1, nz, ny, nx)
        o64 = so.solve(c64, s64)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(side)
        so.solve(c64, s64, out=o64, check=False)
        b.record(side)
        torch.cuda.synchronize()
        so.check()
        ms64 += a.elapsed_time(b)
        del so, c64, s64, o64
    torch.cuda.empty_cache()
    ms64 *= nb
    # separate solves: one handle per subdomain (one band), 12 calls each
    singles = []
    for (nx, ny, nz) in shapes:
        so = rts.Solver(nx, ny, nz, 1, precision="fp32", stream=side)
        singles.append((so, so.solve(chi[:nx * ny * nz].view(1, nz, ny, nx), S[:nx * ny * nz].view(1, nz, ny, nx))))
    views = []
    for (nx, ny, nz), (go, _, _) in zip(shapes, offs):
        n = nx * ny * nz
        views.append([(chi[go + b * n:go + (b + 1) * n].view(1, nz, ny, nx),
                       S[go + b * n:go + (b + 1) * n].view(1, nz, ny, nx)) for b in range(nb)])

    def all_separate():
        for (so, o), vs in zip(singles, views):
            for c, s_ in vs:
                so.solve(c, s_, out=o, check=False)

    ms_s = timed(all_separate, max(1, min(steps, 3)), side)
    for so, _ in singles:
        so.check()
    del singles, views
    torch.cuda.empty_cache()
    upd = sum(nx * ny * nz for nx, ny, nz in shapes) * NDIR * nb
    return {"workload": "64 subdomains, Nx=Ny in {48,64,96,128}, Nz in {96,128,192}, x 12 bands, FP32 sweep + FP64 Q",
            "sweep_kernel": "register (one persistent launch)" if kernel == 2 else "shared (per CTA-width class)",
            "batched_ms": round(ms_b, 3), "separate_ms": round(ms_s, 3), "speedup": round(ms_s / ms_b, 3),
            "batched_gupd_s": round(upd / (ms_b * 1e-3) / 1e9, 3), "separate_gupd_s": round(upd / (ms_s * 1e-3) / 1e9, 3),
            "separate": "768 rts_solve calls (one per subdomain and band), same precision",
            "separate_fp64_ms": round(ms64, 3), "speedup_over_fp64_separate": round(ms64 / ms_b, 3),
            "separate_fp64": "768 plain FP64 rts_solve calls: 64 timed (one band per subdomain) x 12",
            "roofline": roof, "tile_rows": best, "autotune_ms": {str(k): round(v, 3) for k, v in tune_ms.items()},
            "units": st["n_units"], "tiles": st["n_tiles"], "grid": st["grid"], "launch": "cuda graph",
            "sweep_launches_per_solve": 1 if kernel == 2 else None}


def _large_timing(rts, torch):
    """The large anisotropic workload: 512 x 512 x 256, 16 bands, FP32 sweep
    with compensated accumulation; forward solve and the per-band-checkpoint
    adjoint (loss on I_top and Q_rad). Runs last: about 230 GB on the device."""
    from workloads import stratified_atmosphere
    from workloads.atmosphere import _bands

    nx, ny, nz, nb = 512, 512, 256, 16
    T, _, chi0 = stratified_atmosphere(nx, ny, nz, 0)
    cs, ss = _bands("sixteen", nb)
    S4 = T ** 4
    torch.cuda.empty_cache()
    s = rts.Solver(nx, ny, nz, nb, precision="fp32_compensated", adjoint=True, timing=True)
    c = torch.empty((nb, nz, ny, nx), dtype=torch.float32, device="cuda")
    Sd = torch.empty_like(c)
    for b in range(nb):
        c[b] = torch.as_tensor(chi0 * cs[b], dtype=torch.float32)
        Sd[b] = torch.as_tensor(S4 * ss[b], dtype=torch.float32)
    del T, chi0, S4
    out = s.solve(c, Sd)
    gI = torch.randn(out["I_top"].shape, dtype=torch.float32, device="cuda", generator=torch.Generator("cuda").manual_seed(0))
    gQ = 1e-3 * out["Q"]
    g = s.adjoint(c, Sd, gI_top=gI, gQ=gQ)
    s.stats()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(2):
        s.solve(c, Sd, out=out, check=False)
    e1.record()
    torch.cuda.synchronize()
    fwd = e0.elapsed_time(e1) / 2
    st = s.stats()
    e0.record()
    s.adjoint(c, Sd, gI_top=gI, gQ=gQ, out=g, check=False)
    e1.record()
    torch.cuda.synchronize()
    s.check()
    adj = e0.elapsed_time(e1)
    sa = s.stats()
    upd = nx * ny * nz * NDIR * nb
    r = {"workload": "512x512x256, 16 bands (chi x 10^(4b/15), S = T^4/16), FP32 sweep, compensated accumulation",
         "forward_ms": round(fwd, 2), "gupd_s": round(upd / (fwd * 1e-3) / 1e9, 3),
         "phases_ms": {k: round(st[k], 2) for k in ("ms_transpose", "ms_sweep", "ms_reduce", "ms_qstep")},
         "adjoint_ms": round(adj, 2), "adjoint_over_forward": round(adj / fwd, 3),
         "adjoint_phases_ms": [round(x, 2) for x in sa["ms_adjoint"]],
         "checkpoint": f"{sa['adjoint_chunk_bands']} bands (automatic)",
         "wrap": {"mean_warmup_planes": st["mean_warmup_steps"], "max_warmup_planes": st["max_warmup_steps"]}}
    del s, c, Sd, out, g, gI, gQ
    torch.cuda.empty_cache()
    return r


def _extensions_timing(rts, torch, chi, S, solve_ms, peak):
    """The solver's extensions on the bench workload (FP32): the spatial
    decomposition into 4 slabs of levels iterated on their boundary
    intensities (against the undecomposed solve's outputs and time), the
    scattering source iteration S = (1 - eps) J + eps B (eps = 0.3, from
    S = B), and the MHD -> RTS input step (trilinear interpolation of ln T,
    ln rho and the band table lookup) with its bytes against HBM. CUDA
    events on the current stream."""
    import numpy as np
    from workloads.opacity import mhd_fields, synthetic_table

    def timed(fn, n=3):
        fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(n):
            r = fn()
        b.record()
        torch.cuda.synchronize()
        return a.elapsed_time(b) / n, r

    res = {}
    ref = rts.Solver(NX, NY, NZ, NB, precision="fp32").solve(chi, S)
    dsol = rts.DecomposedSolver(NX, NY, NZ, NB, nblocks=4, precision="fp32")
    ms, (out, iters) = timed(lambda: dsol.solve(chi, S))
    dq = float((out["Q"] - ref["Q"]).abs().max() / ref["Q"].abs().max())
    res["decomposition"] = {"slabs": 4, "ms": round(ms, 2), "iterations": iters, "over_undecomposed": round(ms / solve_ms, 2),
                            "q_rad_max_diff_rel_to_max": dq}
    del dsol, out
    ssol = rts.Solver(NX, NY, NZ, NB, precision="fp32", scatter=True)
    eps = torch.full_like(S, 0.3)
    ms, (S_new, out, iters) = timed(lambda: ssol.scatter_solve(chi, S, eps), n=1)
    res["scattering"] = {"eps": 0.3, "ms": round(ms, 2), "iterations": iters, "ms_per_iteration": round(ms / max(iters, 1), 2)}
    del ssol, S_new, out, eps
    T, rho = mhd_fields(NX, NY, NZ, seed=0)
    tab = synthetic_table(nb=NB)
    Td = torch.tensor(T, dtype=torch.float32, device="cuda")
    rd = torch.tensor(rho, dtype=torch.float32, device="cuda")
    tab = dict(tab, ln_kappa=torch.tensor(tab["ln_kappa"], dtype=torch.float32, device="cuda"),
               ln_B=torch.tensor(tab["ln_B"], dtype=torch.float32, device="cuda"))
    fe_out = (torch.empty((NB, NZ, NY, NX), device="cuda"), torch.empty((NB, NZ, NY, NX), device="cuda"))
    ms, _ = timed(lambda: rts.front_end(Td, rd, tab, precision="fp32", out=fe_out), n=20)
    nbytes = (2 + 2 * NB) * 4 * NX * NY * NZ  # T, rho read; chi_b, S_b written
    res["front_end"] = {"ms": round(ms, 3), "algorithmic_bytes": nbytes, "achieved_gbs": round(nbytes / (ms * 1e-3) / 1e9, 1),
                        "frac_of_hbm": round(nbytes / (ms * 1e-3) / 1e9 / peak, 4)}
    del Td, rd, fe_out
    torch.cuda.empty_cache()
    return res


def _sequence_timing(rts, torch, s, chi, S, stream, steps=6):
    """Cold solves and warm-started solves of a slowly changing atmosphere:
    ms per solve (library phase timer: sweep) and the planes each x/y group
    sweeps beyond one period (mean, max)."""
    import numpy as np

    seed = torch.zeros(s.wrap_seed_elems(), dtype=torch.float32, device=chi.device)
    res = {}
    for mode in ("cold", "warm"):
        sweeps, mean_w, max_w = [], [], []
        s.stats()
        for n in range(steps):
            Sn = S * (1.0 + 1e-5 * n) ** 4
            if mode == "cold":
                s.solve(chi, Sn, check=False)
            else:
                s.solve(chi, Sn, check=False, wrap_seed=seed, seed_in=n > 0)
            st = s.stats()
            if n > 0:
                sweeps.append(st["ms_sweep"])
                mean_w.append(st["mean_warmup_steps"])
                max_w.append(st["max_warmup_steps"])
        res[mode] = {"sweep_ms": round(float(np.mean(sweeps)), 3), "extra_planes_mean": round(float(np.mean(mean_w)), 1),
                     "extra_planes_max": int(max(max_w))}
    res["change_per_step"] = "S = T^4 grows by 4e-5 relative per step"
    res["warm_criterion"] = ("the wrap plane's change over a period r and the bound's one-period contraction gam "
                             "(tracked in the first period): every plane of the accumulated period carries at most "
                             "1e-6 relative error (seed error <= r / (1 - gam))")
    return res


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    import paper_2107_08145_b300 as rts
    from workloads import workload

    ws, rank, local = _dist()
    if ws > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    prec = args.precision
    chi64, S64 = workload(WORKLOAD, nx=NX, ny=NY, nz=NZ)
    upd = NX * NY * NZ * NDIR * NB

    def barrier():
        if ws > 1:
            dist.barrier()

    def max_over_ranks(v):
        if ws == 1:
            return v
        t = torch.tensor([v], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    stream = torch.cuda.current_stream()
    if ws > 1:
        # band sharding (weak scaling): the atmosphere has 4 bands per rank;
        # rank r solves bands 4r .. 4r+3 (the 4-band set, sources scaled by
        # 1/ws) and one all-reduce of J, F, Q_rad per solve forms the band sums
        from paper_2107_08145_b300.sharded import ShardedSolver

        sh = ShardedSolver(NX, NY, NZ, NB * ws, precision=prec, timing=True, stream=stream,
                           tile_rows=args.tile_rows)
        assert (sh.b0, sh.b1) == (NB * rank, NB * (rank + 1))
        s = sh.local
        S64 = S64 / ws
        solve = sh.solve
    else:
        s = rts.Solver(NX, NY, NZ, NB, precision=prec, timing=True, stream=stream, tile_rows=args.tile_rows)
        solve = s.solve
    chi = torch.as_tensor(chi64, dtype=s.dtype, device=dev)
    S = torch.as_tensor(S64, dtype=s.dtype, device=dev)
    out = solve(chi, S)
    for _ in range(args.warmup):
        solve(chi, S, out=out, check=False)
    s.check()
    s.stats()  # resets the phase timer
    clk = ClockSampler(local)
    barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with clk:
        e0.record(stream)
        for _ in range(args.steps):
            solve(chi, S, out=out, check=False)
        e1.record(stream)
        torch.cuda.synchronize()
    barrier()
    ms = e0.elapsed_time(e1) / args.steps
    ms = max_over_ranks(ms)
    s.check()
    st = s.stats()
    global TILE_ROWS
    TILE_ROWS = st["tile_rows"]
    value = ws * upd / (ms * 1e-3) / 1e9

    peaks = _peaks()
    hbm = peaks.get("hbm_gbs")
    sweep_ms = st["ms_sweep"]
    alg = sweep_algorithmic_bytes(prec)
    achieved = alg / (sweep_ms * 1e-3) / 1e9
    kname = {2: "sweep_reg_kernel (register-resident persistent tile-DAG sweep, all bands and groups)",
             1: "sweep_kernel (shared-memory persistent tile-DAG sweep, all bands and groups)"}.get(
                 st["sweep_kernel"], "sweep")
    roofline = {"kernel": kname,
                "bound": "hbm", "achieved": round(achieved, 2), "peak": hbm if hbm else 6400.0,
                "unit": "GB/s", "frac": round(achieved / (hbm if hbm else 6400.0), 5),
                "peak_source": "of measured" if hbm else "of fallback",
                "traffic": _traffic_from_profile(prec, (NX, NY, NZ), TILE_ROWS, st["sweep_kernel"]),
                "algorithmic_bytes_per_launch": alg,
                "sweep_ms_mean": round(sweep_ms, 4), "launches_timed": st["timed_solves"]}
    if roofline["traffic"]:  # the same fraction from the DRAM bytes ncu measured
        roofline["frac_dram"] = round(roofline["traffic"] / (sweep_ms * 1e-3) / 1e9 / roofline["peak"], 5)
    phases = {k: round(st[k], 4) for k in ("ms_transpose", "ms_sweep", "ms_reduce", "ms_qstep")}

    extra = {}
    # FP64 solve of the same workload (the plain FP64 reference form)
    if not args.skip_fp64 and prec != "fp64":
        s64 = rts.Solver(NX, NY, NZ, NB, precision="fp64", timing=True, stream=stream)
        c64 = torch.as_tensor(chi64, dtype=torch.float64, device=dev)
        S64d = torch.as_tensor(S64, dtype=torch.float64, device=dev)
        o64 = s64.solve(c64, S64d)
        s64.stats()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        n64 = 2
        for _ in range(n64):
            s64.solve(c64, S64d, out=o64, check=False)
        f1.record(stream)
        torch.cuda.synchronize()
        s64.check()
        ms64 = max_over_ranks(f0.elapsed_time(f1) / n64)
        st64 = s64.stats()
        extra["fp64"] = {"value": round(ws * upd / (ms64 * 1e-3) / 1e9, 4), "unit": "Gupd/s",
                         "ms_per_step": round(ms64, 3), "sweep_ms": round(st64["ms_sweep"], 3),
                         "roofline": _fp64_roofline(st64)}
        extra["fp32_over_fp64"] = round(ms64 / ms, 2)
        del s64, c64, S64d, o64

    # end to end through the public C API with host buffers: pipelined
    # (rts_solve_host_async: each step copies its inputs in and its outputs
    # out, overlapped with the neighbouring steps' solves) and serial
    # (rts_solve_host: copy in, solve, copy out, synchronise)
    e2e = None
    if not args.skip_e2e:
        npdt = np.float64 if prec == "fp64" else np.float32
        tdt = torch.float64 if prec == "fp64" else torch.float32
        hc = torch.from_numpy(chi64.astype(npdt)).pin_memory().numpy()
        hS = torch.from_numpy(S64.astype(npdt)).pin_memory().numpy()
        pin = lambda shape, dt: torch.empty(shape, dtype=dt).pin_memory().numpy()  # noqa: E731
        mk = lambda: dict(I_top=pin((NB, 12, NY, NX), tdt), J=pin((NZ, NY, NX), torch.float64),  # noqa: E731
                          F=pin((3, NZ, NY, NX), torch.float64), Q=pin((NZ, NY, NX), torch.float64))
        houts = [mk(), mk()]
        h2d = hc.nbytes + hS.nbytes
        d2h = sum(v.nbytes for v in houts[0].values())
        sa = rts.Solver(NX, NY, NZ, NB, precision=prec, host_io_async=True, stream=stream)
        for i in range(2):
            sa.solve_host_async(hc, hS, houts[i])
        sa.host_wait()
        ke = max(3, min(args.steps, 10))
        barrier()
        t0 = time.perf_counter()
        for i in range(ke):
            sa.solve_host_async(hc, hS, houts[i & 1])
        sa.host_wait()
        dt = max_over_ranks((time.perf_counter() - t0) / ke)
        del sa
        sh = rts.Solver(NX, NY, NZ, NB, precision=prec, host_io=True, stream=stream)
        sh.solve_host(hc, hS, out=houts[0])
        ks = max(1, min(args.steps, 5))
        t0 = time.perf_counter()
        for _ in range(ks):
            sh.solve_host(hc, hS, out=houts[0])
        dts = max_over_ranks((time.perf_counter() - t0) / ks)
        del sh
        e2e = {"value": round(ws * upd / dt / 1e9, 4), "unit": "Gupd/s", "ms_per_step": round(dt * 1e3, 3),
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "steps": ke,
               "api": "rts_solve_host_async on pinned host buffers, host wall clock over the steps incl. the final "
                      "wait; every step copies its inputs in and its outputs out, overlapped with neighbouring steps",
               "serial": {"value": round(ws * upd / dts / 1e9, 4), "ms_per_step": round(dts * 1e3, 3),
                          "api": "rts_solve_host (copy in, solve, copy out, synchronise)"}}

    # adjoint (rts_adjoint) against the forward solve on the same inputs: the
    # 96^3 x 4-band adjoint workload and the 288^3 x 4 workload
    adj = None
    if not args.skip_adjoint:
        adj = {}
        for name, grid in (("adj96x4", (96, 96, 96)), (WORKLOAD, (NX, NY, NZ))):
            # the default (automatic checkpoint chunk), and one band per checkpoint
            adj[name] = _adjoint_timing(rts, torch, workload, name, grid, prec, stream, max(3, min(args.steps, 10)))
            adj[name + "_one_band_checkpoint"] = _adjoint_timing(rts, torch, workload, name, grid, prec, stream,
                                                                max(3, min(args.steps, 10)), chunk=1)
        ratio = adj[WORKLOAD]["adjoint_over_forward"]
    else:
        ratio = None

    # warm-started time sequence: the atmosphere of step n has T x (1 + 1e-5 n)
    # (a slowly evolving MHD state); every solve is started from the previous
    # solve's wrap planes (rts_boundary.wrap_seed) against the same sequence
    # solved cold, both with the library's phase timer
    sequence = None
    if not args.skip_sequence and prec != "fp64" and ws == 1:
        sequence = _sequence_timing(rts, torch, s, chi, S, stream)

    # the extensions on the same workload: spatial decomposition, scattering
    # iteration, MHD -> RTS input step
    extensions = None
    if not args.skip_extensions and prec != "fp64" and ws == 1:
        extensions = _extensions_timing(rts, torch, chi, S, ms, hbm if hbm else 6400.0)

    batched = None
    if not args.skip_batched:
        batched = _batched_timing(rts, torch, max(3, min(args.steps, 10)))

    large = None
    if not args.skip_large:
        del s, chi, S, out  # the headline solver's ~25 GB, before the ~230 GB large run
        torch.cuda.empty_cache()
        large = _large_timing(rts, torch)

    cpu = None
    if rank == 0 and not args.skip_cpu_baseline:
        cpu = cpu_baseline(args.cpu_seconds)

    line = {"metric": METRIC, "value": round(value, 4), "unit": "Gupd/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(ms, 4), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32" if prec != "fp64" else "f64", "data": "synthetic",
            "config": _config(prec, ws, st["sweep_kernel"]), "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
            "clocks": clk.summary(), "gpu_launches": st["kernels_per_solve"] * args.steps,
            "phases_ms": phases,
            "solve_bytes": (_solve_bytes(prec, ms, roofline["traffic"])
                            if (NX, NY, NZ) == (288, 288, 288) and st["sweep_kernel"] == 2 else None),
            "wrap": {"max_warmup_planes": st["max_warmup_steps"], "mean_warmup_planes": st["mean_warmup_steps"]},
            "adjoint_over_forward": ratio, "adjoint": adj, "batched": batched, "large": large,
            "sequence": sequence, "extensions": extensions}
    line.update(extra)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()


# ----------------------------------------------------------------------------
# CPU oracle
# ----------------------------------------------------------------------------
def _oracle_sample(oracle, chi, S, bands, dirs, threads):
    """Oracle solve of a sample: the given bands, a subset of the 24 rays."""
    n, w = oracle.a4_quadrature()
    P = oracle.Problem(NX, NY, NZ, len(bands), n=n[dirs], w=w[dirs] * (NDIR / len(dirs)), max_wrap_iters=100000)
    t0 = time.perf_counter()
    P.solve(chi[bands], S[bands], nthreads=threads)
    return time.perf_counter() - t0


def cpu_baseline(budget_s):
    """The oracle as it stands on this host's cores, on a bounded sample of
    the workload: bands taken one at a time (all 24 rays) until the budget is
    used; Gupd/s over what was solved."""
    import oracle
    from workloads import workload

    chi, S = workload(WORKLOAD, nx=NX, ny=NY, nz=NZ)
    threads = oracle.default_threads()
    done, t = 0, 0.0
    for b in range(NB):
        t += _oracle_sample(oracle, chi, S, [b], list(range(NDIR)), threads)
        done += 1
        if t >= budget_s:
            break
    return {"value": round(NX * NY * NZ * NDIR * done / t / 1e9, 5), "unit": "Gupd/s", "cores": threads,
            "kind": "oracle", "seconds": round(t, 2),
            "sample": f"bands 0..{done - 1} of rts288x4 (all 24 rays, full 288^3 grid), FP64 C oracle, "
                      f"OpenMP over rays on {threads} threads"}


def run_reference(args):
    """CPU oracle arm: each step solves a bounded sample of the workload."""
    import oracle
    from workloads import workload

    ws, rank, _ = _dist()
    if rank != 0:
        return
    chi, S = workload(WORKLOAD, nx=NX, ny=NY, nz=NZ)
    threads = oracle.default_threads()
    # one step: one band, a chunk of rays (one per thread), cycling through
    # bands and rays so the whole run covers the workload evenly
    chunk = min(NDIR, max(4, threads))
    times, work = [], 0
    for it in range(args.warmup + args.steps):
        b = it % NB
        d0 = (it * chunk) % NDIR
        dirs = [(d0 + k) % NDIR for k in range(chunk)]
        dt = _oracle_sample(oracle, chi, S, [b], dirs, threads)
        if it >= args.warmup:
            times.append(dt)
            work += NX * NY * NZ * len(dirs)
    tot = sum(times)
    value = work / tot / 1e9
    ms = tot / args.steps * 1e3
    sample = (f"per step: one band x {chunk} of the 24 rays of rts288x4 (full 288^3 grid), FP64 C oracle, "
              f"OpenMP over rays on {threads} threads")
    line = {"impl": "reference", "metric": METRIC, "value": round(value, 5), "unit": "Gupd/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 2), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": _config(args.precision),
            "cpu_baseline": {"value": round(value, 5), "unit": "Gupd/s", "cores": threads, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": round(value, 5), "unit": "Gupd/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--precision", choices=("fp32", "fp32_compensated", "fp64"), default="fp32")
    ap.add_argument("--tile-rows", type=int, default=0, help="rows per sweep tile (0 = library default)")
    ap.add_argument("--skip-fp64", action="store_true")
    ap.add_argument("--skip-e2e", action="store_true")
    ap.add_argument("--skip-cpu-baseline", action="store_true")
    ap.add_argument("--skip-adjoint", action="store_true")
    ap.add_argument("--skip-batched", action="store_true")
    ap.add_argument("--skip-large", action="store_true")
    ap.add_argument("--skip-sequence", action="store_true")
    ap.add_argument("--skip-extensions", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--grid", default="288,288,288",
                    help="NX,NY,NZ override (profiling of smaller cases); the metric is quoted at 288^3")
    args = ap.parse_args()
    global NX, NY, NZ
    NX, NY, NZ = (int(v) for v in args.grid.split(","))
    if args.warmup < 3 and args.impl == "ours":
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
