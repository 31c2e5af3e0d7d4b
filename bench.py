"""Benchmark of one ExpRK22 / WENO5 / FFT step on the B300.

A bench "step" is one full ExpRK22 step (Algorithm 2, STEP 1-4: two WENO5
row passes fused with the tau-FFTs and two column passes fused with the
y-FFTs and the phi-multipliers, plus the per-step FP64 diagnostics) over the
FP64 4096 x 2048 stratified-atmosphere workload with a seeded N-wave.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line on rank 0.  Under torchrun each rank advances its own
replica of the workload (independent propagations, no collective): weak
scaling, value = all ranks' grid-point-steps / the slowest rank's time.
``--impl reference`` times the FP64 CPU oracle on the host cores instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2103_06080_b300 import inputs  # noqa: E402

METRIC = "grid-point-steps/s"
UNIT = "pt-steps/s"
WORKLOAD = "fp64 4096x2048 stratified N-wave (sigma-cubic B, A), CFL 0.4"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")


def _peaks():
    try:
        with open(PEAKS_FILE) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0}, "fallback"


# the headers that hold the device code of each timed pass (kernel bodies and
# everything they include); a change to any of them voids a stored capture
_ROW_SRC = ("kzk_common.cuh", "kzk_fft.cuh", "kzk_weno.cuh", "kzk_kernels.cuh")
KERNEL_SOURCES = {
    ("row_stage1", "fp64"): _ROW_SRC, ("row_stage2", "fp64"): _ROW_SRC,
    ("row_stage1", "fp32"): _ROW_SRC + ("kzk_colpipe.cuh", "kzk_rowpair.cuh"),
    ("row_stage2", "fp32"): _ROW_SRC + ("kzk_colpipe.cuh", "kzk_rowpair.cuh"),
    ("col_stage1", "fp64"): _ROW_SRC, ("col_stage2", "fp64"): _ROW_SRC,
    ("col_stage1", "fp32"): _ROW_SRC + ("kzk_colpipe.cuh", "kzk_rowpair.cuh", "kzk_colpair.cuh"),
    ("col_stage2", "fp32"): _ROW_SRC + ("kzk_colpipe.cuh", "kzk_rowpair.cuh", "kzk_colpair.cuh"),
}


def source_hash(files) -> str:
    """First 12 hex digits of the SHA-256 of the named csrc/ files, in order."""
    import hashlib
    d = os.path.join(ROOT, "paper_2103_06080_b300", "csrc")
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(d, f), "rb") as fh:
            h.update(f.encode() + b"\0" + fh.read())
    return h.hexdigest()[:12]


def measured_traffic(kernel: str, prec: str):
    """DRAM bytes (read + write) of one launch of the pass `kernel` from the
    ncu summaries under profiles/ (lines 'traffic <kernel> <prec> <bytes> src
    <hash>'), or None when no capture matches the current device code."""
    d = os.path.join(ROOT, "profiles")
    if (kernel, prec) not in KERNEL_SOURCES:
        return None
    want = source_hash(KERNEL_SOURCES[(kernel, prec)])
    try:
        names = sorted(os.listdir(d))
    except OSError:
        return None
    for f in names:
        if not f.endswith((".md", ".txt")):
            continue
        for line in open(os.path.join(d, f)):
            t = line.strip().strip("`").split()
            if len(t) == 6 and t[0] == "traffic" and t[1] == kernel and t[2] == prec and t[4] == "src" and t[5] == want:
                return float(t[3])
    return None


# --------------------------------------------------------------------------
# algorithmic work per launch (also stated in the design notes)
# --------------------------------------------------------------------------
def row_bytes(nx, ny, w, sub=False):
    """Row pass: read one packed spectral array, write one (N * w bytes each);
    sub (the second stage of FP32 plans on row and column pairs): also reads
    b1, to store b2 - b1."""
    return (3 if sub else 2) * nx * ny * w


def col_bytes(nx, ny, w, stage, comp=False, diff=False):
    """Column pass: stage 1 reads V, b1 and the folded E' (or (E - 1)'), P1'
    (half an array each) and writes V*; stage 2 reads b1, b2 (diff: the one
    array b2 - b1), V*, folded P2' and writes V'.  comp (the compensated FP32
    state): each stage also reads and writes the lo part (a bf16 pair per
    complex value: half an array)."""
    unit = nx * ny * w
    tab = (ny // 2 + 1) * (nx // 2) * 2 * w
    lo = unit if comp else 0                        # lo in + lo out, half an array each
    return (3 * unit + 2 * tab + lo) if stage == 1 else ((3 if diff else 4) * unit + tab + lo)


# WENO5 per point and evaluation: the Jiang-Shu reconstruction counted as
# written (about 130 additions and multiplications for the split fluxes, the
# candidate stencils, the smoothness indicators, the weights and the
# difference) plus its 8 divisions, each counted as one operation
WENO5_FLOPS = 130 + 8


def row_flops(nx, ny, profile=True):
    """Row pass FLOPs (add, mul, div = 1; FMA = 2): two real FFTs of length nx
    (2.5 nx log2(nx/2) each, as complex FFTs of nx/2 points, plus 4 per point
    for the real pre/post-processing), WENO5 (WENO5_FLOPS per point),
    diagnostics (3) and the absorption-deviation term (5 with a profile)."""
    lg = np.log2(nx // 2)
    per_pt = 2 * (2.5 * lg + 4) + WENO5_FLOPS + 3 + (5 if profile else 0)
    return per_pt * nx * ny


def col_flops(nx, ny, stage, ysig=False):
    """Column pass FLOPs: complex FFTs of length ny (5 ny log2 ny each) on
    nx/2 columns -- three in stage 1 (two forward, one inverse) plus two
    complex multiply-adds per element; two in stage 2 plus one complex multiply
    and two complex adds per element.  ysig (FP64 plans carrying the state's
    y-spectrum): two transforms in each stage; stage 1 forms three complex
    products and two sums per element, stage 2 one product and one sum."""
    lg = np.log2(ny)
    ncol = nx // 2
    if ysig:
        return ncol * (2 * 5 * ny * lg + ny * (22 if stage == 1 else 8))
    if stage == 1:
        return ncol * (3 * 5 * ny * lg + ny * 14)
    return ncol * (2 * 5 * ny * lg + ny * 10)


# --------------------------------------------------------------------------
# multi-rank aggregation (replicas: independent work per rank, no collective
# on the data path; only the timing is reduced)
# --------------------------------------------------------------------------
def reduce_max(x: float, device, world: int) -> float:
    """Max of a per-rank scalar over all ranks (identity on one rank)."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(points_per_rank_step: float, steps: int, world: int, seconds_max: float) -> float:
    """Weak scaling: every rank advances its own replica; the job's rate is
    all ranks' grid-point-steps over the slowest rank's time."""
    return points_per_rank_step * steps * world / seconds_max


# --------------------------------------------------------------------------
# clocks sampled during the timed region
# --------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200",
                 "-i", str(self.idx), "-f", self.path],
                stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        try:
            for line in open(self.path):
                f = [x.strip() for x in line.split(",")]
                if len(f) < 9:
                    continue
                try:
                    sm.append(float(f[1]))
                    mx.append(float(f[2]))
                except ValueError:
                    continue
                for n, v in zip(names, f[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(n)
            os.unlink(self.path)
        except Exception:
            pass
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------------------
# reference arm: the FP64 CPU oracle on the host cores
# --------------------------------------------------------------------------
def cpu_oracle_rate(w, n_steps: int, threads: bool = True, budget_s: float = 0.0):
    """Grid-point-steps/s of the oracle as it stands on the full grid of ``w``:
    one untimed first step (it pays the first touch of the oracle's work
    arrays), then m timed steps, each timed inside the oracle (table set-up
    excluded).  With budget_s > 0, m is the number of steps that fit in about
    budget_s seconds estimated from the first step (at most n_steps)."""
    import oracle
    p = oracle.Params(**inputs.oracle_params(w))
    m = max(1, n_steps)
    if budget_s > 0:
        _, s1 = oracle.run_timed(p, w.u0, 2, threads=threads)
        m = max(1, min(n_steps, int(budget_s / max(s1[1], 1e-3))))
    _, sec = oracle.run_timed(p, w.u0, m + 1, threads=threads)
    dt = float(np.sum(sec[1:]))
    return w.nx * w.ny * m / dt, dt, oracle.num_threads(threads), m


def run_reference(args, rank, world):
    """The oracle on the host cores, on this arm's workload and metric.  Each
    bench step is one full-grid oracle step; the number of timed steps is
    bounded (~60 s of CPU work) so the run ends within minutes."""
    if rank != 0:
        return 0
    w = inputs.config(2)
    value, dt, cores, m = cpu_oracle_rate(w, args.steps, budget_s=60.0)
    sample = (f"{m} of the requested {args.steps} full 4096x2048 FP64 steps (time bound), "
              f"OpenMP oracle, first step untimed, then per-step timing inside the oracle")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": m, "warmup": args.warmup, "ms_per_step": 1e3 * dt / m,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "nx": 4096, "ny": 2048},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------------------
# our arm
# --------------------------------------------------------------------------
def run_ours(args, rank, world, local_rank):
    import torch
    import torch.distributed as dist

    from paper_2103_06080_b300 import api

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.current_stream()

    def barrier():
        if world > 1:
            dist.barrier()

    fp32 = args.precision == "fp32"
    w = inputs.config(3 if fp32 else 2)
    tdt = torch.float32 if fp32 else torch.float64
    wsz = 4 if fp32 else 8
    plan = api.Plan.from_workload(w, precision=args.precision)
    u_host = torch.tensor(w.u0, dtype=tdt).pin_memory()
    u = u_host.to(dev, non_blocking=False)

    # warm-up (untimed), then the timed region: exactly K steps
    plan.advance(u, args.warmup, sigma0=0.0)
    torch.cuda.synchronize()
    sampler = ClockSampler(local_rank)
    sampler.start()
    n0 = api.launch_count()
    barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    plan.advance(u, args.steps, sigma0=args.warmup * w.dt)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    ms = e0.elapsed_time(e1)
    launches = api.launch_count() - n0
    clocks = sampler.stop()
    ms_max = reduce_max(ms, dev, world)
    value = whole_job_rate(w.nx * w.ny, args.steps, world, ms_max * 1e-3)

    # per-kernel device times (CUDA events on the launch stream)
    kt = plan.kernel_times(u, min(args.steps, 20), sigma0=0.0)
    names = ["row_stage1", "col_stage1", "row_stage2", "col_stage2"]
    info = plan.info()
    ysig = not fp32 and info["col_kernel"] == "tile"     # FP64 per-tile columns: the y-spectral state
    fl = [row_flops(w.nx, w.ny), col_flops(w.nx, w.ny, 1, ysig), row_flops(w.nx, w.ny), col_flops(w.nx, w.ny, 2, ysig)]
    comp = fp32 and info["fp32_state"] == "compensated"
    # row and column pairs both in use: the stage-2 row pass stores b2 - b1
    diff = info["row_kernel"] == "pair" and info["col_kernel"] == "pair"
    by = [row_bytes(w.nx, w.ny, wsz), col_bytes(w.nx, w.ny, wsz, 1, comp), row_bytes(w.nx, w.ny, wsz, diff),
          col_bytes(w.nx, w.ny, wsz, 2, comp, diff)]
    dom = int(np.argmax(kt))
    peaks, peak_src = _peaks()
    if fp32:
        hbm = peaks["hbm_gbs"] * 1e9
        roof = {"bound": "hbm", "kernel": names[dom], "achieved": by[dom] / (kt[dom] * 1e-3) / 1e9,
                "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": by[dom] / (kt[dom] * 1e-3) / hbm,
                "traffic": measured_traffic(names[dom], "fp32"), "peak_source": f"{peak_src} HBM copy bandwidth",
                "kernel_ms": dict(zip(names, kt))}
    else:
        fp64_peak = api.alu_peak("fp64")
        roof = {"bound": "alu", "kernel": names[dom], "achieved": fl[dom] / (kt[dom] * 1e-3) / 1e12,
                "peak": fp64_peak / 1e12, "unit": "TFLOP/s",
                "frac": fl[dom] / (kt[dom] * 1e-3) / fp64_peak, "traffic": measured_traffic(names[dom], "fp64"),
                "peak_source": "measured FP64 FMA throughput (kzk_alu_peak) on this GPU",
                "kernel_ms": dict(zip(names, kt)),
                "hbm_frac_of_measured": by[dom] / (kt[dom] * 1e-3) / (peaks["hbm_gbs"] * 1e9)}

    # end to end through the public API: pinned host -> device, K steps, result back
    out_host = torch.empty_like(u_host).pin_memory()
    torch.cuda.synchronize()
    barrier()
    t0 = time.perf_counter()
    u.copy_(u_host, non_blocking=True)
    st, _ = plan.advance(u, args.steps, sigma0=0.0, diag=True)
    out_host.copy_(u, non_blocking=True)
    torch.cuda.synchronize()
    t_e2e = time.perf_counter() - t0
    e2e_val = whole_job_rate(w.nx * w.ny, args.steps, world, reduce_max(t_e2e, dev, world))
    state_bytes = w.nx * w.ny * wsz

    extra = {}
    if rank == 0 and not args.quick:
        extra = secondary_reports(args, api, torch, dev, peaks, ms_fp64=None if fp32 else ms_max / args.steps)

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32" if fp32 else "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD.replace("fp64", "fp32") if fp32 else WORKLOAD, "nx": w.nx, "ny": w.ny, "dt": w.dt, "per_rank_instances": 1,
                   "l2": "working set 4 spectral arrays + tables = 0.37 GB > 126 MB L2 (no flush needed)"},
        "roofline": roof,
        "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": state_bytes / args.steps,
                "d2h_bytes_per_step": state_bytes / args.steps,
                "timed": "H2D u0 (pinned) + kzk_advance(K steps, diagnostics) + D2H u; bytes amortised over K",
                "status": st},
        "gpu_launches": int(launches),
        "clocks": clocks,
        "peaks": {"source": peak_src, "hbm_gbs": peaks.get("hbm_gbs")},
    }
    line.update(extra)
    if rank == 0 and not args.no_cpu_baseline:
        w2 = inputs.config(2)
        r, dt, cores, m = cpu_oracle_rate(w2, args.cpu_steps)
        line["cpu_baseline"] = {"value": r, "unit": UNIT, "cores": cores, "kind": "oracle",
                                "sample": f"{m} step(s) of the full 4096x2048 FP64 grid ({dt:.1f} s), "
                                          f"OpenMP oracle, first step untimed, then per-step timing inside the oracle"}
        if not args.quick:
            # the sequential build of the same oracle (the paper's "sequential" column)
            r1, dt1, _, m1 = cpu_oracle_rate(w2, 1, threads=False)
            line["cpu_baseline"]["single_core"] = {
                "value": r1, "unit": UNIT, "cores": 1,
                "sample": f"{m1} step of the full 4096x2048 FP64 grid ({dt1:.1f} s), sequential oracle build"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    plan.close()
    return 0


def cufft_transforms_ms(torch, dev, nx, ny, dtype, reps=20):
    """Device ms of cuFFT (through torch.fft) running only the transforms of
    one step: the tau C2R + R2C of both row passes and the five y transforms
    of the two column passes (three forward, two inverse) -- no WENO, no
    multiplies, no diagnostics.  A timed comparison, not part of the path."""
    u = torch.randn(ny, nx, dtype=dtype, device=dev)
    V = torch.fft.rfft(u, dim=1)

    def one_step():
        for _ in range(2):
            x = torch.fft.irfft(V, n=nx, dim=1)
            torch.fft.rfft(x, dim=1)
        for _ in range(3):
            torch.fft.fft(V, dim=0)
        for _ in range(2):
            torch.fft.ifft(V, dim=0)

    for _ in range(3):
        one_step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        one_step()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


# The paper's four grids (Table 1: N_theta = 7 * 2^(5+s) tau points, N_rho =
# 1250 * 2^(s-1) transverse points, N_sigma = 300 * 2^(s-1) steps) and its
# measured totals on a Titan V (Table 3), as pt-steps/s = N_sigma N_rho
# N_theta / time: context for the same method family on other hardware.
PAPER_SETS = {1: (448, 1250, 300), 2: (896, 2500, 600), 3: (1792, 5000, 1200), 4: (3584, 10000, 2400)}
PAPER_TITANV_S = {"fp64": {1: 1.165, 2: 8.343, 3: 65.13, 4: 851.7}, "fp32": {1: 0.5564, 2: 3.788, 3: 28.31, 4: 392.7}}


def medium_step_work(nx, ny, w):
    """Algorithmic FLOPs and bytes of one random-medium step on the mixed-radix
    path: per stage the coefficient kernel (negligible), the C2R row pass
    (FFT; V in, u out), the y-sweep (y-WENO5 + source; u in, b_y out) and the
    b row pass (tau-WENO5 + FFT; u, b_y in, b out); then the three column
    launches (C1 split in two through the scratch W, C2).  Bytes in units of
    N w (N = nx ny); FP32 adds the lo part of E' (half a unit)."""
    lg = np.log2(nx // 2)
    fft_pt = 2.5 * lg + 4
    stage_flops = nx * ny * (fft_pt + (WENO5_FLOPS + 3) + (2 * fft_pt + WENO5_FLOPS + 3 + 3))
    flops = 2 * stage_flops + col_flops(nx, ny, 1) + col_flops(nx, ny, 2)
    units = 2 * (2 + 2 + 3) + 2.5 + (4.0 if w == 4 else 3.5) + 4.5
    return flops, units * nx * ny * w


def paper_grid_reports(api, torch, dev, sets=None, precisions=("fp64", "fp32"), steps=None, warmup=3):
    """The random-medium step on the paper's mixed-radix grids."""
    peaks, peak_src = _peaks()
    fp64_peak = None
    rep = {"workload": "N-wave through the random medium of Algorithm 1 on the grids of Table 1 "
                       "(tau x y = 7*2^(5+s) x 1250*2^(s-1)); timed steps per set below, pt-steps/s",
           "paper_titan_v": "pt-steps/s from the paper's total times (Table 3; Titan V, its own timing scope)",
           "step_roofline": "whole step: algorithmic FLOPs / time against the measured FP64 FMA peak (fp64), "
                            "algorithmic bytes / time against the measured HBM copy bandwidth (fp32)"}
    for s, (nx, ny, nsig) in PAPER_SETS.items():
        if sets and s not in sets:
            continue
        w = inputs.medium_config(nx, ny, 50)
        row = {"grid": f"{nx}x{ny}", "paper_steps": nsig}
        for name in precisions:
            dtype = torch.float64 if name == "fp64" else torch.float32
            pm = api.Plan.from_workload(w, precision=name)
            u = torch.tensor(w.u0, dtype=dtype, device=dev)
            pm.advance(u, warmup)
            k = steps or max(10, min(200, int(2e9 / (nx * ny * (8 if name == "fp64" else 1)))))
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            pm.advance(u, k)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / k
            ref = nsig * nx * ny / PAPER_TITANV_S[name][s]
            fl, by = medium_step_work(nx, ny, 8 if name == "fp64" else 4)
            if name == "fp64" and fp64_peak is None:
                fp64_peak = api.alu_peak("fp64")      # measured once, on a warm GPU
            roof = ({"bound": "alu", "achieved": fl / (ms * 1e-3) / 1e12, "peak": fp64_peak / 1e12,
                     "unit": "TFLOP/s", "frac": fl / (ms * 1e-3) / fp64_peak} if name == "fp64" else
                    {"bound": "hbm", "achieved": by / (ms * 1e-3) / 1e9, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                     "frac": by / (ms * 1e-3) / (peaks["hbm_gbs"] * 1e9)})
            row[name] = {"value": nx * ny / (ms * 1e-3), "ms_per_step": ms, "steps": k,
                         "stage_ms": pm.kernel_times(u, 3), "step_roofline": roof, "paper_titan_v": ref,
                         "ratio_to_paper": nx * ny / (ms * 1e-3) / ref}
            pm.close()
            del u
        rep[f"set{s}"] = row
    return rep


def small_grid_graph_report(api, torch, dev, reps=5):
    """The plain-method workload (512 x 256, 200 steps) with kzk_advance
    replaying captured step graphs (the default) and with direct launches:
    its arrays (4 x 1 MB FP64) stay in L2 and its kernels are short, so the
    launch path, not HBM, bounds it.  Median of `reps` timed 200-step calls
    after one untimed call."""
    w = inputs.config(1)
    rep = {"workload": "fp64/fp32 512x256 N-wave, 200 steps per call (L2-resident: launch-bound, "
                       "no HBM roofline applies)", "unit": UNIT}
    for prec, dtype in (("fp64", torch.float64), ("fp32", torch.float32)):
        row = {}
        for g in ("on", "off"):
            plan = api.Plan.from_workload(w, precision=prec, graph=g)
            u0 = torch.tensor(w.u0, dtype=dtype, device=dev)
            u = u0.clone()
            plan.advance(u, w.n_steps)
            times = []
            for _ in range(reps):
                u.copy_(u0)
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                plan.advance(u, w.n_steps)
                e1.record()
                torch.cuda.synchronize()
                times.append(e0.elapsed_time(e1))
            ms = statistics.median(times)
            row["graph" if g == "on" else "direct"] = {"value": w.nx * w.ny * w.n_steps / (ms * 1e-3),
                                                       "ms_per_step": ms / w.n_steps}
            plan.close()
        row["graph_speedup"] = row["direct"]["ms_per_step"] / row["graph"]["ms_per_step"]
        rep[prec] = row
    return rep


def secondary_reports(args, api, torch, dev, peaks, ms_fp64=None):
    """FP32 throughput + error, the adjoint/forward cost ratio, the batched
    launch and the cuFFT comparison."""
    out = {}
    # FP32 bulk with FP64-generated tables, same 4096 x 2048 workload
    w3 = inputs.config(3)
    p3 = api.Plan.from_workload(w3, precision="fp32")
    u3 = torch.tensor(w3.u0, dtype=torch.float32, device=dev)
    p3.advance(u3, args.warmup)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    k3 = max(args.steps, 50)
    e0.record()
    p3.advance(u3, k3)
    e1.record()
    torch.cuda.synchronize()
    ms3 = e0.elapsed_time(e1)
    kt3 = p3.kernel_times(u3, 20)
    info3 = p3.info()
    comp3 = info3["fp32_state"] == "compensated"
    # row and column pairs both in use: the stage-2 row pass stores b2 - b1
    diff3 = info3["row_kernel"] == "pair" and info3["col_kernel"] == "pair"
    by3 = [row_bytes(4096, 2048, 4), col_bytes(4096, 2048, 4, 1, comp3), row_bytes(4096, 2048, 4, diff3),
           col_bytes(4096, 2048, 4, 2, comp3, diff3)]
    names = ["row_stage1", "col_stage1", "row_stage2", "col_stage2"]
    dom = int(np.argmax(kt3))
    hbm = peaks["hbm_gbs"] * 1e9
    out["fp32"] = {
        "value": w3.nx * w3.ny * k3 / (ms3 * 1e-3), "unit": UNIT, "ms_per_step": ms3 / k3, "steps": k3,
        "dtype": "f32 (FP64-generated tables rounded once; compensated hi + lo spectral state; FP64 diagnostics)",
        "roofline": {"bound": "hbm", "kernel": names[dom], "achieved": by3[dom] / (kt3[dom] * 1e-3) / 1e9,
                     "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": by3[dom] / (kt3[dom] * 1e-3) / hbm,
                     "traffic": measured_traffic(names[dom], "fp32"), "kernel_ms": dict(zip(names, kt3)),
                     "step_frac": sum(by3) / (sum(kt3) * 1e-3) / hbm},
    }
    # the FP32 passes are bound by instruction issue and latency, not by HBM:
    # the dominant one's algorithmic FLOPs against the measured FP32 FMA peak
    # (the faster of scalar FFMA and packed FFMA2 chains)
    fl3 = [row_flops(4096, 2048), col_flops(4096, 2048, 1), row_flops(4096, 2048), col_flops(4096, 2048, 2)]
    fp32_peak = api.alu_peak("fp32")
    out["fp32"]["roofline"]["alu"] = {
        "achieved": fl3[dom] / (kt3[dom] * 1e-3) / 1e12, "peak": fp32_peak / 1e12, "unit": "TFLOP/s",
        "frac": fl3[dom] / (kt3[dom] * 1e-3) / fp32_peak,
        "peak_source": "measured FP32 FMA throughput (kzk_alu_peak: max of FFMA and FFMA2 chains) on this GPU"}
    if info3["col_kernel"] == "pair":
        # the column passes' tiles (16-byte rows of a column pair, 2048 rows at a
        # 16 KB pitch) go through the tensor memory accelerator; its copy rate
        # for that pattern, measured alone, bounds them before HBM does
        unit = 4096 * 2048 * 4                              # one spectral array
        tab = (2048 // 2 + 8) * 16 * (4096 // 4)            # one pair table (pair_tab_rows x 16 B per pair)
        tma1 = 3 * unit + 2 * tab + unit                    # C1: b1, V, V again, two tables in; V* out
        tma2 = (2 if diff3 else 3) * unit + tab             # C2: b2 - b1 (or b1, b2), V*, P2' in
        strip = api.tile_copy_rate(2048, 2048, "strip")
        contig = api.tile_copy_rate(2048, 2048, "contiguous")
        out["fp32"]["roofline"]["tile_copy_ceiling"] = {
            "strip_gbs": strip / 1e9, "contiguous_gbs": contig / 1e9,
            "col_stage1_tma_gbs": tma1 / (kt3[1] * 1e-3) / 1e9, "col_stage2_tma_gbs": tma2 / (kt3[3] * 1e-3) / 1e9,
            "note": "kzk_tile_copy_rate: copy-only kernel, one CTA per column pair, as many CTAs per SM as the "
                    "stage-1 column pass; strip = the column passes' tile boxes, contiguous = the same bytes per "
                    "CTA as one run; col_stage*_tma = bytes the column passes move through the tensor memory "
                    "accelerator per launch / kernel time"}
    p3.close()
    del u3
    # FP32 error of the precision workload (1024 x 512, 2000 steps, and the full
    # 4096 x 2048 grid) against the FP64 path of this library, which the tests
    # hold to the FP64 oracle within 1e-11 (the oracle itself, 1024 x 512 x
    # 2000 steps, is compared in tests/test_gpu_parity.py)
    if not args.no_error:
        errs = {}
        for nx, ny in ((args.err_nx, args.err_ny), (4096, 2048)):
            we = inputs.config(3, nx=nx, ny=ny, n_steps=args.err_steps)
            res = {}
            for prec in ("fp64", "fp32"):
                pe = api.Plan.from_workload(we, precision=prec)
                ue = torch.tensor(we.u0, dtype=torch.float64 if prec == "fp64" else torch.float32, device=dev)
                pe.advance(ue, we.n_steps)
                res[prec] = ue.double()
                pe.close()
            d = res["fp32"] - res["fp64"]
            errs[f"{nx}x{ny}"] = {"rel_l2": float(d.norm() / res["fp64"].norm()),
                                  "rel_linf": float(d.abs().max() / res["fp64"].abs().max())}
        out["fp32"]["error_vs_fp64"] = {**errs, "case": f"{args.err_steps} steps of the seeded precision "
                                                      "workload; reference: the FP64 path (oracle parity 1e-11)"}
    # adjoint / forward on the adjoint workload (2048 x 1024, checkpoint every 32), FP64 and FP32
    w4 = inputs.config(4, n_steps=args.adj_steps)

    def timed(fn):
        torch.cuda.synchronize()
        t = time.perf_counter()
        r = fn()
        torch.cuda.synchronize()
        return time.perf_counter() - t, r

    def adjoint_cost(prec):
        p4 = api.Plan.from_workload(w4, precision=prec)
        u4 = torch.tensor(w4.u0, dtype=torch.float64 if prec == "fp64" else torch.float32, device=dev)
        y = u4.clone()
        p4.advance(y, 4)                                            # warm-up
        t_fwd, _ = timed(lambda: p4.advance(y, w4.n_steps))
        y = u4.clone()
        t_fwd_ck, _ = timed(lambda: p4.advance_checkpointed(y, w4.n_steps, 0.0, 32))
        g_end = 2 * w4.dtau * y
        t_bwd, _ = timed(lambda: p4.adjoint_checkpointed(g_end))
        t_full, _ = timed(lambda: p4.adjoint(u4, g_end, w4.n_steps, ckpt_every=32))
        p4.close()
        return {"forward_s": t_fwd, "forward_with_checkpoints_s": t_fwd_ck, "backward_s": t_bwd,
                "backward_over_forward": t_bwd / t_fwd,
                "full_gradient_s": t_full, "full_gradient_over_forward": t_full / t_fwd}

    out["adjoint"] = {"workload": f"fp64 2048x1024, {w4.n_steps} steps, checkpoint every 32",
                      **adjoint_cost("fp64"),
                      "note": "backward = per-segment recompute from stored checkpoints + reverse sweep "
                              "(the autograd backward); full gradient = kzk_adjoint from u0 (forward sweep "
                              "with checkpoints + backward)"}
    out["adjoint"]["fp32"] = adjoint_cost("fp32")
    # batched persistent launch: 64 heterogeneous FP32 propagations
    if not args.no_batched:
        ws = inputs.batched_config(seed=5, count=args.batch_count, n_steps=500)
        pts = sum(w.nx * w.ny for w in ws)
        out["batched"] = {"workload": f"{len(ws)} FP32 N-wave propagations, Nx in 1024..8192, Ny in 256..2048 "
                                      f"(seeded), own dsigma and profiles each; {args.batch_steps} steps per call",
                          "unit": UNIT, "points_per_step": pts}
        for mode in ("persistent", "streams"):
            t0 = time.perf_counter()
            bp = api.BatchedPlan(ws, precision="fp32", autotune=True, mode=mode)
            t_plan = time.perf_counter() - t0
            us = [torch.tensor(w.u0, dtype=torch.float32, device=dev) for w in ws]
            bp.advance(us, args.batch_steps)              # captures the graph
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            bp.advance(us, args.batch_steps)
            e1.record()
            torch.cuda.synchronize()
            msb = e0.elapsed_time(e1)
            out["batched"][mode] = {
                "value": pts * args.batch_steps / (msb * 1e-3), "ms_per_step": msb / args.batch_steps,
                "plan_create_s": t_plan, "launch": bp.info(),
                "note": ("one cooperative persistent kernel per call (all instances, grid barriers between "
                         "passes), replayed from a CUDA graph" if mode == "persistent" else
                         "one CUDA graph per call: every instance's own kernels on its own captured stream, "
                         "the instances concurrently")}
            bp.close()
            del us
    out["small_grid_graphs"] = small_grid_graph_report(api, torch, dev)
    # random medium of Algorithm 1 (the paper's inhomogeneous workload) on the same grid
    wm = inputs.medium_config(4096, 2048, 500)
    med = {"workload": f"N-wave through the random medium of Algorithm 1 ({wm.medium.n_modes} modes), 4096x2048, "
                       f"homogeneous B, A; dt from the paper's |U| <= 0.05",
           "dt": wm.dt}
    for name, dtype, k in (("fp64", torch.float64, 20), ("fp32", torch.float32, 100)):
        pm = api.Plan.from_workload(wm, precision=name)
        um = torch.tensor(wm.u0, dtype=dtype, device=dev)
        pm.advance(um, 3)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        pm.advance(um, k)
        e1.record()
        torch.cuda.synchronize()
        msm = e0.elapsed_time(e1) / k
        ktm = pm.kernel_times(um, 5)
        med[name] = {"value": wm.nx * wm.ny / (msm * 1e-3), "unit": UNIT, "ms_per_step": msm, "steps": k,
                     "stage_ms": dict(zip(["rows_stage1 (coefficients + C2R + b pass)", "col_stage1",
                                           "rows_stage2 (coefficients + C2R + b pass)", "col_stage2"], ktm))}
        pm.close()
        del um
    out["random_medium"] = med
    out["paper_grids"] = paper_grid_reports(api, torch, dev)
    # cuFFT comparison on the 4096 x 2048 grid
    cmp = {}
    for name, dtype, ms_ours in (("fp64", torch.float64, ms_fp64), ("fp32", torch.float32, out["fp32"]["ms_per_step"])):
        ms_fft = cufft_transforms_ms(torch, dev, 4096, 2048, dtype)
        cmp[name] = {"cufft_transforms_ms_per_step": ms_fft, "ours_step_ms": ms_ours,
                     "ours_over_cufft": (ms_ours / ms_fft) if ms_ours else None}
    cmp["note"] = ("cuFFT through torch.fft doing only the 4 tau and 5 y transforms of one step (no WENO5, "
                   "no phi-multiplies); ours = the whole fused step through kzk_advance")
    out["cufft_comparison"] = cmp
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--quick", action="store_true", help="skip the FP32 / adjoint secondary reports")
    ap.add_argument("--precision", choices=["fp64", "fp32"], default="fp64",
                    help="precision of the headline workload (fp64: 4096x2048 FP64; fp32: same grid, FP32 bulk)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-error", action="store_true")
    ap.add_argument("--cpu-steps", type=int, default=1)
    ap.add_argument("--ref-steps-per-sample", type=int, default=1)
    ap.add_argument("--err-nx", type=int, default=1024)
    ap.add_argument("--err-ny", type=int, default=512)
    ap.add_argument("--err-steps", type=int, default=2000)
    ap.add_argument("--adj-steps", type=int, default=1000)
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--batch-count", type=int, default=64)
    ap.add_argument("--batch-steps", type=int, default=500)
    ap.add_argument("--paper-set", type=int, choices=[1, 2, 3, 4], default=None,
                    help="instead of the headline: the random-medium step on Set S of the paper's Table 1 "
                         "(mixed-radix grid), --steps timed steps at --precision; prints that report")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.paper_set and args.impl == "ours":
        import torch
        from paper_2103_06080_b300 import api
        rep = paper_grid_reports(api, torch, torch.device("cuda", 0), sets=[args.paper_set],
                                 precisions=(args.precision,), steps=args.steps, warmup=args.warmup)
        print(json.dumps(rep), flush=True)
        return 0
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    rc = run_ours(args, rank, world, local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return rc


if __name__ == "__main__":
    sys.exit(main())
