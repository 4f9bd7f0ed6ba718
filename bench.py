"""Benchmark of the fused FP32 time-stepper on the 16384^2 single-grid
workload (n0 = 0.35, sigma0 = 4, a = 0.8, chi0 = 1, inoculum bM = 0.71 with
r0^2 = 32^2, dt = 0.2 x the stability limit).

One benchmark step = `--window` time steps (one fused kernel launch per two
time steps) followed by one diagnostics reduction (masses, invariant,
envelope radius).  The metric is grid-cell updates per second.  Every input
is larger than L2 (3.2 GB read per time step), so no L2 flush is needed
between iterations.

The same line carries, under "records", the other parts of the metric,
each timed the same way with its own roofline and clock samples: the FP64
state at 4096^2 (against the FP64 pipe's rate, measured in this run by
cx_alu_peak), the paper's own scheme (Heun, sigma redrawn every step from a
triangular law) at 16384^2, and the 512-instance batched parameter sweep
(sweep points per hour).  The CPU leg times the FP64 oracle on one core and
on all host cores, and checks each record's path against the oracle on a
small case of the same configuration ("oracle_error").

Multi-GPU (torchrun): every rank runs its own replica of the grid (the
workload partitions into independent simulations; no data-path
collective); the time is the maximum over ranks and the value counts the
cells of all ranks (weak scaling).

--impl reference times the FP64 CPU oracle (the reference arm) on a bounded
sample of the same workload on the host cores.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# algorithmic HBM bytes per cell and time step.  One pass reads b, n (and
# the sigma array for static noise) and writes b', n'.  Unfused, Euler takes
# one pass per step and Heun two, the second also reading the start-of-step
# state pointwise; fused (time block 2), one pass takes two Euler steps or a
# whole Heun step.
def bytes_per_cell(prec, scheme, noise, time_block=1):
    w = 4 if prec == "f32" else 8
    one_pass = (5 if noise == "static" else 4) * w
    if time_block == 2:
        return one_pass / 2 if scheme == "euler" else one_pass
    return one_pass if scheme == "euler" else one_pass + one_pass + 2 * w


# kernel launches of cx_step(S)
def launches_per_window(scheme, time_block, S):
    if time_block == 2:
        return S // 2 + S % 2 if scheme == "euler" else S
    return S if scheme == "euler" else 2 * S


# Algorithmic floating-point work per cell-update of the scheme as written
# (receptor law, central mobility; a multiply-add counts two): 14 flops per
# face (sums, differences, the receptor weight with one division, the flux
# products), two faces per cell, 15 for the update (reaction, divergences and
# their scale factors); Heun takes two stages and the mean (u0 + u) / 2 of b
# and n.  Peak rates from the unit counts at the
# sampled maximum SM clock: 128 FP32 lanes per SM, and for FP64 2
# multiply-adds per SM and clock (GB300's nominal 1.25 TFLOP/s at 2.07 GHz on
# 152 SMs), a multiply-add being two flops.
FLOPS_PER_CELL_UPDATE = {"euler": 2 * 14 + 15, "heun": 2 * (2 * 14 + 15) + 4}
SMS = 152


def alu_peak_tflops(prec, sm_mhz):
    fma_per_sm = 128 if prec == "f32" else 2
    return 2 * fma_per_sm * SMS * sm_mhz * 1e6 / 1e12


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--window", type=int, default=100, help="time steps per benchmark step")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=16384, help="grid side")
    ap.add_argument("--chi0", type=float, default=1.0)
    ap.add_argument("--precision", default="f32", choices=["f32", "f64"])
    ap.add_argument("--scheme", default="euler", choices=["euler", "heun"])
    ap.add_argument("--noise", default="static", choices=["static", "per-step"])
    ap.add_argument("--dist", default="uniform", choices=["uniform", "triangular"])
    ap.add_argument("--time-block", type=int, default=None, choices=[1, 2],
                    help="explicit stages per pass over the grid (temporal blocking depth); "
                         "default: the library's (2 for FP32, 1 for FP64)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default="grid",
                    choices=["grid", "sweep", "validated", "screen-training"],
                    help="grid: the 16384^2 single grid; sweep: the batched parameter sweep; "
                         "validated: validated sweep points/hour with the learned screen "
                         "(solver-labelled training runs at 1024^2, held-out points on the "
                         "512..2048 size mix; several minutes); screen-training: Adam steps "
                         "of the screen's 8-member network (batch 256)")
    ap.add_argument("--n-train", type=int, default=8192, help="validated: training runs")
    ap.add_argument("--n-test", type=int, default=1024, help="validated: held-out points")
    ap.add_argument("--count", type=int, default=512, help="sweep instances")
    ap.add_argument("--point-steps", type=int, default=20000, help="time steps per sweep point")
    ap.add_argument("--tune", action="store_true", help="autotune the batch before timing")
    ap.add_argument("--no-records", action="store_true",
                    help="time only the headline grid (no FP64, paper-scheme or sweep records)")
    return ap.parse_args()


def workload(spec):
    """The single-grid workload dict of a spec (a dict with n and chi0, or
    the parsed command line)."""
    from paper_1301_5058_gb300 import workloads as W
    get = spec.get if isinstance(spec, dict) else lambda k: getattr(spec, k)
    return dict(W.CONFIG1, nx=get("n"), ny=get("n"), chi0=get("chi0"))


def config_block(spec, cfg, world=1):
    get = spec.get if isinstance(spec, dict) else lambda k: getattr(spec, k)
    w = 4 if get("precision") == "f32" else 8
    fields = 2 if get("noise") == "per-step" else 3
    read = fields * cfg["nx"] * cfg["ny"] * w
    return {"workload": f"single grid {cfg['nx']}x{cfg['ny']} {get('precision')} state, "
                        f"n0={cfg['n0']} sigma0={cfg['sigma0']} a={cfg['noise_amp']} "
                        f"chi0={cfg['chi0']} receptor law, {get('noise')} {get('dist')} noise, "
                        f"{'forward Euler' if get('scheme') == 'euler' else 'Heun RK2'}, "
                        f"dt=0.2 x limit",
            "nx": cfg["nx"], "ny": cfg["ny"], "time_steps_per_step": get("window"),
            "time_block": get("time_block"),
            "diagnostics_per_step": 1,
            "l2": f"inputs larger than L2 ({fields} fields x {read / fields / 2**20:.0f} MiB read "
                  "per pass); no flush",
            "parallelism": f"replicas x{world}" if world > 1 else "single GPU"}


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def _traffic_record(name):
    """profiles/<name>_traffic.json, or None when it is missing or any kernel
    source it lists changed since the capture."""
    path = os.path.join(ROOT, "profiles", f"{name}_traffic.json")
    csrc = os.path.join(ROOT, "paper_1301_5058_gb300", "csrc")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        rec = json.load(f)
    if not rec.get("sources_sha256_16"):
        return None
    for src, h in rec["sources_sha256_16"].items():
        p = os.path.join(csrc, src)
        if not os.path.exists(p) or hashlib.sha256(open(p, "rb").read()).hexdigest()[:16] != h:
            return None
    return rec


def kernel_traffic(prec, name, nx, ny, scheme, noise):
    """ncu DRAM bytes per launch of kernel `name` ("step_kernel" or
    "fused_kernel") on an nx x ny grid, if recorded for that grid, scheme and
    noise mode and the current sources of that kernel (null otherwise)."""
    rec = _traffic_record(name)
    if rec is None or nx != ny:
        return None
    entries = rec.get(prec, [])
    for entry in entries if isinstance(entries, list) else [entries]:
        if (entry.get("scheme"), entry.get("noise")) == (scheme, noise):
            v = entry.get(f"dram_bytes_per_launch_{nx}sq")
            if v is not None:
                return v
    return None


def sweep_issue_count(count, tuning):
    """ncu warp instructions per launch of the two-stage batch kernel on the
    512-instance sweep, recorded with its traffic (null otherwise)."""
    rec = _traffic_record("batch_fused_kernel")
    if rec is None or count != 512:
        return None
    entry = rec.get("f32", {})
    if any(tuning.get(k) != v for k, v in entry.get("tuning", {}).items()):
        return None
    return entry.get("warp_instructions_per_launch")


def kernel_issue_count(prec, name, nx, ny, scheme, noise):
    """ncu warp instructions per launch of kernel `name` on an nx x ny grid,
    recorded with the traffic (null when not recorded or the sources changed)."""
    rec = _traffic_record(name)
    if rec is None or nx != ny:
        return None
    entries = rec.get(prec, [])
    for entry in entries if isinstance(entries, list) else [entries]:
        if (entry.get("scheme"), entry.get("noise")) == (scheme, noise):
            return entry.get(f"warp_instructions_per_launch_{nx}sq")
    return None


def issue_roofline(warp_inst_per_launch, cell_updates_per_launch, rate, sm_mhz):
    """Instruction-issue roofline of a launch: its warp instructions per
    cell-update times the measured cell-update rate, against one warp
    instruction per scheduler and clock (4 schedulers per SM)."""
    if not warp_inst_per_launch:
        return None
    w = warp_inst_per_launch / cell_updates_per_launch
    peak = 4 * SMS * sm_mhz * 1e6
    return {"bound": "issue", "unit": "warp instructions/s",
            "warp_instructions_per_cell_update": w, "achieved": w * rate, "peak": peak,
            "frac": w * rate / peak,
            "peak_kind": f"4 schedulers x {SMS} SMs x {sm_mhz:.0f} MHz (median SM clock of "
                         "the timed region), one warp instruction each per clock",
            "source": "ncu smsp__inst_executed.sum per launch, recorded with the traffic"}


def sweep_traffic(count, tuning):
    """ncu DRAM bytes per launch of the two-stage batch kernel on the
    512-instance sweep, if recorded for this tuning and the current sources
    (null otherwise)."""
    rec = _traffic_record("batch_fused_kernel")
    if rec is None or count != 512:
        return None
    entry = rec.get("f32", {})
    if any(tuning.get(k) != v for k, v in entry.get("tuning", {}).items()):
        return None
    return entry.get("dram_bytes_per_launch")


class ClockSampler:
    """nvidia-smi samples of the SM clock and throttle reasons, taken during
    the timed region."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                mx = float(f[1])
            except ValueError:
                continue
            for nm, v in zip(names, f[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# Cross-rank pieces (replicas: each rank runs an independent grid; only the
# timing crosses ranks)

def replica_seed(base: int, rank: int) -> int:
    """Seed of rank's replica: the workload's seed plus the rank, so the
    replicas are independent draws of the same configuration."""
    return int(base) + int(rank)


def max_over_ranks(values, world):
    """Element-wise maximum over ranks of a list of floats (the slowest rank
    sets the time); identity when world == 1.  Uses the current process
    group (NCCL tensors live on the GPU, gloo tensors on the CPU)."""
    if world <= 1:
        return [float(v) for v in values]
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.tolist()]


def grid_spec(args):
    """What one single-grid measurement runs, from the command line."""
    return dict(n=args.n, chi0=args.chi0, precision=args.precision, scheme=args.scheme,
                noise=args.noise, dist=args.dist, time_block=args.time_block,
                window=args.window)


def _sim_params(cx, spec, cfg):
    from paper_1301_5058_gb300 import workloads as W
    grid, params, seed = W.split(cfg)
    params["precision"] = cx.CX_PREC_F32 if spec["precision"] == "f32" else cx.CX_PREC_F64
    params["scheme"] = cx.CX_SCHEME_EULER if spec["scheme"] == "euler" else cx.CX_SCHEME_HEUN
    params["noise_mode"] = cx.CX_NOISE_STATIC if spec["noise"] == "static" else cx.CX_NOISE_PER_STEP
    params["noise_dist"] = cx.CX_NOISE_UNIFORM if spec["dist"] == "uniform" else cx.CX_NOISE_TRIANGULAR
    return grid, params, seed


def gpu_uuid(dev):
    import torch
    try:
        return "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        i = dev.index or 0
        return os.environ.get("CUDA_VISIBLE_DEVICES", str(i)).split(",")[i]


def run_grid(spec, K, Wm, rank, world, local_rank, with_e2e):
    """Time K benchmark steps (after Wm warm-up steps) of one single grid;
    with_e2e also times the same loop end to end with host buffers."""
    import ctypes

    import torch

    import paper_1301_5058_gb300 as cx

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    cfg = workload(spec)
    grid, params, seed = _sim_params(cx, spec, cfg)
    seed = replica_seed(seed, rank)
    sim = cx.Sim(grid["nx"], grid["ny"], grid["dx"], seed=seed, **params)
    stream = torch.cuda.current_stream(dev)
    cx.cx_set_stream(sim.h, stream.cuda_stream)
    if spec["time_block"] is not None:
        cx.cx_set_time_block(sim.h, spec["time_block"])
    time_block = cx.cx_get_time_block(sim.h)
    cells = cfg["nx"] * cfg["ny"]
    S = spec["window"]

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    def bench_step(ev=None):
        if ev is not None:
            ev[0].record(stream)
        cx.cx_step(sim.h, S)
        if ev is not None:
            ev[1].record(stream)
        return cx.cx_diagnostics(sim.h)

    for _ in range(Wm):
        bench_step()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(K)]
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.synchronize()
    with ClockSampler(gpu_uuid(dev)) as clk:
        start.record(stream)
        for k in range(K):
            d = bench_step(evs[k])
        stop.record(stream)
        torch.cuda.synchronize()
    barrier()
    elapsed = start.elapsed_time(stop) / 1e3
    kernel_s = sum(a.elapsed_time(b) for a, b in evs) / 1e3
    per_step = kernel_s / (K * S)

    # end to end through the C ABI with host buffers: every step uploads its
    # inputs (b, n) from pinned host memory and reads the diagnostics back.
    # The upload of the next step's inputs is staged (cx_stage_state) while
    # the current step computes, and committed before that step starts.
    e2e = None
    if with_e2e:
        f32 = spec["precision"] == "f32"
        hb = torch.empty((cfg["ny"], cfg["nx"]), dtype=torch.float32 if f32 else torch.float64,
                         pin_memory=True)
        hn = torch.empty_like(hb, pin_memory=True)
        cx.cx_get_field(sim.h, cx.CX_FIELD_B, hb.numpy())
        cx.cx_get_field(sim.h, cx.CX_FIELD_N, hn.numpy())

        def e2e_run(steps):
            cx.cx_stage_state(sim.h, hb, hn)
            for k in range(steps):
                cx.cx_commit_state(sim.h)
                cx.cx_step(sim.h, S)
                if k + 1 < steps:
                    cx.cx_stage_state(sim.h, hb, hn)
                cx.cx_diagnostics(sim.h)

        e2e_run(max(1, Wm))
        # the two uploads alone (nothing to hide them behind), best of three
        up = []
        for _ in range(3):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            cx.cx_stage_state(sim.h, hb, hn)
            cx.cx_commit_state(sim.h)
            torch.cuda.synchronize()
            up.append(time.perf_counter() - t0)
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e2e_run(K)
        torch.cuda.synchronize()
        barrier()
        e2e_s = time.perf_counter() - t0
        nbytes = 2 * cells * hb.element_size()
        e2e = {"seconds": e2e_s,
               "h2d_bytes_per_step": nbytes,
               "d2h_bytes_per_step": ctypes.sizeof(cx.cx_diag) + 64,
               "uploads_alone_ms": min(up) * 1e3,
               "upload_gbs": nbytes / min(up) / 1e9}
    diag = d.as_dict()
    sim.close()
    return {"elapsed": elapsed, "kernel_s": kernel_s, "per_step": per_step, "cells": cells,
            "clocks": clk.summary(), "e2e": e2e, "diag": diag, "cfg": cfg,
            "time_block": time_block}


LIMITER_TB2 = ("instruction issue: two stages per pass halve the HBM bytes per cell-update, "
               "and the pass is then held by the thread instructions it issues per cell "
               "(profiles/fused_kernel_f32_16384sq.md)")
LIMITER_HEUN = ("instruction issue: both Heun stages and the Philox draw of sigma run in one "
                "pass, so each cell-update issues two stages' face arithmetic plus the "
                "generator (profiles/fused_kernel_f32_16384sq.md)")


def grid_line(spec, r, K, world, peak, peak_kind, alu_peaks):
    """The JSON fields of one single-grid measurement."""
    cfg, cells, S = r["cfg"], r["cells"], spec["window"]
    tb = r["time_block"]
    prec, scheme, noise = spec["precision"], spec["scheme"], spec["noise"]
    units = cells * S * K * world
    bpc = bytes_per_cell(prec, scheme, noise, tb)
    lpw = launches_per_window(scheme, tb, S)
    kernel = "fused_kernel" if tb == 2 else "step_kernel"
    per_step = r["per_step"]
    rate = cells / per_step  # cell-updates/s of the step kernels alone
    sm_mhz = r["clocks"].get("sm_max_mhz") or 2070.0
    measured = alu_peaks.get(prec)
    alu = {"bound": "alu", "unit": "TFLOP/s",
           "flops_per_cell_update": FLOPS_PER_CELL_UPDATE[scheme],
           "achieved": FLOPS_PER_CELL_UPDATE[scheme] * rate / 1e12}
    if measured:
        alu["peak"] = measured / 1e12
        alu["peak_kind"] = ("measured in this run: cx_alu_peak, register-only multiply-add "
                            f"kernel in {prec}")
    else:
        alu["peak"] = alu_peak_tflops(prec, sm_mhz)
        alu["peak_kind"] = (f"derived: {'128 FP32' if prec == 'f32' else '2 FP64'} multiply-adds "
                            f"per SM and clock x {SMS} SMs x {sm_mhz:.0f} MHz")
    alu["frac"] = alu["achieved"] / alu["peak"]
    achieved = bpc * rate / 1e9
    hbm = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
           "frac": achieved / peak, "peak_kind": f"{peak_kind} hbm_gbs",
           "kernel": kernel,
           "traffic": kernel_traffic(prec, kernel, cfg["nx"], cfg["ny"], scheme, noise),
           "algorithmic_bytes_per_cell": bpc,
           "kernel_ms_per_time_step": per_step * 1e3,
           # the HBM-roofline rate of a one-step-per-pass stepper (20 B per
           # FP32 cell-update): temporal blocking may pass it
           "one_step_pass_roofline_cell_updates_per_s":
               peak * 1e9 / bytes_per_cell(prec, scheme, noise, 1),
           "kernel_cell_updates_per_s": rate,
           "launches_per_time_step": lpw / S}
    if prec == "f64":
        # the FP64 pass is bound by the FP64 pipe: that is its roofline
        roofline = dict(alu, kernel=kernel, traffic=hbm["traffic"], kernel_cell_updates_per_s=rate,
                        kernel_ms_per_time_step=per_step * 1e3, hbm=hbm)
    else:
        roofline = dict(hbm, alu_fp32=alu)
        if tb == 2:
            roofline["limiter"] = LIMITER_TB2 if scheme == "euler" else LIMITER_HEUN
            clock = r["clocks"].get("sm_mhz") or sm_mhz
            roofline["issue"] = issue_roofline(
                kernel_issue_count(prec, kernel, cfg["nx"], cfg["ny"], scheme, noise),
                cells * (2 if scheme == "euler" else 1), rate, clock)
    return {
        "value": units / r["elapsed"],
        "unit": "cell-updates/s",
        "ms_per_step": r["elapsed"] / K * 1e3,
        "dtype": prec,
        "config": config_block(dict(spec, time_block=tb), cfg, world),
        "roofline": roofline,
        "gpu_launches": K * (lpw + 2),
        "clocks": r["clocks"],
        "diagnostics_last": {k: r["diag"][k] for k in ("step", "t", "invariant", "r_env", "min_b",
                                                        "min_n")},
    }


def cpu_baseline_sample(cfg, side=4096, steps=8, threads=0):
    """Time the FP64 oracle (as it stands; threads > 0: its threaded build
    on that many host threads) on the central side x side window of the
    workload for `steps` time steps."""
    import oracle
    # same parameters and noise law; the inoculum sits at the window's centre
    s = oracle.sigma_field(side, side, cfg["seed"], cfg["sigma0"], cfg["noise_amp"])
    b, n = oracle.initial_state(side, side, cfg["dx"], cfg["n0"], cfg["bM"], cfg["r0sq"])
    dt = cfg["cfl_frac"] * oracle.dt_limit(dx=cfg["dx"], Dn=cfg["Dn"], theta=cfg["theta"],
                                           chi0=cfg["chi0"], n0=cfg["n0"], bM=cfg["bM"],
                                           sigma0=cfg["sigma0"], amp=cfg["noise_amp"])
    kw = dict(dx=cfg["dx"], dt=dt, Dn=cfg["Dn"], theta=cfg["theta"], chi0=cfg["chi0"],
              threads=threads)
    if threads:
        oracle.run(s, b, n, 1, **kw)  # build and warm the threaded library
    t0 = time.perf_counter()
    oracle.run(s, b, n, steps, **kw)
    sec = time.perf_counter() - t0
    how = "threaded build, gcc -O2 -fopenmp" if threads else "gcc -O2, one thread"
    return side * side * steps / sec, sec, \
        f"central {side}x{side} window of the workload, {steps} FP64 oracle steps ({sec:.1f} s; {how})"


# ---------------------------------------------------------------------------
# The CPU leg's parity checks: each record's path, on a small grid of the same
# configuration, against the FP64 oracle from the same initial state.

ORACLE_CHECK_STEPS = 200


def _rel_l2(x, y):
    import numpy as np
    d = float(np.linalg.norm((np.asarray(x, np.float64) - y).ravel()))
    return d / max(float(np.linalg.norm(np.asarray(y).ravel())), 1e-300)


def _oracle_reference(cfg, spec, nx, ny, seed, steps):
    """The oracle's run of `steps` steps of configuration cfg on nx x ny;
    returns (b0, n0, b, n)."""
    import oracle
    per_step = spec["noise"] == "per-step"
    dist = 0 if spec["dist"] == "uniform" else 1
    s = oracle.sigma_field(nx, ny, seed, cfg["sigma0"], cfg["noise_amp"], dist=dist)
    b0, n0 = oracle.initial_state(nx, ny, cfg["dx"], cfg["n0"], cfg["bM"], cfg["r0sq"])
    dt = cfg["cfl_frac"] * oracle.dt_limit(dx=cfg["dx"], Dn=cfg["Dn"], theta=cfg["theta"],
                                           chi0=cfg["chi0"], n0=cfg["n0"], bM=cfg["bM"],
                                           sigma0=cfg["sigma0"], amp=cfg["noise_amp"])
    b, n, _ = oracle.run(s, b0, n0, steps, dx=cfg["dx"], dt=dt, Dn=cfg["Dn"], theta=cfg["theta"],
                         chi0=cfg["chi0"], scheme=0 if spec["scheme"] == "euler" else 1,
                         noise_mode=1 if per_step else 0, seed=seed, sigma0=cfg["sigma0"],
                         amp=cfg["noise_amp"], dist=dist,
                         recipe=1 if spec["precision"] == "f32" else 0)
    return b0, n0, b, n


def oracle_error_grid(spec, nx=288, ny=200, steps=ORACLE_CHECK_STEPS):
    """Relative L2 error of the record's path (precision, scheme, noise,
    stages per pass) against the oracle on an nx x ny grid of the same
    parameters, from the oracle's initial state."""
    import paper_1301_5058_gb300 as cx
    cfg = dict(workload(spec), nx=nx, ny=ny)
    grid, params, seed = _sim_params(cx, spec, cfg)
    b0, n0, ob, on = _oracle_reference(cfg, spec, nx, ny, seed, steps)
    with cx.Sim(nx, ny, grid["dx"], seed=seed, **params) as sim:
        if spec["time_block"] is not None:
            cx.cx_set_time_block(sim.h, spec["time_block"])
        sim.set_field(cx.CX_FIELD_B, b0)
        sim.set_field(cx.CX_FIELD_N, n0)
        sim.step(steps)
        gb, gn = sim.field(cx.CX_FIELD_B), sim.field(cx.CX_FIELD_N)
        tb = cx.cx_get_time_block(sim.h)
    tol = 1e-4 if spec["precision"] == "f32" else 1e-12
    eb, en = _rel_l2(gb, ob), _rel_l2(gn, on)
    return {"rel_l2_b": eb, "rel_l2_n": en, "tolerance": tol, "pass": max(eb, en) <= tol,
            "case": f"{nx}x{ny}, {steps} steps, same parameters, stages per pass {tb}, "
                    f"oracle's initial state"}


def oracle_error_sweep(tuning, steps=ORACLE_CHECK_STEPS):
    """The batch path with the sweep's tuning, on three instances of the
    sweep's kind (smaller sides, one ragged), each against the oracle."""
    import paper_1301_5058_gb300 as cx
    from paper_1301_5058_gb300 import workloads as W
    specs = W.sweep_specs(3, seed=0, steps=steps)
    for sp, side in zip(specs, (160, 224, 97)):
        sp["nx"] = sp["ny"] = side
    spec = dict(precision="f32", scheme="euler", noise="static", dist="uniform")
    worst = (0.0, 0.0)
    with cx.Batch(specs) as bt:
        bt.tune(tuning["tile_rows"], tuning["graph_steps"], tuning["group_bytes"],
                tuning["resident_steps"], tuning["time_block"])
        refs = []
        for i, sp in enumerate(specs):
            cfg = dict(W.CONFIG1, **{k: v for k, v in sp.items() if k != "precision"})
            b0, n0, ob, on = _oracle_reference(cfg, spec, sp["nx"], sp["ny"], sp["seed"], steps)
            bt.set_field(i, cx.CX_FIELD_B, b0)
            bt.set_field(i, cx.CX_FIELD_N, n0)
            refs.append((ob, on))
        bt.step(steps)
        for i, (ob, on) in enumerate(refs):
            gb, gn = bt.field(i, cx.CX_FIELD_B), bt.field(i, cx.CX_FIELD_N)
            worst = (max(worst[0], _rel_l2(gb, ob)), max(worst[1], _rel_l2(gn, on)))
    return {"rel_l2_b": worst[0], "rel_l2_n": worst[1], "tolerance": 1e-4,
            "pass": max(worst) <= 1e-4,
            "case": f"3 instances (160^2, 224^2, 97^2) of the sweep's kind, {steps} steps, "
                    "the sweep's tuning, worst instance"}


def measure_alu_peaks():
    """FP64 and FP32 multiply-add rates of this GPU, measured by cx_alu_peak."""
    import paper_1301_5058_gb300 as cx
    return {"f64": cx.cx_alu_peak(cx.CX_PREC_F64), "f32": cx.cx_alu_peak(cx.CX_PREC_F32)}


RECORDS = {
    "fp64_4096": dict(n=4096, precision="f64", scheme="euler", noise="static", dist="uniform",
                      time_block=None),
    "paper_scheme_16384": dict(n=16384, precision="f32", scheme="heun", noise="per-step",
                               dist="triangular", time_block=None),
}


def screen_training_record(args, members=8, rows=8192, batch=256):
    """Adam steps of the screen's network (members trained together, each on
    its own rows of random data): `warmup` steps, then `steps` steps timed by
    the host clock around the library's synchronous training call (the
    network runs on its own stream)."""
    import numpy as np
    import paper_1301_5058_gb300 as cx
    from paper_1301_5058_gb300 import surrogate
    rng = np.random.default_rng(0)
    X = rng.uniform(-1, 1, (members, rows, 4)).astype(np.float32)
    T = rng.normal(size=(members, rows, 2)).astype(np.float32)
    theta = np.concatenate([surrogate.init_params(k) for k in range(members)])
    with cx.Mlp(rows, theta, members=members) as net:
        net.train(X, T, batch, max(args.warmup, 1), 1e-3)
        t0 = time.perf_counter()
        losses = net.train(X, T, batch, args.steps, 1e-3)
        sec = time.perf_counter() - t0
    return {"metric": "screen training steps/s", "value": args.steps / sec, "unit": "steps/s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * sec / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "bf16 products, f32 accumulation", "data": "synthetic",
            "gpu_launches": 4 * args.steps,
            "config": {"workload": f"surrogate network 4-256-256-2, {members} members trained "
                                   f"together, minibatch {batch} of {rows} rows each"},
            "final_loss": float(np.mean(losses[:, -1]))}


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        return main_reference(args, rank, world)
    if args.workload == "validated":
        import torch
        torch.cuda.set_device(local_rank)
        from paper_1301_5058_gb300 import surrogate
        with ClockSampler(gpu_uuid(torch.device("cuda", local_rank))) as clk:
            v = surrogate.validated_sweep(n_train=args.n_train, n_test=args.n_test,
                                          steps=args.point_steps, verbose=False,
                                          save=os.environ.get("CX_VALIDATED_SAVE"))
        print(json.dumps({"metric": "validated sweep points/hour",
                          "value": v["screened_points_per_hour"], "unit": "points/h",
                          "n_gpus": 1, "higher_is_better": True, "scaling": "weak",
                          "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                          "config": {"workload": "learned screen + batched solver over the "
                                                 "sweep box, sides 512..2048, 20000 steps per "
                                                 "point"},
                          "validated": v, "clocks": clk.summary()}))
        return
    if args.workload == "screen-training":
        import torch
        torch.cuda.set_device(local_rank)
        print(json.dumps(screen_training_record(args)))
        return
    if args.workload == "sweep":
        import torch
        torch.cuda.set_device(local_rank)
        rec = sweep_record(args)
        if not args.no_cpu_baseline:
            rec["oracle_error"] = oracle_error_sweep(rec["config"]["tuning"])
        print(json.dumps(dict({"metric": "sweep points/hour", "n_gpus": 1, "steps": args.steps,
                               "warmup": args.warmup, "higher_is_better": True,
                               "scaling": "weak", "vs_baseline": None, "data": "synthetic"},
                              **rec)))
        return

    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    import torch
    torch.cuda.set_device(local_rank)
    alu_peaks = measure_alu_peaks()

    spec = grid_spec(args)
    K = args.steps
    r = run_grid(spec, K, args.warmup, rank, world, local_rank, not args.no_e2e)
    elapsed, e2e_s, per_step = max_over_ranks(
        [r["elapsed"], (r["e2e"] or {}).get("seconds") or 0.0, r["per_step"]], world)
    r.update(elapsed=elapsed, per_step=per_step)

    # the other parts of the metric, each on this rank's GPU (replicas)
    records = {}
    if not args.no_records:
        for name, rs in RECORDS.items():
            rspec = dict(rs, chi0=args.chi0, window=args.window)
            rr = run_grid(rspec, K, args.warmup, rank, world, local_rank, False)
            el, ps = max_over_ranks([rr["elapsed"], rr["per_step"]], world)
            rr.update(elapsed=el, per_step=ps)
            records[name] = (rspec, rr)
    sweep = None
    if not args.no_records and world == 1:
        sweep = sweep_record(args)

    if rank != 0:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return

    peak, peak_kind = peaks()
    cells = r["cells"]
    units = cells * args.window * K * world
    line = grid_line(spec, r, K, world, peak, peak_kind, alu_peaks)
    out = {
        "metric": "grid-cell updates/s",
        "value": line["value"],
        "unit": "cell-updates/s",
        "n_gpus": world,
        "steps": K,
        "warmup": args.warmup,
        "ms_per_step": line["ms_per_step"],
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": args.precision,
        "data": "synthetic (seeded sigma field and Gaussian inoculum)",
        "config": line["config"],
        "roofline": line["roofline"],
        "gpu_launches": line["gpu_launches"],
        "clocks": line["clocks"],
        "diagnostics_last": line["diagnostics_last"],
        "alu_peaks_measured": {"f64_tflops": alu_peaks["f64"] / 1e12,
                               "f32_tflops": alu_peaks["f32"] / 1e12,
                               "how": "cx_alu_peak: 8 independent multiply-add chains per thread, "
                                      "4 blocks of 256 threads per SM, best of 5, CUDA events"},
    }
    if r["e2e"]:
        out["e2e"] = {"value": units / e2e_s, "unit": "cell-updates/s",
                      "h2d_bytes_per_step": r["e2e"]["h2d_bytes_per_step"],
                      "d2h_bytes_per_step": r["e2e"]["d2h_bytes_per_step"],
                      "uploads_alone_ms": r["e2e"]["uploads_alone_ms"],
                      "upload_gbs": r["e2e"]["upload_gbs"],
                      "how": "cx_stage_state (b, n from pinned host memory, overlapping the "
                             "previous step), cx_commit_state, cx_step, cx_diagnostics "
                             "(device-to-host read) every step; host wall clock"}
    cpu_leg = not args.no_cpu_baseline and world == 1
    if records or sweep:
        out["records"] = {}
        for name, (rspec, rr) in records.items():
            rec = grid_line(rspec, rr, K, world, peak, peak_kind, alu_peaks)
            rec["metric"] = "grid-cell updates/s"
            if cpu_leg:
                rec["oracle_error"] = oracle_error_grid(rspec)
            out["records"][name] = rec
        if sweep:
            if cpu_leg:
                sweep["oracle_error"] = oracle_error_sweep(sweep["config"]["tuning"])
            out["records"]["sweep_512"] = sweep
    if cpu_leg:
        out["oracle_error"] = oracle_error_grid(spec)
        v, sec, sample = cpu_baseline_sample(r["cfg"])
        out["cpu_baseline"] = {"value": v, "unit": "cell-updates/s", "cores": 1, "kind": "oracle",
                               "sample": sample}
        try:
            import oracle
            threads = os.cpu_count() or 1
            v, sec, sample = cpu_baseline_sample(r["cfg"], steps=32, threads=threads)
            out["cpu_baseline_all_cores"] = {"value": v, "unit": "cell-updates/s",
                                             "cores": oracle.omp_threads(), "kind": "oracle",
                                             "sample": sample}
        except Exception as e:  # no OpenMP on this host: report why
            out["cpu_baseline_all_cores"] = {"unavailable": f"{type(e).__name__}: {e}"}
    print(json.dumps(out))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def sweep_record(args):
    """Batched parameter sweep (512 instances, sides 512..2048, FP32): sweep
    points per hour of the batch, and of the same points stepped one
    simulation at a time through cx_step (both measured in this run; each
    point is `--point-steps` time steps plus its creation)."""
    import torch

    import paper_1301_5058_gb300 as cx
    from paper_1301_5058_gb300 import autotune
    from paper_1301_5058_gb300 import workloads as W

    specs = W.sweep_specs(args.count, seed=0, steps=args.point_steps)
    S, K, Wm = args.window, args.steps, args.warmup
    cells = sum(s["nx"] * s["ny"] for s in specs)
    stream = torch.cuda.Stream()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    bt = cx.Batch(specs)
    create_s = time.perf_counter() - t0
    cx.cx_batch_set_stream(bt.h, stream.cuda_stream)
    bt._stream = stream
    if args.tune:
        autotune.tune_batch(bt, steps=64, reps=2, use_cache=False)
    else:
        # the autotuner's choice on this sweep (128-row tiles, 64-step graphs,
        # two stages per pass), fixed so that the default run needs no search
        bt.tune(128, 64, 0, 0, 2)
    choice = cx.cx_batch_get_tuning(bt.h)
    depth = cx.cx_batch_get_time_block(bt.h)

    def timed(step_fn, diag_fn):
        for _ in range(Wm):
            step_fn(S)
            diag_fn()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(K)]
        start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        start.record(stream)
        for k in range(K):
            evs[k][0].record(stream)
            step_fn(S)
            evs[k][1].record(stream)
            diag_fn()
        stop.record(stream)
        stop.synchronize()
        return start.elapsed_time(stop) / 1e3, sum(a.elapsed_time(b) for a, b in evs) / 1e3

    with ClockSampler(gpu_uuid(torch.device("cuda", torch.cuda.current_device()))) as clk:
        elapsed, kernel_s = timed(bt.step, bt.diagnostics)
    per_step = elapsed / (K * S)
    batch_pph = args.count * 3600.0 / (args.point_steps * per_step + create_s)
    bt.close()

    # the same points, one simulation at a time (one per size class timed)
    single = {}
    for side in sorted({s["nx"] for s in specs}):
        spec = next(s for s in specs if s["nx"] == side)
        kw = {k: v for k, v in spec.items() if k not in ("nx", "ny", "dx", "seed")}
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sim = cx.Sim(side, side, 1.0, seed=spec["seed"], **kw)
        c_s = time.perf_counter() - t0
        cx.cx_set_stream(sim.h, stream.cuda_stream)
        el, _ = timed(sim.step, sim.diagnostics)
        single[side] = (el / (K * S), c_s)
        sim.close()
    single_total = sum(args.point_steps * single[s["nx"]][0] + single[s["nx"]][1] for s in specs)
    single_pph = args.count * 3600.0 / single_total
    peak, peak_kind = peaks()
    bpc = bytes_per_cell("f32", "euler", "static", depth)
    achieved = bpc * cells / (kernel_s / (K * S)) / 1e9
    tuning = {"tile_rows": choice[0], "graph_steps": choice[1], "group_bytes": choice[2],
              "resident_steps": choice[3], "time_block": depth}
    return {
        "metric": "sweep points/hour", "value": batch_pph, "unit": "points/h",
        "ms_per_step": elapsed / K * 1e3, "dtype": "f32",
        "config": {"workload": f"batched sweep: {args.count} instances, sides from "
                               f"{sorted(set(s['nx'] for s in specs))}, (n0, chi0, sigma0) log grid, "
                               f"static uniform noise a=0.5, forward Euler, {args.point_steps} steps "
                               f"per point", "cells_per_time_step": cells,
                   "time_steps_per_step": S, "tuning": tuning,
                   "l2": "inputs larger than L2 (20 GB of state); no flush"},
        "cell_updates_per_s": cells / per_step,
        "single_instance_points_per_hour": single_pph,
        "single_instance_ms_per_time_step": {str(k): v[0] * 1e3 for k, v in single.items()},
        "speedup_vs_single_instance": batch_pph / single_pph,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "peak_kind": f"{peak_kind} hbm_gbs",
                     "traffic": sweep_traffic(args.count, tuning),
                     "kernel": "batch_fused_kernel" if depth == 2 else "batch_step_kernel",
                     "algorithmic_bytes_per_cell": bpc,
                     "issue": issue_roofline(sweep_issue_count(args.count, tuning) if depth == 2
                                             else None, 2 * cells, cells / (kernel_s / (K * S)),
                                             clk.summary().get("sm_mhz") or 2070.0)},
        "gpu_launches": K * (launches_per_window("euler", depth, S) + 2),
        "clocks": clk.summary(),
    }


def main_reference(args, rank, world):
    """The reference arm: the FP64 oracle on the host cores, each step one
    oracle time step on the central 4096^2 window of the same workload."""
    if rank != 0:
        return
    cfg = workload(args)
    import oracle
    side = min(4096, cfg["nx"])
    s = oracle.sigma_field(side, side, cfg["seed"], cfg["sigma0"], cfg["noise_amp"])
    b, n = oracle.initial_state(side, side, cfg["dx"], cfg["n0"], cfg["bM"], cfg["r0sq"])
    dt = cfg["cfl_frac"] * oracle.dt_limit(dx=cfg["dx"], Dn=cfg["Dn"], theta=cfg["theta"],
                                           chi0=cfg["chi0"], n0=cfg["n0"], bM=cfg["bM"],
                                           sigma0=cfg["sigma0"], amp=cfg["noise_amp"])
    kw = dict(dx=cfg["dx"], dt=dt, Dn=cfg["Dn"], theta=cfg["theta"], chi0=cfg["chi0"])
    for _ in range(args.warmup):
        b, n = oracle.step(s, b, n, **kw)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        b, n = oracle.step(s, b, n, **kw)
    sec = time.perf_counter() - t0
    value = side * side * args.steps / sec
    sample = f"central {side}x{side} window of the workload, one FP64 oracle step per benchmark step"
    print(json.dumps({
        "impl": "reference", "metric": "grid-cell updates/s", "value": value,
        "unit": "cell-updates/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": sec / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": config_block(args, cfg),
        "cpu_baseline": {"value": value, "unit": "cell-updates/s", "cores": 1, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "cell-updates/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }))


if __name__ == "__main__":
    main()
