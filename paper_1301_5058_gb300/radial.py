"""Radial colony runs, the 2D workload of Sec. 3: a colony grows from the
central Gaussian inoculum (Eq. inibacexp) on the full grid, and its envelope
radius R_env(t) (the largest cell-centre distance with b >= b_th) is sampled
as it spreads.  The envelope velocity is the FP64 least-squares slope of
R_env(t) over the second half of the run; the branch count is the number of
circular runs of b >= b_th on the circle r = 0.8 R_env.

Usage: python -m paper_1301_5058_gb300.radial [--n=16384] [--steps=50000]
       [--samples=50] [--chi0=0,1] [--precision=f32]
prints one JSON line per chi0.
"""
from __future__ import annotations

import json
import sys
import time

import numpy as np

import paper_1301_5058_gb300 as cx
from paper_1301_5058_gb300 import workloads as W
from paper_1301_5058_gb300.surrogate import count_runs, lsq_slope


def radial_run(cfg: dict, steps: int, samples: int = 50, precision: int = cx.CX_PREC_F32,
               nsamples: int = 4096) -> dict:
    """Run `cfg` (a workload dict) for `steps` steps, sampling the
    diagnostics `samples` times.  Returns the R_env series, the velocity fit,
    conservation and positivity at the end, and the final branch count."""
    grid, params, seed = W.split(cfg)
    params["precision"] = precision
    every = max(1, steps // samples)
    t, r = [], []
    t0 = time.perf_counter()
    with cx.Sim(grid["nx"], grid["ny"], grid["dx"], seed=seed, **params) as sim:
        d0 = sim.diagnostics()
        for _ in range(samples):
            sim.step(every)
            d = sim.diagnostics(check=False)
            t.append(d["t"])
            r.append(d["r_env"])
        p = cx.cx_get_config(sim.h)[1]
        level = p.b_threshold if p.b_threshold > 0 else 0.1 * p.theta * p.n0
        prof = cx.cx_polar_profile(sim.h, 0.8 * d["r_env"], nsamples)
    wall = time.perf_counter() - t0
    t, r = np.asarray(t), np.asarray(r)
    half = samples // 2
    return {
        "nx": grid["nx"], "ny": grid["ny"], "n0": cfg["n0"], "chi0": cfg["chi0"],
        "sigma0": cfg["sigma0"], "noise_amp": cfg["noise_amp"], "steps": every * samples,
        "t": t.tolist(), "r_env": r.tolist(),
        "velocity_second_half": lsq_slope(t[half:], r[half:]),
        "velocity_last_quarter": lsq_slope(t[3 * samples // 4:], r[3 * samples // 4:]),
        "invariant_rel_drift": abs(d["invariant"] - d0["invariant"]) / d0["invariant"],
        "min_b": d["min_b"], "min_n": d["min_n"], "finite": d["finite"],
        "branches": count_runs(prof, level), "wall_seconds": wall,
    }


def main(argv):
    kw = dict(n=16384, steps=50000, samples=50, chi0="0,1", precision="f32")
    for a in argv:
        k, _, v = a.lstrip("-").partition("=")
        kw[k] = v
    n, steps, samples = int(kw["n"]), int(kw["steps"]), int(kw["samples"])
    prec = cx.CX_PREC_F32 if kw["precision"] == "f32" else cx.CX_PREC_F64
    for chi0 in (float(c) for c in str(kw["chi0"]).split(",")):
        cfg = dict(W.CONFIG1, nx=n, ny=n, chi0=chi0)
        print(json.dumps(radial_run(cfg, steps, samples, prec)), flush=True)


if __name__ == "__main__":
    main(sys.argv[1:])
