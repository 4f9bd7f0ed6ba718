"""Front speed of the one-dimensional system of Sec. 4.2 (Eq. velo-system-1d):

    n_t = n_xx - n b,   b_t = (sigma0 n b b_x - chi0 sigma0 n b^2 n_x)_x + n b

on [0, 20] with no-flux ends, n(x, 0) = n0 and b(x, 0) = bM exp(-x^2 / 6.25),
bM = 0.71, sigma0 = 1, constant chemotactic sensitivity.  The half-domain
with a no-flux end at x = 0 is the mirror image of [-20, 20] with the
inoculum at the centre, which is how it runs here: each case is an
nx x 1 strip (a wall in y) of one batch, stepped by the library's kernels.

The front position is the envelope radius at level n0/2 (the midpoint of
the front, as the paper tracks "a point in the vicinity of 0.5"); the speed
is the least-squares slope of that radius against time while the front is
between 30% and 80% of the half-length, after the initial transient.

Run as ``python -m paper_1301_5058_gb300.front_speed`` for the paper's grid
n0 in {0.35, 0.71, 1.07, 2, 3, 4} x chi0 in {0, 1, 2.5, 5, 10}.
"""
from __future__ import annotations

import json
import sys

import numpy as np

import paper_1301_5058_gb300 as cx

PAPER_N0 = (0.35, 0.71, 1.07, 2.0, 3.0, 4.0)
PAPER_CHI0 = (0.0, 1.0, 2.5, 5.0, 10.0)


def strip_spec(n0, chi0, sigma0=1.0, half_length=20.0, dx=0.1, precision=cx.CX_PREC_F64,
               mobility=cx.CX_MOBILITY_CENTRAL):
    nx = int(round(2 * half_length / dx))
    return dict(nx=nx, ny=1, dx=dx, seed=0, n0=n0, chi0=chi0, sigma0=sigma0, noise_amp=0.0,
                bM=0.71, r0sq=6.25, chemo_law=cx.CX_CHEMO_CONSTANT, b_threshold=0.5 * n0,
                precision=precision, mobility=mobility)


def fit_speed(t, r, lo, hi):
    """Least-squares slope of r(t) over the samples with lo <= r <= hi (FP64)."""
    t = np.asarray(t, np.float64)
    r = np.asarray(r, np.float64)
    m = (r >= lo) & (r <= hi)
    if m.sum() < 5:
        return float("nan")
    tt, rr = t[m], r[m]
    tm, rm = tt.mean(), rr.mean()
    return float(((tt - tm) * (rr - rm)).sum() / ((tt - tm) ** 2).sum())


def measure(cases, half_length=20.0, dx=0.1, every=None, max_steps=20_000_000, t_max=400.0,
            precision=cx.CX_PREC_F64, lo_frac=0.3, hi_frac=0.8,
            mobility=cx.CX_MOBILITY_CENTRAL):
    """Front speeds of the (n0, chi0[, sigma0]) `cases`, run as one batch.
    A case is finished when its front passes hi_frac x half_length or its
    time passes t_max.  Returns one dict per case with the speed, the
    furthest front position and the smallest b seen."""
    specs = [strip_spec(*c, half_length=half_length, dx=dx, precision=precision,
                        mobility=mobility) for c in cases]
    hi_r = hi_frac * half_length
    with cx.Batch(specs) as bt:
        d0 = bt.diagnostics()
        dts = [d["dt"] for d in d0]
        # sample often enough that the fastest case crosses the fit window in
        # a few hundred samples
        if every is None:
            every = max(50, int(min(dts) ** -1 * 0.002))
        series = [([], []) for _ in cases]
        done = [False] * len(cases)
        min_b = [0.0] * len(cases)
        steps = 0
        while not all(done) and steps < max_steps:
            bt.step(every)
            steps += every
            for i, d in enumerate(bt.diagnostics(check=False)):
                series[i][0].append(d["t"])
                series[i][1].append(d["r_env"])
                min_b[i] = min(min_b[i], d["min_b"])
                if d["r_env"] >= hi_r or d["t"] >= t_max:
                    done[i] = True
    out = []
    for (case, (t, r), dt, mb) in zip(cases, series, dts, min_b):
        out.append(dict(n0=case[0], chi0=case[1], dt=dt, dx=dx,
                        speed=fit_speed(t, r, lo_frac * half_length, hi_r),
                        samples=len(t), reached=max(r) if r else 0.0, min_b=mb))
    return out


def main(argv):
    if "--refine" in argv:
        # resolution study of the cases with the largest chi0 n0
        for mob in (cx.CX_MOBILITY_CENTRAL, cx.CX_MOBILITY_UPWIND):
            for dx in (0.1, 0.05, 0.025):
                for r in measure([(3.0, 5.0), (4.0, 10.0), (2.0, 2.5)], dx=dx, mobility=mob,
                                 t_max=50.0):
                    r["mobility"] = mob
                    print(json.dumps(r), flush=True)
        return
    cases = [(n0, chi0) for n0 in PAPER_N0 for chi0 in PAPER_CHI0]
    if "--quick" in argv:
        cases = [(n0, chi0) for n0 in (2.0, 3.0) for chi0 in (0.0, 1.0)]
    for r in measure(cases):
        print(json.dumps(r), flush=True)


if __name__ == "__main__":
    main(sys.argv[1:])
