"""Named synthetic workloads and seeded input generators.

Holds parameter sets and random-number recipes only; none of the method's
arithmetic.  Shared by the tests (for both the CUDA path and the oracle), the
benchmark and the smoke check.

CONFIG0   -- 256^2 plain-method case the oracle finishes in seconds
             (Dn = theta = 1, chi0 = 0.5, n0 = 0.7, sigma0 = 4, a = 0.5,
             bM = 0.5, r0^2 = 16, dt = 0.2 x limit, 2000 steps, seed 0)
CONFIG1   -- 16384^2 single large grid, FP32 state, dense-branching regime
             n0 = 0.35, sigma0 = 4, a = 0.8, chi0 in {0, 1}, inoculum
             bM = 0.71 with r0^2 = 32^2, 50000 steps (the paper's run
             geometry scaled up from its 2048^2 grid of Sec. 3)
PAPER_2D  -- the paper's own 2D runs (Sec. 3, Table tabresparam): L = 680,
             N = 2048, dx = L/N, bM = 0.71, r0^2 = 6.25, triangular noise
"""
from __future__ import annotations

import numpy as np

CONFIG0 = dict(nx=256, ny=256, dx=1.0, n0=0.7, chi0=0.5, sigma0=4.0, noise_amp=0.5,
               Dn=1.0, theta=1.0, bM=0.5, r0sq=16.0, cfl_frac=0.2, steps=2000, seed=0)

CONFIG1 = dict(nx=16384, ny=16384, dx=1.0, n0=0.35, chi0=1.0, sigma0=4.0, noise_amp=0.8,
               Dn=1.0, theta=1.0, bM=0.71, r0sq=32.0 ** 2, cfl_frac=0.2, steps=50000, seed=0)

PAPER_2D = dict(nx=2048, ny=2048, dx=680.0 / 2048, n0=0.71, chi0=5.0, sigma0=1.0,
                noise_amp=1.0, noise_dist=1, Dn=1.0, theta=1.0, bM=0.71, r0sq=6.25,
                seed=0)

GRID_KEYS = ("nx", "ny", "dx")
PARAM_KEYS = ("n0", "chi0", "sigma0", "noise_amp", "Dn", "theta", "bM", "r0sq", "dt",
              "cfl_frac", "b_threshold", "chemo_law", "mobility", "noise_dist", "noise_mode",
              "scheme", "precision")


def split(cfg: dict):
    """(grid dict, params dict, seed) of a workload dict."""
    grid = {k: cfg[k] for k in GRID_KEYS}
    params = {k: cfg[k] for k in PARAM_KEYS if k in cfg}
    return grid, params, int(cfg.get("seed", 0))


def perturbed_fields(nx: int, ny: int, seed: int, b_level=0.3, n_level=0.6, amp=0.2):
    """Seeded positive random fields (b, n) with a smooth and a rough part,
    for parity cases away from the Gaussian inoculum."""
    rng = np.random.default_rng(seed)
    y, x = np.mgrid[0:ny, 0:nx]
    kx, ky = rng.uniform(0.5, 3.0, 2)
    smooth = np.cos(2 * np.pi * kx * (x + 0.5) / max(nx, 1)) * np.cos(2 * np.pi * ky * (y + 0.5) / max(ny, 1))
    b = b_level * (1 + amp * smooth + 0.5 * amp * rng.uniform(-1, 1, (ny, nx)))
    n = n_level * (1 - amp * smooth + 0.5 * amp * rng.uniform(-1, 1, (ny, nx)))
    return b.astype(np.float64), n.astype(np.float64)


SWEEP_SIDES = (512, 1024, 1536, 2048)


def sweep_specs(count: int = 512, seed: int = 0, precision: int = 1, steps: int = 20000):
    """Batched sweep: `count` instances with sides drawn uniformly from
    512..2048, (n0, chi0, sigma0) from sweep_points, instance seeds
    0..count-1, static uniform noise a = 0.5, inoculum bM = 0.71 with
    r0^2 = 32^2, FP32 state, dt = 0.2 x limit."""
    rng = np.random.default_rng(seed + 1)
    sides = rng.choice(SWEEP_SIDES, size=count)
    n0, chi0, sigma0 = sweep_points(count, seed)
    return [dict(nx=int(s), ny=int(s), dx=1.0, seed=i, n0=float(n0[i]), chi0=float(chi0[i]),
                 sigma0=float(sigma0[i]), noise_amp=0.5, bM=0.71, r0sq=32.0 ** 2,
                 precision=precision) for i, s in enumerate(sides)]


def sweep_points(count: int, seed: int):
    """(n0, chi0, sigma0) on the log-spaced sweep box n0 in [0.1, 1.5],
    chi0 in {0} u [0.05, 4], sigma0 in [1, 8], drawn with a seeded generator."""
    rng = np.random.default_rng(seed)
    n0 = np.exp(rng.uniform(np.log(0.1), np.log(1.5), count))
    chi0 = np.exp(rng.uniform(np.log(0.05), np.log(4.0), count))
    chi0[rng.uniform(size=count) < 0.1] = 0.0
    sigma0 = np.exp(rng.uniform(np.log(1.0), np.log(8.0), count))
    return n0, chi0, sigma0
