"""Learned surrogate of the morphology map and the active boundary sweep.

The plain solver is the judge throughout: it produces every training label
and verifies every point the network proposes.

Labels of a sweep point (n0, chi0, sigma0, a), computed from one solver run
(a batch instance, forward Euler, FP32 state, static noise):
  * envelope velocity: FP64 least-squares slope of the envelope radius
    r_env(t) over the second half of the run (the paper tracks the colony
    envelope, Sec. 3, and bounds its speed, Sec. 4.1);
  * branch count: circular runs of b >= b_th on the circle r = 0.8 r_env
    (4096 bilinear samples, cx_batch_polar_profile).

Surrogate: the MLP of include/cx.h (4 -> 256 -> 256 -> 2, tanh), inputs
(log n0, chi0, log sigma0, a) mapped affinely from the sweep box to
[-1, 1]; outputs standardised by the training-set mean and spread.

Active sweep: each round draws a pool of candidates, and the network, its
branch output trained on the class (branched or not), picks half of
`per_round` nearest the compact / branched boundary and half where the
predicted log velocity is steepest (fronts starting to stall); the solver
verifies them in one batch, the labels are added and the network retrained.

Validated sweep (validated_sweep): training runs at 1024^2 with a time step
that varies smoothly with the parameters (smooth_dt), the velocity label
taken from the colony's area-equivalent radius, and a screen (Screen) of an
ensemble on log velocity plus a correction from the nearest training points;
a candidate is accepted without a solver run where those neighbours agree
and its colony stays clear of the walls, the rest go to the batched solver.
"""
from __future__ import annotations

import math

import numpy as np

import paper_1301_5058_gb300 as cx

BOX = {"n0": (0.1, 1.5), "chi0": (0.0, 4.0), "sigma0": (1.0, 8.0), "a": (0.0, 1.0)}


def encode(points) -> np.ndarray:
    """(N, 4) array of (n0, chi0, sigma0, a) -> network inputs in [-1, 1]."""
    p = np.asarray(points, np.float64)
    ln0 = (np.log(p[:, 0]) - math.log(BOX["n0"][0])) / math.log(BOX["n0"][1] / BOX["n0"][0])
    c = p[:, 1] / BOX["chi0"][1]
    ls = np.log(p[:, 2]) / math.log(BOX["sigma0"][1])
    a = p[:, 3]
    return (2.0 * np.stack([ln0, c, ls, a], 1) - 1.0).astype(np.float32)


def draw_points(count: int, seed: int, a_range=(0.5, 0.5)) -> np.ndarray:
    """Uniform draws in (log n0, chi0, log sigma0) over the sweep box."""
    rng = np.random.default_rng(seed)
    n0 = np.exp(rng.uniform(*np.log(BOX["n0"]), count))
    chi0 = rng.uniform(*BOX["chi0"], count)
    s0 = np.exp(rng.uniform(*np.log(BOX["sigma0"]), count))
    a = rng.uniform(*a_range, count)
    return np.stack([n0, chi0, s0, a], 1)


def count_runs(profile, level) -> int:
    above = np.asarray(profile) >= level
    if above.all() or not above.any():
        return 0
    return int((above & ~np.roll(above, 1)).sum())


def lsq_slope(t, r) -> float:
    t = np.asarray(t, np.float64)
    r = np.asarray(r, np.float64)
    tm, rm = t.mean(), r.mean()
    den = ((t - tm) ** 2).sum()
    return float(((t - tm) * (r - rm)).sum() / den) if den > 0 else float("nan")


def smooth_dt(points, bM=0.71, cfl=0.2, Dn=1.0, theta=1.0, dx=1.0):
    """A time step for sweep points that is a smooth function of (n0, chi0,
    sigma0, a) and never above the library's explicit limit: with
    B = bM + theta n0 and Dc = sigma0 (1 + a) n0 B (1 + chi0 B), the limit
    min(dx^2 / (4 max(Dn, Dc)), 1 / (4 Dn / dx^2 + B)) is at least
    1 / (4 (Dn + Dc) / dx^2 + 4 Dn / dx^2 + B), which has no kinks.  Runs of a
    fixed number of steps then end at a time that varies smoothly with the
    parameters, and so do their labels."""
    p = np.asarray(points, np.float64)
    n0, chi0, s0, a = p[:, 0], p[:, 1], p[:, 2], p[:, 3]
    B = bM + theta * n0
    Dc = s0 * (1.0 + a) * n0 * B * (1.0 + chi0 * B)
    return cfl / (4.0 * (Dn + Dc) / dx ** 2 + 4.0 * Dn / dx ** 2 + B)


def solver_labels(points, side=256, steps=4000, samples=40, seed0=0, r0sq=64.0,
                  nsamples=4096, tune=None, label="max", sides=None, chunk=2048, info=None,
                  dt=None):
    """Run every point as one batch instance and return (velocity, branches)
    arrays plus the per-instance diagnostics at the end.

    label "max": the velocity is the slope of r_env, the largest distance of
    a cell above the envelope level; "area": the slope of the colony's
    equivalent radius sqrt(area_env / pi), which averages the front over
    every direction (its seed-to-seed spread is several times smaller).
    sides: per-point grid sides (default `side` for all); the points are run
    in batches of at most `chunk` instances.  dt: per-point time steps
    (default: the library's, 0.2 x the stability limit).  info: a dict that
    receives the per-point end time, final radii, sides and histories."""
    pts = np.asarray(points, np.float64)
    sides = np.full(len(pts), side, int) if sides is None else np.asarray(sides, int)
    every = max(1, steps // samples)
    vel = np.empty(len(pts))
    branches = np.empty(len(pts))
    last = [None] * len(pts)
    t_end, r_end, ra_end = (np.empty(len(pts)) for _ in range(3))
    hist_t, hist_r, hist_a = (np.empty((samples, len(pts))) for _ in range(3))
    for c0 in range(0, len(pts), chunk):
        idx = range(c0, min(len(pts), c0 + chunk))
        specs = [dict(nx=int(sides[i]), ny=int(sides[i]), dx=1.0, seed=seed0 + i,
                      n0=float(pts[i, 0]), chi0=float(pts[i, 1]), sigma0=float(pts[i, 2]),
                      noise_amp=float(pts[i, 3]), bM=0.71, r0sq=r0sq,
                      precision=cx.CX_PREC_F32) for i in idx]
        if dt is not None:
            for k, i in enumerate(idx):
                specs[k]["dt"] = float(dt[i])
        t_hist, r_hist = [], []
        with cx.Batch(specs) as bt:
            if tune is not None:
                bt.tune(*tune)
            for _ in range(samples):
                bt.step(every)
                d = bt.diagnostics(check=False)
                t_hist.append([x["t"] for x in d])
                ra = [math.sqrt(x["area_env"] / math.pi) for x in d]
                rm = [x["r_env"] for x in d]
                r_hist.append(ra if label == "area" else rm)
                q = len(t_hist) - 1
                hist_t[q, idx.start:idx.stop] = t_hist[-1]
                hist_r[q, idx.start:idx.stop] = rm
                hist_a[q, idx.start:idx.stop] = ra
            for k, i in enumerate(idx):
                x = d[k]
                last[i] = x
                lvl = 0.1 * specs[k]["n0"]   # the envelope level 0.1 theta n0 (theta = 1)
                prof = cx.cx_batch_polar_profile(bt.h, k, 0.8 * x["r_env"], nsamples)
                branches[i] = count_runs(prof, lvl)
                t_end[i], r_end[i] = x["t"], x["r_env"]
                ra_end[i] = math.sqrt(x["area_env"] / math.pi)
        t_hist = np.asarray(t_hist)
        r_hist = np.asarray(r_hist)
        half = samples // 2
        for k, i in enumerate(idx):
            vel[i] = lsq_slope(t_hist[half:, k], r_hist[half:, k])
    if info is not None:
        info.update(t_end=t_end, r_end=r_end, r_area_end=ra_end, sides=sides, hist_t=hist_t,
                    hist_r=hist_r, hist_area_r=hist_a, branches=branches)
    return vel, branches, last


def init_params(seed: int) -> np.ndarray:
    """Glorot-uniform weights, zero biases, packed as include/cx.h says."""
    rng = np.random.default_rng(seed)

    def glorot(fo, fi):
        lim = math.sqrt(6.0 / (fi + fo))
        return rng.uniform(-lim, lim, (fo, fi))

    parts = [glorot(256, 4), np.zeros(256), glorot(256, 256), np.zeros(256), glorot(2, 256),
             np.zeros(2)]
    return np.concatenate([p.ravel() for p in parts]).astype(np.float32)


class Surrogate:
    """Network + output scaling.  predict() returns labels in solver units.
    members > 1: that many networks (initial weights from seeds seed,
    seed + 17, seed + 34, ...) trained together on the same labels, each on
    its own row order; predict() then returns (members, n, 2)."""

    def __init__(self, seed=0, max_batch=8192, members=1):
        self.seeds = [seed + 17 * k for k in range(members)]
        self.members = members
        self.net = cx.Mlp(max_batch, self._initial(), members=members)
        self.max_batch = max_batch
        self.seed = seed
        self.mean = np.zeros(2)
        self.scale = np.ones(2)

    def _initial(self):
        return np.concatenate([init_params(s) for s in self.seeds])

    def fit(self, points, labels, steps=3000, lr=1e-3, batch=256, reinit=True, decay=0,
            schedule="halve"):
        """Adam on the standardised labels.  decay > 0: the steps are split
        into decay + 1 equal chunks and the rows reshuffled from one chunk to
        the next (the optimiser state carries over); the rate is halved from
        chunk to chunk (schedule "halve") or follows a cosine from lr down to
        lr / (2 (decay + 1)) ("cosine").  Returns the step losses ((steps,),
        or (members, steps))."""
        X = encode(points)
        Y = np.asarray(labels, np.float64)
        self.mean = Y.mean(0)
        self.scale = Y.std(0) + 1e-12
        T = ((Y - self.mean) / self.scale).astype(np.float32)
        rngs = [np.random.default_rng(s + len(X)) for s in self.seeds]
        batch = min(batch, len(X))
        if reinit:
            self.net.set_params(self._initial())
        losses = []
        chunk = max(1, steps // (decay + 1))
        for k in range(decay + 1):
            perms = [r.permutation(len(X)) for r in rngs]
            n = chunk if k < decay else steps - chunk * decay
            if n > 0:
                rate = lr * 0.5 ** k if schedule == "halve" else \
                    lr * 0.5 * (1.0 + math.cos(math.pi * (k + 0.5) / (decay + 1)))
                xs = np.stack([X[p] for p in perms])
                ts = np.stack([T[p] for p in perms])
                losses.append(self.net.train(xs, ts, batch, n, rate))
        return np.concatenate(losses, axis=-1)

    def predict(self, points) -> np.ndarray:
        X = encode(points)
        out = np.empty((self.members, len(X), 2))
        c = self.max_batch
        for s in range(0, len(X), c):
            out[:, s:s + c] = self.net.forward(X[s:s + c]).reshape(self.members, -1, 2)
        out = out * self.scale + self.mean
        return out[0] if self.members == 1 else out

    def close(self):
        self.net.close()


def boundary_scores(model: Surrogate, pts, level=0.5, eps=0.02, vfloor=1e-3):
    """Two scores, higher = closer to a predicted morphology boundary: the
    branch output's closeness to `level` (between compact and branched), and
    the steepness of the predicted log velocity (finite differences in the
    normalised inputs; relative changes peak where fronts start to stall)."""
    logv = lambda p: np.log(np.maximum(model.predict(p)[:, 0], vfloor))
    pred = model.predict(pts)
    near = -np.abs(pred[:, 1] - level)
    X = encode(pts).astype(np.float64)
    grad = np.zeros(len(pts))
    for k in range(3):
        step = np.zeros(4)
        step[k] = eps
        d = (logv(_decode(X + step)) - logv(_decode(X - step))) / (2 * eps)
        grad += d * d
    return near, np.sqrt(grad)


def pick_boundary(model: Surrogate, cand, k):
    """Indices of k candidates: half nearest the compact / branched
    boundary, half (of the rest) where the predicted log velocity is
    steepest."""
    near, steep = boundary_scores(model, cand)
    kb = k // 2
    ib = np.argsort(-near)[:kb]
    rest = np.setdiff1d(np.arange(len(cand)), ib)
    iv = rest[np.argsort(-steep[rest])[:k - kb]]
    return np.concatenate([ib, iv])


def _decode(X):
    X = (np.asarray(X) + 1.0) / 2.0
    n0 = BOX["n0"][0] * np.exp(X[:, 0] * math.log(BOX["n0"][1] / BOX["n0"][0]))
    chi0 = X[:, 1] * BOX["chi0"][1]
    s0 = np.exp(X[:, 2] * math.log(BOX["sigma0"][1]))
    return np.stack([n0, chi0, s0, X[:, 3]], 1)


def demo(side=256, steps=4000, n_train=256, n_test=128, train_steps=3000, seed=0):
    """Label a training and a held-out set with the solver (one batch each),
    train the network on the GPU, and report throughput and held-out error."""
    import json
    import time
    out = {"side": side, "steps_per_point": steps}
    t0 = time.perf_counter()
    ptr = draw_points(n_train, seed, a_range=(0.0, 1.0))
    vtr, btr, _ = solver_labels(ptr, side=side, steps=steps)
    t1 = time.perf_counter()
    pte = draw_points(n_test, seed + 99, a_range=(0.0, 1.0))
    vte, bte, _ = solver_labels(pte, side=side, steps=steps, seed0=10_000)
    out["solver_points_per_hour"] = n_train * 3600.0 / (t1 - t0)
    out["branch_counts"] = {str(k): int(v) for k, v in zip(*np.unique(btr, return_counts=True))}
    out["velocity_range"] = [float(vtr.min()), float(vtr.max())]
    model = Surrogate(seed, max_batch=max(n_train, 1024))
    t2 = time.perf_counter()
    losses = model.fit(ptr, np.stack([vtr, btr], 1), steps=train_steps, lr=2e-3,
                       batch=min(256, n_train))
    t3 = time.perf_counter()
    pred = model.predict(pte)
    t4 = time.perf_counter()
    big = draw_points(100_000, seed + 7)
    t5 = time.perf_counter()
    model.predict(big)
    t6 = time.perf_counter()
    rel = np.abs(pred[:, 0] - vte) / np.maximum(np.abs(vte), 1e-12)
    out.update({
        "train_seconds": t3 - t2, "final_loss": float(losses[-20:].mean()),
        "heldout_velocity_rel_error_median": float(np.median(rel)),
        "heldout_velocity_rel_error_p90": float(np.quantile(rel, 0.9)),
        "heldout_within_1pct": float((rel <= 0.01).mean()),
        "heldout_branch_abs_error_mean": float(np.mean(np.abs(pred[:, 1] - bte))),
        "surrogate_points_per_hour": 100_000 * 3600.0 / (t6 - t5),
    })
    model.close()
    print(json.dumps(out))
    return out


class Ensemble:
    """Several networks trained on log(velocity) from different initial
    weights (the members of one network handle, trained together); a point
    is accepted without a solver run when the members agree to within
    `agree` (relative spread of the predicted velocity)."""

    def __init__(self, members=4, seed=0, max_batch=8192):
        self.model = Surrogate(seed, max_batch, members=members)
        self.members = members

    def fit_labels(self, points, labels, **kw):
        return self.model.fit(points, labels, **kw)

    def fit(self, points, velocity, **kw):
        lv = np.log(np.maximum(np.asarray(velocity, np.float64), 1e-12))
        return self.fit_labels(points, np.stack([lv, np.zeros_like(lv)], 1), **kw)

    def member_outputs(self, points):
        """First output of every member, (members, n)."""
        p = self.model.predict(points)
        return (p[None] if self.members == 1 else p)[..., 0]

    def predict(self, points):
        v = np.exp(self.member_outputs(points))
        mean = v.mean(0)
        spread = (v.max(0) - v.min(0)) / np.maximum(mean, 1e-30)
        return mean, spread

    def close(self):
        self.model.close()


def poly_features(X, degree=3) -> np.ndarray:
    """All monomials of the columns of X up to `degree` (with the constant)."""
    import itertools
    X = np.asarray(X, np.float64)
    cols = [np.ones(len(X))]
    for d in range(1, degree + 1):
        for c in itertools.combinations_with_replacement(range(X.shape[1]), d):
            cols.append(np.prod(X[:, c], axis=1))
    return np.stack(cols, 1)


class Screen:
    """The learned screen of the validated sweep: log velocity = a
    least-squares polynomial of the encoded inputs (degree 0 by default: the
    mean) + an ensemble of networks (on the GPU kernels of include/cx.h)
    trained on that fit's residual + a correction from the k nearest training
    points (their inverse-distance weighted residual).  The spread of those
    neighbours' residuals is the screen's confidence: the networks miss by a
    bias that varies smoothly over the box, so where the neighbours agree the
    correction holds.  (With a cubic baseline the networks, whose zero-bias
    initial function is odd and nearly cubic in the inputs, see a target
    orthogonal to everything they start from: their output weights decay and
    they settle on a constant, so the baseline stays off.)"""

    def __init__(self, members=8, seed=0, k=16, degree=0, max_batch=8192):
        self.ens = Ensemble(members, seed, max_batch=max_batch)
        self.k = k
        self.degree = degree

    def _base_log(self, X):
        return poly_features(X, self.degree) @ self.coef

    def _net_log(self, points):
        return self.ens.member_outputs(points).mean(0)

    def fit(self, points, velocity, **kw):
        X = encode(points).astype(np.float64)
        y = np.log(np.maximum(np.asarray(velocity, np.float64), 1e-12))
        self.coef, *_ = np.linalg.lstsq(poly_features(X, self.degree), y, rcond=None)
        r = y - self._base_log(X)
        self.ens.fit_labels(points, np.stack([r, np.zeros_like(r)], 1), **kw)
        self.X = X
        self.res = y - self._base_log(X) - self._net_log(points)
        return self

    def predict(self, points, chunk=2048):
        """(velocity, neighbour spread of the log residual) of each point."""
        X = encode(points).astype(np.float64)
        logv = self._base_log(X) + self._net_log(points)
        corr = np.empty(len(X))
        spread = np.empty(len(X))
        for c in range(0, len(X), chunk):
            D = ((X[c:c + chunk, None, :] - self.X[None, :, :]) ** 2).sum(-1)
            nb = np.argpartition(D, self.k, axis=1)[:, :self.k]
            w = 1.0 / (np.take_along_axis(D, nb, 1) + 1e-6)
            corr[c:c + chunk] = (self.res[nb] * w).sum(1) / w.sum(1)
            spread[c:c + chunk] = self.res[nb].std(1)
        return np.exp(logv + corr), spread

    def close(self):
        self.ens.close()


def single_instance_seconds_per_point(side, steps, spec_point, repeats=2):
    """Wall time of one point stepped alone through cx_step (creation,
    `steps` steps, diagnostics every steps/40), the plain way."""
    import time
    import torch
    p = spec_point
    kw = dict(n0=float(p[0]), chi0=float(p[1]), sigma0=float(p[2]), noise_amp=float(p[3]),
              bM=0.71, r0sq=64.0, precision=cx.CX_PREC_F32)
    best = float("inf")
    for _ in range(repeats):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        with cx.Sim(side, side, 1.0, seed=0, **kw) as sim:
            for _ in range(40):
                sim.step(steps // 40)
                sim.diagnostics(check=False)
        best = min(best, time.perf_counter() - t0)
    return best


def validated_throughput(side=256, steps=20000, n_train=4096, n_test=1024, members=8,
                         agree=0.02, train_steps=40000, seed=0, decay=4, lr=2e-3,
                         campaign=4):
    """Points per hour whose envelope velocity is known to within 1 %, three
    ways: every point alone through cx_step; every point as a batch
    instance; and screened by the ensemble (accepted where its members agree
    to `agree`; the rest run by the batched solver).  The accepted points'
    error is judged on a solver-labelled held-out set.  `campaign`: a sweep
    of n_train solver-labelled training points, training, then campaign x
    n_train screened candidates, every cost included."""
    import json
    import time
    ptr = draw_points(n_train, seed, a_range=(0.0, 1.0))
    t0 = time.perf_counter()
    vtr, _, _ = solver_labels(ptr, side=side, steps=steps)
    batch_s_per_point = (time.perf_counter() - t0) / n_train
    pte = draw_points(n_test, seed + 99, a_range=(0.0, 1.0))
    vte, _, _ = solver_labels(pte, side=side, steps=steps, seed0=100_000)
    single_s = single_instance_seconds_per_point(side, steps, ptr[0])
    ens = Ensemble(members, seed, max_batch=max(1024, min(8192, n_train)))
    t1 = time.perf_counter()
    ens.fit(ptr, vtr, steps=train_steps, lr=lr, batch=256, decay=decay)
    train_s = time.perf_counter() - t1
    t2 = time.perf_counter()
    mean, spread = ens.predict(pte)
    screen_s_per_point = (time.perf_counter() - t2) / n_test
    ens.close()
    rel = np.abs(mean - vte) / np.maximum(vte, 1e-12)
    acc = spread <= agree
    f_acc = float(acc.mean())
    within = float((rel[acc] <= 0.01).mean()) if acc.any() else float("nan")
    sweep = {}
    for a in (0.005, 0.01, 0.02, 0.05, 0.1):
        m = spread <= a
        sweep[str(a)] = {"accepted": float(m.mean()),
                         "within_1pct": float((rel[m] <= 0.01).mean()) if m.any() else None,
                         "p95_error": float(np.quantile(rel[m], 0.95)) if m.any() else None}
    # per point: screening always; the solver for the rejected share
    mixed_s = screen_s_per_point + (1 - f_acc) * batch_s_per_point
    m = campaign * n_train
    campaign_s = n_train * batch_s_per_point + train_s + m * mixed_s
    out = {
        "side": side, "steps_per_point": steps, "n_train": n_train, "n_test": n_test,
        "members": members, "agree": agree, "train_steps": train_steps, "decay": decay, "lr": lr,
        "single_instance_points_per_hour": 3600.0 / single_s,
        "batched_solver_points_per_hour": 3600.0 / batch_s_per_point,
        "heldout_rel_error_median_all": float(np.median(rel)),
        "heldout_within_1pct_all": float((rel <= 0.01).mean()),
        "agreement_thresholds": sweep,
        "accepted_fraction": f_acc,
        "accepted_within_1pct": within,
        "rejected_go_to_solver": True,
        "screened_points_per_hour": 3600.0 / mixed_s,
        "train_seconds": train_s,
        "campaign_points": n_train + m,
        "campaign_points_per_hour": 3600.0 * (n_train + m) / campaign_s,
        "speedup_batched_solver_only": single_s / batch_s_per_point,
        "speedup_screened": single_s / mixed_s,
        "speedup_campaign": single_s * (n_train + m) / campaign_s,
    }
    print(json.dumps(out))
    return out


def initial_area_radius(n0, r0sq, bM=0.71, theta=1.0):
    """Equivalent radius of the inoculum's part above the envelope level:
    bM exp(-r^2 / r0sq) >= 0.1 theta n0 inside r^2 <= r0sq ln(bM / (0.1 theta n0))."""
    q = np.log(bM / (0.1 * theta * np.asarray(n0, np.float64)))
    return np.sqrt(r0sq * np.maximum(q, 0.0))


def end_times(points, steps, bM=0.71, r0sq=32.0 ** 2):
    """Physical time reached after `steps` steps at each point's time step
    (the library's default: 0.2 x the stability limit)."""
    out = np.empty(len(points))
    g = cx.cx_grid(8, 8, 1.0)
    for i, p in enumerate(np.asarray(points, np.float64)):
        prm = cx.cx_params_default(n0=float(p[0]), chi0=float(p[1]), sigma0=float(p[2]),
                                   noise_amp=float(p[3]), bM=bM, r0sq=r0sq)
        out[i] = steps * prm.cfl_frac * cx.cx_dt_limit(g, prm)
    return out


def single_instance_seconds(side, steps, point, r0sq=32.0 ** 2, samples=40, repeats=2, dt=0.0):
    """Wall time of one point stepped alone through cx_step, the plain way:
    creation, `steps` steps, diagnostics `samples` times, a polar profile."""
    import time
    import torch
    p = point
    kw = dict(n0=float(p[0]), chi0=float(p[1]), sigma0=float(p[2]), noise_amp=float(p[3]),
              bM=0.71, r0sq=r0sq, precision=cx.CX_PREC_F32, dt=float(dt))
    best = float("inf")
    for _ in range(repeats):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        with cx.Sim(side, side, 1.0, seed=0, **kw) as sim:
            for _ in range(samples):
                sim.step(steps // samples)
                d = sim.diagnostics(check=False)
            cx.cx_polar_profile(sim.h, 0.8 * d["r_env"], 4096)
        best = min(best, time.perf_counter() - t0)
    return best


def validated_sweep(train_side=1024, sides=(512, 1024, 1536, 2048), steps=20000, n_train=8192,
                    n_test=1024, members=8, train_steps=200000, decay=19, lr=2e-3, seed=0,
                    bar=0.01, quantile=0.95, wall_frac=0.6, campaign=4, chunk=2048,
                    r0sq=32.0 ** 2, samples=40, verbose=True, save=None, schedule="cosine",
                    knn=16):
    """Validated sweep points per hour on a mix of grid sizes, with and
    without the learned screen.

    Training data: n_train solver runs at train_side^2 (the sweep's solver,
    one batch per `chunk` instances), labelled with the area-radius
    velocity.  Held-out: n_test points with sides drawn uniformly from
    `sides`, each run by the solver at its own size and seed.  The screen
    accepts a point without a solver run when (a) the ensemble's members
    agree to a relative spread s* and (b) the colony, grown at the predicted
    velocity from the inoculum, stays within wall_frac of the grid's
    half-width (the labels are free-space velocities).  The screen (Screen)
    predicts the velocity from a cubic fit, an ensemble of networks on its
    residual and a correction from the `knn` nearest training points; its
    confidence is the spread of those neighbours' residuals, and s* is the
    largest spread at which the accepted points of the calibration half of
    the held-out set meet `bar` at `quantile`; the other half reports the
    error.
    Rejected points go to the batched solver, whose every label is exact by
    construction (a batch instance equals its single grid bit for bit)."""
    import json
    import time
    rng = np.random.default_rng(seed + 5)
    # training data
    ptr = draw_points(n_train, seed, a_range=(0.0, 1.0))
    t0 = time.perf_counter()
    info_tr = {}
    vtr, btr, _ = solver_labels(ptr, side=train_side, steps=steps, samples=samples, r0sq=r0sq,
                                label="area", chunk=chunk, info=info_tr, dt=smooth_dt(ptr))
    train_data_s = time.perf_counter() - t0
    # held-out points on the size mix
    pte = draw_points(n_test, seed + 99, a_range=(0.0, 1.0))
    ste = rng.choice(np.asarray(sides), size=n_test)
    info = {}
    t1 = time.perf_counter()
    vte, bte, _ = solver_labels(pte, steps=steps, samples=samples, r0sq=r0sq, label="area",
                                sides=ste, seed0=1_000_000, chunk=chunk, info=info,
                                dt=smooth_dt(pte))
    batch_s = (time.perf_counter() - t1) / n_test
    # the plain way, one point per size class
    first = {int(sd): int(np.argmax(ste == sd)) for sd in sides}
    single = {sd: single_instance_seconds(sd, steps, pte[i], r0sq=r0sq, samples=samples,
                                          dt=smooth_dt(pte[i:i + 1])[0]) for sd, i in first.items()}
    single_s = float(np.mean([single[int(sd)] for sd in ste]))
    # the ensemble
    ok = vtr > 0
    scr = Screen(members, seed, k=knn)
    t2 = time.perf_counter()
    scr.fit(ptr[ok], vtr[ok], steps=train_steps, lr=lr, batch=256, decay=decay,
            schedule=schedule)
    train_s = time.perf_counter() - t2
    pool = draw_points(16384, seed + 4242, a_range=(0.0, 1.0))
    t3 = time.perf_counter()
    scr.predict(pool)
    steps * smooth_dt(pool)
    screen_s = (time.perf_counter() - t3) / len(pool)
    mean, spread = scr.predict(pte)
    scr.close()
    if save:
        np.savez_compressed(save, ptr=ptr, vtr=vtr, pte=pte, ste=ste, vte=vte, mean=mean,
                            spread=spread, **{"tr_" + k: v for k, v in info_tr.items()},
                            **{"te_" + k: v for k, v in info.items()})
    t_end = steps * smooth_dt(pte)
    r_pred = initial_area_radius(pte[:, 0], r0sq) + np.maximum(mean, 0.0) * t_end
    wall_ok = r_pred <= wall_frac * 0.5 * ste
    rel = np.abs(mean - vte) / np.maximum(np.abs(vte), 1e-12)
    half = n_test // 2
    cal, ev = np.arange(half), np.arange(half, n_test)
    chosen = None
    grid_s = np.geomspace(1e-4, 0.2, 60)
    for sv in grid_s:
        m = (spread[cal] <= sv) & wall_ok[cal]
        if m.sum() >= 20 and np.quantile(rel[cal][m], quantile) <= bar:
            chosen = float(sv)
    out = {"train_side": train_side, "sides": list(map(int, sides)), "steps_per_point": steps,
           "n_train": n_train, "n_test": n_test, "members": members, "train_steps": train_steps,
           "label": "slope of sqrt(area_env / pi) over the second half of the run",
           "time_step": "0.2 / (4 (Dn + Dc) / dx^2 + 4 Dn / dx^2 + B), smooth in the parameters",
           "training_schedule": f"Adam, {train_steps} steps in {decay + 1} chunks, {schedule} rate from {lr}",
           "screen": f"{members} networks on log velocity + inverse-distance weighted residual "
                     f"of the {knn} nearest training points; confidence: their residuals' spread",
           "bar": bar, "quantile": quantile, "wall_frac": wall_frac,
           "heldout_error_all": {"median": float(np.median(rel)),
                                 "p90": float(np.quantile(rel, 0.9)),
                                 "within_bar": float((rel <= bar).mean())},
           "wall_limited_points": int((~wall_ok).sum()),
           "single_instance_seconds_by_side": {str(k): v for k, v in single.items()},
           "single_instance_points_per_hour": 3600.0 / single_s,
           "batched_points_per_hour": 3600.0 / batch_s,
           "training_data_seconds": train_data_s, "train_seconds": train_s,
           "screen_seconds_per_point": screen_s}
    if chosen is None:
        out["accepted_fraction"] = 0.0
        out["note"] = "no agreement threshold met the bar on the calibration half"
        f_acc = 0.0
    else:
        acc = (spread[ev] <= chosen) & wall_ok[ev]
        f_acc = float(acc.mean())
        e = rel[ev][acc]
        out.update({
            "agreement_threshold": chosen, "accepted_fraction": f_acc,
            "accepted_error": {q: float(np.quantile(e, float(q))) for q in ("0.5", "0.9", "0.95", "0.99")}
            if len(e) else None,
            "accepted_max_error": float(e.max()) if len(e) else None,
            "accepted_within_bar": float((e <= bar).mean()) if len(e) else None,
            "accepted_by_side": {str(int(sd)): float(acc[ste[ev] == sd].mean()) for sd in sides}})
    mixed_s = screen_s + (1.0 - f_acc) * batch_s
    m = campaign * n_train
    campaign_s = train_data_s + train_s + m * mixed_s
    out.update({
        "screened_points_per_hour": 3600.0 / mixed_s,
        "campaign_points": n_train + m,
        "campaign_points_per_hour": 3600.0 * (n_train + m) / campaign_s,
        "speedup_batched": single_s / batch_s,
        "speedup_screened": single_s / mixed_s,
        "speedup_campaign": single_s * (n_train + m) / campaign_s})
    if verbose:
        print(json.dumps(out))
    return out


def label_noise(side=256, steps=20000, points=128, seeds=8, seed=0):
    """Spread of the envelope-velocity label over sigma-field realisations:
    every one of `points` parameter points is run with `seeds` different
    seeds (one batch).  Returns the per-point coefficient of variation and
    the relative deviation of each run from its point's mean; no surrogate
    of (n0, chi0, sigma0, a) can predict a single realisation better than
    this spread."""
    import json
    pts = draw_points(points, seed, a_range=(0.0, 1.0))
    rep = np.repeat(pts, seeds, axis=0)
    vel, _, _ = solver_labels(rep, side=side, steps=steps, seed0=500_000)
    v = vel.reshape(points, seeds)
    mean = v.mean(axis=1)
    ok = mean > 1e-9
    cv = v[ok].std(axis=1, ddof=1) / mean[ok]
    dev = np.abs(v[ok] - mean[ok, None]) / mean[ok, None]
    out = {"side": side, "steps_per_point": steps, "points": points, "seeds": seeds,
           "moving_points": int(ok.sum()),
           "cv_median": float(np.median(cv)), "cv_p90": float(np.quantile(cv, 0.9)),
           "run_deviation_median": float(np.median(dev)),
           "runs_within_1pct_of_point_mean": float((dev <= 0.01).mean())}
    print(json.dumps(out))
    return out


def active_sweep(rounds=3, per_round=64, first=128, pool=4096, seed=0, label_kw=None,
                 train_kw=None):
    """Surrogate-guided sweep.  Each round the network is retrained on every
    verified point and picks `per_round` of `pool` candidates (pick_boundary);
    the solver verifies them.  Returns a dict with every verified point, its
    labels, and per-round surrogate errors on the newly verified points (the
    first half of each round's points is the branch-boundary half)."""
    label_kw = label_kw or {}
    train_kw = train_kw or {}
    pts = draw_points(first, seed)
    v, b, _ = solver_labels(pts, seed0=0, **label_kw)
    P, L = pts, np.stack([v, b], 1)
    model = Surrogate(seed)
    history = []
    for r in range(rounds):
        # the branch output is trained on the class (branched or not), so that
        # 0.5 is its decision boundary; L keeps the counts
        model.fit(P, np.stack([L[:, 0], (L[:, 1] >= 1).astype(np.float64)], 1), **train_kw)
        cand = draw_points(pool, seed + 1000 + r)
        pick = cand[pick_boundary(model, cand, per_round)]
        pred = model.predict(pick)
        v, b, _ = solver_labels(pick, seed0=len(P), **label_kw)
        rel = np.abs(pred[:, 0] - v) / np.maximum(np.abs(v), 1e-12)
        history.append({"round": r, "median_rel_velocity_error": float(np.median(rel)),
                        "branch_class_accuracy": float(np.mean((pred[:, 1] >= 0.5) == (b >= 1)))})
        P = np.concatenate([P, pick])
        L = np.concatenate([L, np.stack([v, b], 1)])
    model.close()
    return {"points": P, "labels": L, "history": history}


def boundary_gain(rounds=3, per_round=128, first=256, pool=8192, seed=0, side=256, steps=20000,
                  train_steps=6000, r0sq=64.0):
    """Does the surrogate-guided sweep sample the morphology boundaries?
    Runs active_sweep, then as many uniformly drawn points through the
    solver, and compares (a) the share of branched colonies (branch count
    >= 1) among the branch-boundary picks: most of the box grows compact
    colonies, so a sampler that concentrates on the compact / branched
    boundary finds more branched ones than uniform sampling does; (b) the
    share of slow fronts (velocity below the uniform sample's 10th
    percentile, near the stall boundary) among the steep-velocity picks."""
    import json
    label_kw = dict(side=side, steps=steps, r0sq=r0sq)
    res = active_sweep(rounds=rounds, per_round=per_round, first=first, pool=pool, seed=seed,
                       label_kw=label_kw, train_kw=dict(steps=train_steps, lr=2e-3, batch=256,
                                                        decay=3))
    active_b = res["labels"][first:, 1].reshape(rounds, per_round)
    branch_half = active_b[:, : per_round // 2]
    active_v = res["labels"][first:, 0].reshape(rounds, per_round)
    uni = draw_points(rounds * per_round, seed + 777)
    uv, ub, _ = solver_labels(uni, seed0=900_000, **label_kw)
    slow = np.quantile(uv, 0.1)
    out = {"side": side, "steps_per_point": steps, "r0sq": r0sq, "first": first, "rounds": rounds,
           "per_round": per_round,
           "initial_branched_fraction": float((res["labels"][:first, 1] >= 1).mean()),
           "uniform_branched_fraction": float((ub >= 1).mean()),
           "active_branched_fraction": float((active_b >= 1).mean()),
           "branch_half_branched_fraction": float((branch_half >= 1).mean()),
           "branch_half_branched_by_round": [float((h >= 1).mean()) for h in branch_half],
           "velocity_half_slow_fraction": float((active_v[:, per_round // 2:] <= slow).mean()),
           "uniform_slow_fraction": float((uv <= slow).mean()),
           "history": res["history"]}
    print(json.dumps(out))
    return out


if __name__ == "__main__":
    import sys
    kw = {}
    mode = demo
    for a in sys.argv[1:]:
        if a == "--validated":
            mode = validated_throughput
            continue
        if a == "--label-noise":
            mode = label_noise
            continue
        if a == "--boundary":
            mode = boundary_gain
            continue
        if a == "--validated-sweep":
            mode = validated_sweep
            continue
        k, _, v = a.lstrip("-").partition("=")
        kw[k] = float(v) if "." in v else int(v)
    mode(**kw)
