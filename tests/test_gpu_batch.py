"""Batched sweeps (cx_batch_*): every instance must evolve bit for bit as a
single-grid handle with the same grid, parameters and seed, whatever the
tuning (tile height, graph chunk, L2 groups); the batch diagnostics agree with
the single-grid ones to round-off; one instance is also checked against the
oracle directly."""
import numpy as np
import pytest

import oracle
from paper_1301_5058_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cx():
    from paper_1301_5058_gb300 import _build
    _build.build()
    import paper_1301_5058_gb300 as cx
    return cx


SIZES = [(64, 48), (130, 70), (513, 33), (7, 5), (600, 97), (1, 1)]


def specs(prec, scheme=0, sizes=SIZES, noise=None):
    """Instances of a sweep; noise=(mode, dist) sets the sigma noise (default
    static uniform)."""
    n0, chi0, sigma0 = W.sweep_points(len(sizes), seed=4)
    out = []
    for i, (nx, ny) in enumerate(sizes):
        out.append(dict(nx=nx, ny=ny, dx=1.0, seed=100 + i, n0=float(n0[i]), chi0=float(chi0[i]),
                        sigma0=float(sigma0[i]), noise_amp=0.5, bM=0.71, r0sq=16.0,
                        precision=prec, scheme=scheme))
        if noise is not None:
            out[-1].update(noise_mode=noise[0], noise_dist=noise[1])
    return out


def single_runs(cx, sp, steps, dtype):
    out = []
    for s in sp:
        kw = {k: v for k, v in s.items() if k not in ("nx", "ny", "dx", "seed")}
        with cx.Sim(s["nx"], s["ny"], s["dx"], seed=s["seed"], **kw) as sim:
            sim.step(steps)
            out.append((sim.field(cx.CX_FIELD_B, dtype), sim.field(cx.CX_FIELD_N, dtype),
                        sim.diagnostics()))
    return out


@pytest.mark.parametrize("prec,scheme", [(1, 0), (0, 0), (1, 1)])
@pytest.mark.parametrize("tuning", [(32, 0, 0, 0), (8, 10, 0, 0), (64, 64, 0, 0),
                                    (16, 12, 400_000, 0), (8, 0, 400_000, 7), (4, 0, 0, 50),
                                    (32, 0, 0, 1), (32, 0, 0, 0, 1), (8, 10, 0, 0, 1),
                                    (64, 64, 0, 0, 2), (16, 12, 400_000, 0, 2), (5, 6, 0, 0, 2),
                                    (3, 0, 0, 0, 2)])
def test_batch_matches_single_grids_bitwise(cx, prec, scheme, tuning):
    sp = specs(prec, scheme)
    dtype = np.float32 if prec == 1 else np.float64
    steps = 131   # odd: exercises the parity handling around graph chunks
    ref = single_runs(cx, sp, steps, dtype)
    with cx.Batch(sp) as bt:
        bt.tune(*tuning)
        bt.step(60)
        bt.step(steps - 60)
        diags = bt.diagnostics()
        for i in range(len(sp)):
            assert np.array_equal(bt.field(i, cx.CX_FIELD_B, dtype), ref[i][0]), i
            assert np.array_equal(bt.field(i, cx.CX_FIELD_N, dtype), ref[i][1]), i
    for d, (_, _, r) in zip(diags, ref):
        for k in ("mass_b", "mass_n", "invariant"):
            assert d[k] == pytest.approx(r[k], rel=1e-13)
        for k in ("min_b", "min_n", "max_b", "r_env", "area_env", "step", "t", "dt", "finite"):
            assert d[k] == r[k], k


# The paper's own scheme in a sweep (Sec. 3): sigma redrawn at every point and
# step from a triangular law, with forward Euler or Heun.  Each instance draws
# from (its seed, cell, step) exactly as a single grid does, so it must match
# that grid bit for bit under every tuning, across two calls (the step index
# carries over) and through graph replays (the step is read on the device).
@pytest.mark.parametrize("prec,scheme", [(1, 0), (1, 1), (0, 0), (0, 1)])
@pytest.mark.parametrize("tuning", [(32, 0, 0, 0), (8, 10, 0, 0), (16, 12, 400_000, 0),
                                    (4, 0, 0, 50), (32, 0, 0, 0, 1), (8, 10, 0, 0, 1),
                                    (64, 64, 0, 0, 2), (5, 6, 0, 0, 2)])
def test_batch_per_step_noise_matches_single_grids_bitwise(cx, prec, scheme, tuning):
    sp = specs(prec, scheme, noise=(1, 1))
    dtype = np.float32 if prec == 1 else np.float64
    steps = 131
    ref = single_runs(cx, sp, steps, dtype)
    with cx.Batch(sp) as bt:
        bt.tune(*tuning)
        bt.step(60)
        bt.step(steps - 60)
        for i in range(len(sp)):
            assert np.array_equal(bt.field(i, cx.CX_FIELD_B, dtype), ref[i][0]), i
            assert np.array_equal(bt.field(i, cx.CX_FIELD_N, dtype), ref[i][1]), i


@pytest.mark.parametrize("prec,scheme,tol", [(1, 1, 1e-4), (0, 1, 1e-12), (1, 0, 1e-4)])
def test_batch_per_step_noise_instance_matches_oracle(cx, prec, scheme, tol):
    # the oracle redraws sigma before every step by the recipe of the state's
    # precision (FP32 state: the four-cells-per-block FP32 recipe)
    sp = specs(prec, scheme, sizes=[(90, 70), (33, 40)], noise=(1, 1))
    steps = 300
    with cx.Batch(sp) as bt:
        s = sp[0]
        b, n = oracle.initial_state(90, 70, 1.0, s["n0"], s["bM"], s["r0sq"])
        bt.set_field(0, cx.CX_FIELD_B, b)
        bt.set_field(0, cx.CX_FIELD_N, n)
        bt.step(steps)
        gb = bt.field(0, cx.CX_FIELD_B)
        gn = bt.field(0, cx.CX_FIELD_N)
        dt = bt.diagnostics()[0]["dt"]
    ob, on, _ = oracle.run(np.zeros((70, 90)), b, n, steps, dx=1.0, dt=dt, Dn=1.0, theta=1.0,
                           chi0=s["chi0"], scheme=scheme, noise_mode=1, seed=s["seed"],
                           sigma0=s["sigma0"], amp=s["noise_amp"], dist=1,
                           recipe=1 if prec == 1 else 0)
    assert np.linalg.norm(gb - ob) <= tol * np.linalg.norm(ob)
    assert np.linalg.norm(gn - on) <= tol * np.linalg.norm(on)


def test_batch_instance_matches_oracle(cx):
    sp = specs(0, 0, sizes=[(90, 70), (33, 40)])
    with cx.Batch(sp) as bt:
        bt.step(300)
        gb = bt.field(0, cx.CX_FIELD_B)
        gn = bt.field(0, cx.CX_FIELD_N)
        dt = bt.diagnostics()[0]["dt"]
    s = sp[0]
    sig = oracle.sigma_field(90, 70, s["seed"], s["sigma0"], s["noise_amp"])
    b, n = oracle.initial_state(90, 70, 1.0, s["n0"], s["bM"], s["r0sq"])
    ob, on, _ = oracle.run(sig, b, n, 300, dx=1.0, dt=dt, Dn=1.0, theta=1.0, chi0=s["chi0"])
    assert np.linalg.norm(gb - ob) <= 1e-12 * np.linalg.norm(ob)
    assert np.linalg.norm(gn - on) <= 1e-12 * np.linalg.norm(on)


def test_batch_field_io_and_errors(cx):
    sp = specs(1, 0, sizes=[(20, 10), (31, 17)])
    with cx.Batch(sp) as bt:
        x = np.linspace(0.1, 0.9, 31 * 17).reshape(17, 31)
        bt.set_field(1, cx.CX_FIELD_B, x)
        assert np.array_equal(bt.field(1, cx.CX_FIELD_B, np.float32), x.astype(np.float32))
        with pytest.raises(cx.CxError):
            cx.cx_batch_get_field(bt.h, 2, cx.CX_FIELD_B, np.empty((17, 31)))
        with pytest.raises(cx.CxError):
            cx.cx_batch_get_field(bt.h, 0, cx.CX_FIELD_B, np.empty(5))
        with pytest.raises(cx.CxError):
            bt.tune(0, 1, 0)
        with pytest.raises(cx.CxError):
            bt.tune(8, 0, 0, -1)
        assert cx.cx_batch_get_time(bt.h) == (2, 0)


def test_resident_barrier_timeout_is_reported(cx, monkeypatch):
    # failure detection without a GPU fault: a spin limit of 0 makes every
    # grid-barrier wait give up at once; the kernel returns, the context
    # stays usable, and the host reports CX_ERR_TIMEOUT
    monkeypatch.setenv("CX_BARRIER_SPIN_LIMIT", "0")
    sp = specs(1, 0, sizes=[(600, 97), (513, 33), (130, 70)])
    with cx.Batch(sp) as bt:
        bt.tune(4, 0, 0, 20)
        bt.step(40)
        with pytest.raises(cx.CxError) as e:
            cx.cx_batch_synchronize(bt.h)
        assert e.value.code == cx.CX_ERR_TIMEOUT
        cx.cx_batch_synchronize(bt.h)          # the flag was cleared
    monkeypatch.delenv("CX_BARRIER_SPIN_LIMIT")
    with cx.Batch(specs(1, 0, sizes=[(64, 48)])) as bt2:  # the device still works
        bt2.tune(8, 0, 0, 10)
        bt2.step(20)
        assert bt2.diagnostics()[0]["finite"] == 1


def test_batch_time_block_default_and_validation(cx):
    for prec, default, rows in ((1, 2, 128), (0, 1, 32)):
        with cx.Batch(specs(prec, 0, sizes=[(64, 48), (7, 5)])) as bt:
            assert cx.cx_batch_get_time_block(bt.h) == default
            assert cx.cx_batch_get_tuning(bt.h)[0] == rows   # default tile height by depth
            for bad in (0, 3):
                with pytest.raises(cx.CxError) as e:
                    cx.cx_batch_set_time_block(bt.h, bad)
                assert e.value.code == cx.CX_ERR_INVALID_ARG
            cx.cx_batch_set_time_block(bt.h, 3 - default)
            assert cx.cx_batch_get_time_block(bt.h) == 3 - default


def test_single_grid_tile_rows_do_not_change_results(cx):
    cfg = dict(W.CONFIG0, nx=300, ny=257)
    grid, params, seed = W.split(cfg)
    outs = []
    for rows in (1, 8, 32, 100, 300):
        with cx.Sim(300, 257, 1.0, seed=seed, **dict(params, precision=1)) as sim:
            cx.cx_set_tile_rows(sim.h, rows)
            assert cx.cx_get_tile_rows(sim.h) == rows
            sim.step(77)
            outs.append(sim.field(cx.CX_FIELD_B, np.float32))
    for o in outs[1:]:
        assert np.array_equal(o, outs[0])
