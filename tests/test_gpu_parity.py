"""Parity of the CUDA path (called through the C ABI) with the FP64 oracle.

Tolerances: relative L2 <= 1e-12 for the FP64 state and <= 1e-4 for the FP32
state over at most 1000 steps; sigma bit for bit; masses and the conserved
invariant to round-off; integer-decided outputs (the envelope radius) by
computing both sides on the same state.
"""
import math
import os

import numpy as np
import pytest

import oracle
from paper_1301_5058_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL32 = 1e-4


@pytest.fixture(scope="module")
def cx():
    from paper_1301_5058_gb300 import _build
    _build.build()
    import paper_1301_5058_gb300 as cx
    return cx


def rel_l2(x, y):
    d = np.linalg.norm((np.asarray(x, np.float64) - y).ravel())
    return d / max(np.linalg.norm(np.asarray(y).ravel()), 1e-300)


def make_sim(cx, cfg, precision, **over):
    cfg = dict(cfg, **over)
    grid, params, seed = W.split(cfg)
    params["precision"] = precision
    return cx.Sim(grid["nx"], grid["ny"], grid["dx"], seed=seed, **params), cfg


def oracle_inputs(cfg):
    s = oracle.sigma_field(cfg["nx"], cfg["ny"], cfg.get("seed", 0), cfg["sigma0"],
                           cfg["noise_amp"], dist=cfg.get("noise_dist", 0))
    b, n = oracle.initial_state(cfg["nx"], cfg["ny"], cfg["dx"], cfg["n0"], cfg["bM"], cfg["r0sq"])
    return s, b, n


def oracle_dt(cfg):
    return cfg.get("cfl_frac", 0.2) * oracle.dt_limit(
        dx=cfg["dx"], Dn=cfg["Dn"], theta=cfg["theta"], chi0=cfg["chi0"], n0=cfg["n0"],
        bM=cfg["bM"], sigma0=cfg["sigma0"], amp=cfg["noise_amp"])


def oracle_run(cfg, s, b, n, steps):
    return oracle.run(s, b, n, steps, dx=cfg["dx"], dt=oracle_dt(cfg), Dn=cfg["Dn"],
                      theta=cfg["theta"], chi0=cfg["chi0"], chemo_law=cfg.get("chemo_law", 0),
                      mobility=cfg.get("mobility", 0))[:2]


# ---------------------------------------------------------------------------

@pytest.mark.parametrize("dist", [0, 1])
def test_sigma_field_is_bit_exact(cx, dist):
    cfg = dict(W.CONFIG0, nx=300, ny=77, seed=12345, noise_dist=dist)
    ref = oracle.sigma_field(300, 77, 12345, cfg["sigma0"], cfg["noise_amp"], dist=dist)
    with make_sim(cx, cfg, cx.CX_PREC_F64)[0] as sim:
        assert np.array_equal(sim.field(cx.CX_FIELD_SIGMA), ref)
    with make_sim(cx, cfg, cx.CX_PREC_F32)[0] as sim:
        assert np.array_equal(sim.field(cx.CX_FIELD_SIGMA, np.float32), ref.astype(np.float32))


def test_initial_state_matches(cx):
    cfg = dict(W.CONFIG0, nx=130, ny=97, dx=0.37)
    _, b, n = oracle_inputs(cfg)
    with make_sim(cx, cfg, cx.CX_PREC_F64)[0] as sim:
        gb, gn = sim.field(cx.CX_FIELD_B), sim.field(cx.CX_FIELD_N)
    assert np.array_equal(gn, n)
    # exp() of the CUDA math library and of libm may differ in the last place
    assert np.max(np.abs(gb - b) / np.maximum(np.abs(b), 1e-300)) <= 4e-16
    assert rel_l2(gb, b) <= 1e-15


@pytest.mark.parametrize("own_ic", [False, True])
def test_fp64_parity_config0(cx, own_ic):
    cfg = W.CONFIG0
    s, b, n = oracle_inputs(cfg)
    sim, _ = make_sim(cx, cfg, cx.CX_PREC_F64)
    with sim:
        if not own_ic:
            sim.set_field(cx.CX_FIELD_B, b)
            sim.set_field(cx.CX_FIELD_N, n)
        ob, on = b, n
        for chunk in (500, 500):
            sim.step(chunk)
            ob, on = oracle_run(cfg, s, ob, on, chunk)
            gb, gn = sim.field(cx.CX_FIELD_B), sim.field(cx.CX_FIELD_N)
            assert rel_l2(gb, ob) <= TOL64 and rel_l2(gn, on) <= TOL64, (rel_l2(gb, ob), rel_l2(gn, on))


def test_fp64_config0_full_length(cx):
    # the whole 2000-step run of the plain-method case: beyond 1000 steps the
    # check is conservation plus the envelope radius (round-off is amplified
    # by the growth of the colony, not by the scheme)
    cfg = W.CONFIG0
    s, b, n = oracle_inputs(cfg)
    with make_sim(cx, cfg, cx.CX_PREC_F64)[0] as sim:
        sim.set_field(cx.CX_FIELD_B, b)
        sim.set_field(cx.CX_FIELD_N, n)
        d0 = sim.diagnostics()
        sim.step(2000)
        d1 = sim.diagnostics()
        gb, gn = sim.field(cx.CX_FIELD_B), sim.field(cx.CX_FIELD_N)
    ob, on = oracle_run(cfg, s, b, n, 2000)
    od = oracle.diagnostics(ob, on, dx=1.0, theta=1.0, b_th=0.1 * 0.7)
    assert rel_l2(gb, ob) <= 1e-10 and rel_l2(gn, on) <= 1e-10
    assert abs(d1["invariant"] - d0["invariant"]) <= 1e-12 * d0["invariant"]
    assert abs(d1["r_env"] - od["r_env"]) <= 0.01 * od["r_env"]
    assert d1["min_b"] >= 0 and d1["min_n"] >= 0


def test_fp32_parity_config0(cx):
    cfg = W.CONFIG0
    s, b, n = oracle_inputs(cfg)
    with make_sim(cx, cfg, cx.CX_PREC_F32)[0] as sim:
        sim.step(1000)
        gb, gn = sim.field(cx.CX_FIELD_B), sim.field(cx.CX_FIELD_N)
        d = sim.diagnostics()
    ob, on = oracle_run(cfg, s, b, n, 1000)
    e = (rel_l2(gb, ob), rel_l2(gn, on))
    assert max(e) <= TOL32, e
    od = oracle.diagnostics(ob, on, dx=1.0, theta=1.0, b_th=0.07)
    assert d["invariant"] == pytest.approx(od["invariant"], rel=1e-6)


@pytest.mark.parametrize("law", [0, 1])
@pytest.mark.parametrize("mob", [0, 1])
def test_fp64_parity_all_flux_options(cx, law, mob):
    cfg = dict(W.CONFIG0, nx=96, ny=80, chi0=2.0, chemo_law=law, mobility=mob, seed=3)
    s, b, n = oracle_inputs(cfg)
    with make_sim(cx, cfg, cx.CX_PREC_F64)[0] as sim:
        sim.set_field(cx.CX_FIELD_B, b)
        sim.set_field(cx.CX_FIELD_N, n)
        sim.step(300)
        gb, gn = sim.field(cx.CX_FIELD_B), sim.field(cx.CX_FIELD_N)
    ob, on = oracle_run(cfg, s, b, n, 300)
    assert rel_l2(gb, ob) <= TOL64 and rel_l2(gn, on) <= TOL64


@pytest.mark.parametrize("nx,ny", [(1, 1), (1, 37), (37, 1), (7, 5), (3, 3), (4, 5), (513, 70),
                                   (1030, 33), (129, 65), (512, 32)])
def test_fp64_parity_ragged_shapes(cx, nx, ny):
    # random fields exercise every face; shapes span several tiles with
    # ragged tails in x (512 cells per block) and y (32 rows per block)
    cfg = dict(W.CONFIG0, nx=nx, ny=ny, chi0=1.5, seed=nx * 1000 + ny)
    s = oracle.sigma_field(nx, ny, cfg["seed"], cfg["sigma0"], cfg["noise_amp"])
    b, n = W.perturbed_fields(nx, ny, seed=cfg["seed"])
    with make_sim(cx, cfg, cx.CX_PREC_F64)[0] as sim:
        sim.set_field(cx.CX_FIELD_B, b)
        sim.set_field(cx.CX_FIELD_N, n)
        sim.step(40)
        gb, gn = sim.field(cx.CX_FIELD_B), sim.field(cx.CX_FIELD_N)
    ob, on = oracle_run(cfg, s, b, n, 40)
    assert rel_l2(gb, ob) <= TOL64 and rel_l2(gn, on) <= TOL64, (rel_l2(gb, ob), rel_l2(gn, on))


@pytest.mark.parametrize("nx,ny", [(5, 3), (513, 70), (1030, 33)])
def test_fp32_parity_ragged_shapes(cx, nx, ny):
    cfg = dict(W.CONFIG0, nx=nx, ny=ny, chi0=1.5, seed=7)
    s = oracle.sigma_field(nx, ny, 7, cfg["sigma0"], cfg["noise_amp"])
    b, n = W.perturbed_fields(nx, ny, seed=8)
    with make_sim(cx, cfg, cx.CX_PREC_F32)[0] as sim:
        sim.set_field(cx.CX_FIELD_B, b)
        sim.set_field(cx.CX_FIELD_N, n)
        sim.step(40)
        gb, gn = sim.field(cx.CX_FIELD_B), sim.field(cx.CX_FIELD_N)
    ob, on = oracle_run(cfg, s.astype(np.float32).astype(np.float64), b.astype(np.float32).astype(np.float64),
                        n.astype(np.float32).astype(np.float64), 40)
    assert rel_l2(gb, ob) <= TOL32 and rel_l2(gn, on) <= TOL32


@pytest.mark.parametrize("prec", [0, 1])
def test_diagnostics_match_oracle_on_the_same_state(cx, prec):
    cfg = dict(W.CONFIG0, nx=300, ny=200)
    with make_sim(cx, cfg, prec)[0] as sim:
        sim.step(400)
        d = sim.diagnostics()
        dt = np.float64 if prec == 0 else np.float32
        gb, gn = sim.field(cx.CX_FIELD_B, dt), sim.field(cx.CX_FIELD_N, dt)
    od = oracle.diagnostics(gb.astype(np.float64), gn.astype(np.float64), dx=1.0, theta=1.0,
                            b_th=0.1 * 0.7)
    for k in ("mass_b", "mass_n", "invariant"):
        assert d[k] == pytest.approx(od[k], rel=1e-13)
    for k in ("min_b", "min_n", "max_b"):
        assert d[k] == od[k]
    assert d["r_env"] == pytest.approx(od["r_env"], rel=1e-14)
    assert d["area_env"] == od["area_env"] and d["area_env"] > 0
    assert d["finite"] == 1 and d["step"] == 400


def test_conservation_fp64_and_fp32(cx):
    cfg = dict(W.CONFIG0, nx=200, ny=180, theta=0.7, Dn=1.3)
    for prec, tol in ((0, 1e-12), (1, 2e-6)):
        with make_sim(cx, cfg, prec)[0] as sim:
            d0 = sim.diagnostics()
            sim.step(2000)
            d1 = sim.diagnostics()
        assert abs(d1["invariant"] - d0["invariant"]) <= tol * d0["invariant"]
        assert d1["mass_b"] > 3 * d0["mass_b"]


def test_checkpoint_resume_is_bitwise(cx, tmp_path):
    cfg = dict(W.CONFIG0, nx=100, ny=90)
    for prec in (0, 1):
        with make_sim(cx, cfg, prec)[0] as a, make_sim(cx, cfg, prec)[0] as b:
            a.step(137)
            b.step(60)
            path = str(tmp_path / f"c{prec}.ckpt")
            cx.cx_save(b.h, path)
            with cx.Sim.load(path) as c:
                c.step(77)
                assert cx.cx_get_time(c.h)[0] == 137
                for w in (cx.CX_FIELD_B, cx.CX_FIELD_N, cx.CX_FIELD_SIGMA):
                    assert np.array_equal(a.field(w), c.field(w))


def test_runs_are_deterministic(cx):
    cfg = dict(W.CONFIG0, nx=200, ny=150)
    out = []
    for _ in range(2):
        with make_sim(cx, cfg, 1)[0] as sim:
            sim.step(300)
            out.append((sim.field(cx.CX_FIELD_B, np.float32), sim.diagnostics()["invariant"]))
    assert np.array_equal(out[0][0], out[1][0]) and out[0][1] == out[1][1]


def test_health_flags(cx):
    cfg = dict(W.CONFIG0, nx=40, ny=30)
    with make_sim(cx, cfg, 0)[0] as sim:
        b = sim.field(cx.CX_FIELD_B)
        b[5, 6] = -1e-3
        sim.set_field(cx.CX_FIELD_B, b)
        with pytest.raises(cx.CxError) as e:
            sim.diagnostics()
        assert e.value.code == cx.CX_ERR_NEGATIVE
        b[5, 6] = np.nan
        sim.set_field(cx.CX_FIELD_B, b)
        d = sim.diagnostics(check=False)
        assert d["finite"] == 0 and d["status"] == cx.CX_ERR_NONFINITE


def test_field_io_converts_precision(cx):
    cfg = dict(W.CONFIG0, nx=33, ny=17)
    with make_sim(cx, cfg, 1)[0] as sim:
        b32 = sim.field(cx.CX_FIELD_B, np.float32)
        b64 = sim.field(cx.CX_FIELD_B, np.float64)
        assert np.array_equal(b32.astype(np.float64), b64)
        x = np.linspace(0, 1, 33 * 17).reshape(17, 33)
        sim.set_field(cx.CX_FIELD_N, x)
        assert np.array_equal(sim.field(cx.CX_FIELD_N, np.float32), x.astype(np.float32))
        with pytest.raises(cx.CxError):
            cx.cx_get_field(sim.h, cx.CX_FIELD_B, np.empty(10), )


# ---------------------------------------------------------------------------
# The 16384^2 FP32 workload, in the launch configuration the benchmark times
# (two Euler steps per pass): the oracle checks one pass, two steps, on
# sampled windows (corners, edges, interior, the ragged ends of blocks) from
# the same FP32 state.

def _envelope_series(cx, cfg, prec, steps, samples):
    with make_sim(cx, cfg, prec)[0] as sim:
        d0 = sim.diagnostics()
        t, r = [], []
        for _ in range(samples):
            sim.step(steps // samples)
            d = sim.diagnostics()
            t.append(d["t"])
            r.append(d["r_env"])
        gb = sim.field(cx.CX_FIELD_B)
    return np.array(t), np.array(r), d0, d, gb


def test_long_run_fp32_against_fp64_envelope(cx):
    # beyond 1000 steps round-off is amplified by the growth of the colony, so
    # long runs are compared on the envelope radius and its velocity (within
    # 1 %) and on conservation; the FP64 GPU path is itself pinned to the
    # oracle at 1e-12 (tests above)
    cfg = dict(W.CONFIG1, nx=2048, ny=2048, r0sq=32.0 ** 2)
    t64, r64, a64, z64, b64 = _envelope_series(cx, cfg, cx.CX_PREC_F64, 20000, 20)
    t32, r32, a32, z32, b32 = _envelope_series(cx, cfg, cx.CX_PREC_F32, 20000, 20)
    assert np.allclose(t32, t64, rtol=1e-12)
    assert np.max(np.abs(r32 - r64) / r64) <= 0.01
    h = len(t64) // 2
    v64 = np.polyfit(t64[h:], r64[h:], 1)[0]
    v32 = np.polyfit(t32[h:], r32[h:], 1)[0]
    assert abs(v32 - v64) <= 0.01 * abs(v64)
    assert abs(z64["invariant"] - a64["invariant"]) <= 1e-12 * a64["invariant"]
    assert abs(z32["invariant"] - a32["invariant"]) <= 1e-5 * a32["invariant"]
    print(f"\nFP32 vs FP64, 2048^2, 20000 steps: rel L2(b) = {rel_l2(b32, b64):.3e}, "
          f"max rel r_env diff = {np.max(np.abs(r32 - r64) / r64):.3e}, v32 = {v32:.6f}, "
          f"v64 = {v64:.6f}, FP32 invariant drift = "
          f"{abs(z32['invariant'] - a32['invariant']) / a32['invariant']:.3e}")


@pytest.mark.parametrize("n,steps", [(256, 100), (256, 1000), (1024, 1000)])
def test_error_table_fp32_fp64_against_oracle(cx, n, steps):
    # relative L2 error of both GPU precisions against the FP64 oracle
    cfg = dict(W.CONFIG0, nx=n, ny=n)
    s, b, n0 = oracle_inputs(cfg)
    ob, on = oracle_run(cfg, s, b, n0, steps)
    errs = {}
    for prec in (cx.CX_PREC_F64, cx.CX_PREC_F32):
        with make_sim(cx, cfg, prec)[0] as sim:
            sim.set_field(cx.CX_FIELD_B, b)
            sim.set_field(cx.CX_FIELD_N, n0)
            sim.step(steps)
            errs[prec] = (rel_l2(sim.field(cx.CX_FIELD_B), ob), rel_l2(sim.field(cx.CX_FIELD_N), on))
    print(f"\n{n}^2 x {steps} steps: FP64 rel L2 (b, n) = {errs[0][0]:.2e}, {errs[0][1]:.2e}; "
          f"FP32 = {errs[1][0]:.2e}, {errs[1][1]:.2e}")
    assert max(errs[0]) <= TOL64 and max(errs[1]) <= TOL32


def _window_error(cfg, dt, s, b0, n0, b1, n1, windows, size=40, steps=2):
    nx, ny = cfg["nx"], cfg["ny"]
    worst = 0.0
    for (x0, y0) in windows:
        xa, ya = max(x0, 0), max(y0, 0)
        xb, yb = min(x0 + size, nx), min(y0 + size, ny)
        sub = lambda a: a[ya:yb, xa:xb].astype(np.float64)
        ob, on, _ = oracle.run(sub(s), sub(b0), sub(n0), steps, dx=cfg["dx"], dt=dt,
                               Dn=cfg["Dn"], theta=cfg["theta"], chi0=cfg["chi0"])
        # the window's own edges are walls for the oracle: compare only cells
        # whose dependence cone (`steps` cells) lies inside the window or
        # reaches only the true domain wall
        m = np.ones(ob.shape, bool)
        if xa > 0: m[:, :steps] = False
        if xb < nx: m[:, -steps:] = False
        if ya > 0: m[:steps, :] = False
        if yb < ny: m[-steps:, :] = False
        eb = np.abs(ob - b1[ya:yb, xa:xb])[m].max()
        en = np.abs(on - n1[ya:yb, xa:xb])[m].max()
        worst = max(worst, eb, en)
    return worst


def test_full_size_fp32_sampled_windows(cx):
    cfg = dict(W.CONFIG1)
    nx, ny = cfg["nx"], cfg["ny"]
    c = nx // 2
    edges = [(0, 0), (nx - 40, 0), (0, ny - 40), (nx - 40, ny - 40), (c - 20, 0), (0, c - 20),
             (511 - 10, c + 30), (4095, 31 * 32 - 5), (nx - 513, ny - 33),
             (480 - 20, 64 * 7 - 20), (119 - 20, c), (34 * 480 - 20, ny - 70)]
    centre = [(c - 20, c - 20), (c - 60, c - 3), (c + 5, c - 50), (c - 45, c + 10)]
    with make_sim(cx, cfg, cx.CX_PREC_F32)[0] as sim:
        assert cx.cx_get_time_block(sim.h) == 2  # the benchmark's configuration
        dt = cx.cx_get_time(sim.h)[2]
        d0 = sim.diagnostics()
        # phase 1: the inoculum after 200 steps (the colony is near the centre)
        sim.step(200)
        s = sim.field(cx.CX_FIELD_SIGMA, np.float32)
        b0 = sim.field(cx.CX_FIELD_B, np.float32)
        n0 = sim.field(cx.CX_FIELD_N, np.float32)
        sim.step(2)
        b1 = sim.field(cx.CX_FIELD_B, np.float32)
        n1 = sim.field(cx.CX_FIELD_N, np.float32)
        d1 = sim.diagnostics()
        assert abs(d1["invariant"] - d0["invariant"]) <= 1e-6 * d0["invariant"]
        assert d1["min_b"] >= 0 and d1["min_n"] >= 0 and d1["finite"] == 1
        assert _window_error(cfg, dt, s, b0, n0, b1, n1, centre + edges) <= 2e-6
        # phase 2: seeded random fields everywhere, so every window is busy
        rng = np.random.default_rng(2024)
        b0 = (0.05 + 0.5 * rng.random((ny, nx), dtype=np.float32)).astype(np.float32)
        n0 = (0.05 + 0.4 * rng.random((ny, nx), dtype=np.float32)).astype(np.float32)
        sim.set_field(cx.CX_FIELD_B, b0)
        sim.set_field(cx.CX_FIELD_N, n0)
        sim.step(2)
        b1 = sim.field(cx.CX_FIELD_B, np.float32)
        n1 = sim.field(cx.CX_FIELD_N, np.float32)
    assert _window_error(cfg, dt, s, b0, n0, b1, n1, centre + edges) <= 4e-6


# ---------------------------------------------------------------------------
# The paper's own scheme (Sec. 3): second-order Runge-Kutta (Heun) and sigma
# redrawn from a triangular law at every grid point and time step.

@pytest.mark.parametrize("prec", [0, 1])
def test_per_step_sigma_is_bit_exact(cx, prec):
    cfg = dict(W.CONFIG0, nx=130, ny=70, noise_mode=1, noise_dist=1, noise_amp=1.0, seed=21)
    recipe = oracle.sigma_field if prec == 0 else oracle.sigma_field_f32
    with make_sim(cx, cfg, prec)[0] as sim:
        for k in (0, 3):
            sim.step(k)
            step = cx.cx_get_time(sim.h)[0]
            ref = recipe(130, 70, 21, cfg["sigma0"], 1.0, dist=1, step=step)
            assert np.array_equal(sim.field(cx.CX_FIELD_SIGMA), ref)


@pytest.mark.parametrize("scheme", [0, 1])
@pytest.mark.parametrize("noise_mode", [0, 1])
def test_fp64_parity_scheme_and_noise(cx, scheme, noise_mode):
    cfg = dict(W.CONFIG0, nx=150, ny=131, chi0=1.0, scheme=scheme, noise_mode=noise_mode,
               noise_dist=1, noise_amp=1.0, seed=5)
    s, b, n = oracle_inputs(cfg)
    with make_sim(cx, cfg, cx.CX_PREC_F64)[0] as sim:
        sim.set_field(cx.CX_FIELD_B, b)
        sim.set_field(cx.CX_FIELD_N, n)
        sim.step(400)
        gb, gn = sim.field(cx.CX_FIELD_B), sim.field(cx.CX_FIELD_N)
    ob, on, _ = oracle.run(s, b, n, 400, dx=1.0, dt=oracle_dt(cfg), Dn=1.0, theta=1.0, chi0=1.0,
                           scheme=scheme, noise_mode=noise_mode, seed=5, sigma0=cfg["sigma0"],
                           amp=1.0, dist=1, recipe=0)
    assert rel_l2(gb, ob) <= TOL64 and rel_l2(gn, on) <= TOL64, (rel_l2(gb, ob), rel_l2(gn, on))


@pytest.mark.parametrize("scheme", [0, 1])
def test_fp32_parity_paper_scheme(cx, scheme):
    cfg = dict(W.CONFIG0, nx=200, ny=190, chi0=1.0, scheme=scheme, noise_mode=1, noise_dist=1,
               noise_amp=1.0, seed=8)
    s, b, n = oracle_inputs(cfg)
    with make_sim(cx, cfg, cx.CX_PREC_F32)[0] as sim:
        sim.step(1000)
        gb, gn = sim.field(cx.CX_FIELD_B), sim.field(cx.CX_FIELD_N)
    ob, on, _ = oracle.run(s, b, n, 1000, dx=1.0, dt=oracle_dt(cfg), Dn=1.0, theta=1.0, chi0=1.0,
                           scheme=scheme, noise_mode=1, seed=8, sigma0=cfg["sigma0"], amp=1.0,
                           dist=1, recipe=1)
    assert rel_l2(gb, ob) <= TOL32 and rel_l2(gn, on) <= TOL32


@pytest.mark.parametrize("nx,ny", [(1, 1), (7, 5), (513, 70), (1030, 33)])
def test_fp64_heun_ragged_shapes(cx, nx, ny):
    cfg = dict(W.CONFIG0, nx=nx, ny=ny, chi0=1.5, scheme=1, noise_mode=1, noise_dist=1, seed=nx + ny)
    b, n = W.perturbed_fields(nx, ny, seed=cfg["seed"])
    with make_sim(cx, cfg, cx.CX_PREC_F64)[0] as sim:
        sim.set_field(cx.CX_FIELD_B, b)
        sim.set_field(cx.CX_FIELD_N, n)
        sim.step(30)
        gb, gn = sim.field(cx.CX_FIELD_B), sim.field(cx.CX_FIELD_N)
    ob, on, _ = oracle.run(np.zeros((ny, nx)), b, n, 30, dx=1.0, dt=oracle_dt(cfg), Dn=1.0,
                           theta=1.0, chi0=1.5, scheme=1, noise_mode=1, seed=cfg["seed"],
                           sigma0=cfg["sigma0"], amp=cfg["noise_amp"], dist=1, recipe=0)
    assert rel_l2(gb, ob) <= TOL64 and rel_l2(gn, on) <= TOL64


def test_heun_conserves_and_resumes_bitwise(cx, tmp_path):
    cfg = dict(W.CONFIG0, nx=120, ny=100, scheme=1, noise_mode=1, noise_dist=1, theta=0.8)
    for prec, tol in ((0, 1e-12), (1, 2e-6)):
        with make_sim(cx, cfg, prec)[0] as a, make_sim(cx, cfg, prec)[0] as b:
            d0 = a.diagnostics()
            a.step(500)
            d1 = a.diagnostics()
            assert abs(d1["invariant"] - d0["invariant"]) <= tol * d0["invariant"]
            b.step(200)
            path = str(tmp_path / f"h{prec}.ckpt")
            cx.cx_save(b.h, path)
            with cx.Sim.load(path) as c:
                c.step(300)
                for w in (cx.CX_FIELD_B, cx.CX_FIELD_N):
                    assert np.array_equal(a.field(w), c.field(w))
