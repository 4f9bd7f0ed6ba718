"""Temporal blocking (cx_set_time_block): a pass that takes two explicit
stages must reproduce, bit for bit, the passes it replaces (two Euler steps,
or both Heun stages), on ragged shapes that cut through its 120-column warps,
480-column blocks and row tiles, for every flux, noise and scheme option and
both precisions; and it stays within the parity tolerances of the FP64
oracle."""
import numpy as np
import pytest

import oracle
from paper_1301_5058_gb300 import workloads as W

from _layout import natural

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


def run(cx, cfg, prec, steps, time_block, rows=None, fields=None):
    grid, params, seed = W.split(cfg)
    params["precision"] = prec
    with cx.Sim(grid["nx"], grid["ny"], grid["dx"], seed=seed, **params) as sim:
        cx.cx_set_time_block(sim.h, time_block)
        assert cx.cx_get_time_block(sim.h) == time_block
        if rows is not None:
            cx.cx_set_tile_rows(sim.h, rows)
        if fields is not None:
            sim.set_field(cx.CX_FIELD_B, fields[0])
            sim.set_field(cx.CX_FIELD_N, fields[1])
        sim.step(steps)
        dtype = np.float64 if prec == 0 else np.float32
        d = sim.diagnostics(check=False)
        return sim.field(cx.CX_FIELD_B, dtype), sim.field(cx.CX_FIELD_N, dtype), d


SHAPES = [(1, 1), (2, 3), (5, 1), (1, 9), (119, 7), (120, 5), (121, 33), (239, 4), (480, 6),
          (481, 17), (484, 9), (485, 40), (963, 11), (1030, 33)]


@pytest.mark.parametrize("nx,ny", SHAPES)
@pytest.mark.parametrize("prec", [0, 1])
def test_fused_euler_is_bitwise_ragged(cx, nx, ny, prec):
    cfg = dict(W.CONFIG0, nx=nx, ny=ny, chi0=1.5, seed=nx * 7 + ny)
    f = W.perturbed_fields(nx, ny, seed=cfg["seed"])
    a = run(cx, cfg, prec, 7, 1, fields=f)
    b = run(cx, cfg, prec, 7, 2, fields=f)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    assert a[2]["step"] == b[2]["step"] == 7


@pytest.mark.parametrize("law", [0, 1])
@pytest.mark.parametrize("mob", [0, 1])
@pytest.mark.parametrize("scheme", [0, 1])
@pytest.mark.parametrize("noise_mode", [0, 1])
@pytest.mark.parametrize("prec", [0, 1])
def test_fused_is_bitwise_every_option(cx, law, mob, scheme, noise_mode, prec):
    cfg = dict(W.CONFIG0, nx=611, ny=45, chi0=2.0, chemo_law=law, mobility=mob, scheme=scheme,
               noise_mode=noise_mode, noise_dist=1, noise_amp=1.0, seed=3)
    f = W.perturbed_fields(611, 45, seed=11)
    a = run(cx, cfg, prec, 9, 1, fields=f)
    b = run(cx, cfg, prec, 9, 2, fields=f)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


@pytest.mark.parametrize("rows", [1, 2, 3, 5, 32, 200])
def test_fused_tile_heights(cx, rows):
    cfg = dict(W.CONFIG0, nx=500, ny=123, chi0=1.0, noise_mode=1, seed=2)
    f = W.perturbed_fields(500, 123, seed=5)
    a = run(cx, cfg, 1, 12, 1, fields=f)
    b = run(cx, cfg, 1, 12, 2, rows=rows, fields=f)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_fused_config0_against_oracle(cx):
    cfg = dict(W.CONFIG0)
    s = oracle.sigma_field(cfg["nx"], cfg["ny"], cfg["seed"], cfg["sigma0"], cfg["noise_amp"])
    b0, n0 = oracle.initial_state(cfg["nx"], cfg["ny"], cfg["dx"], cfg["n0"], cfg["bM"],
                                  cfg["r0sq"])
    dt = cfg["cfl_frac"] * oracle.dt_limit(dx=cfg["dx"], Dn=cfg["Dn"], theta=cfg["theta"],
                                           chi0=cfg["chi0"], n0=cfg["n0"], bM=cfg["bM"],
                                           sigma0=cfg["sigma0"], amp=cfg["noise_amp"])
    ob, on, _ = oracle.run(s, b0, n0, 1000, dx=cfg["dx"], dt=dt, Dn=cfg["Dn"],
                           theta=cfg["theta"], chi0=cfg["chi0"])
    for prec, tol in ((0, TOL64), (1, TOL32)):
        gb, gn, _ = run(cx, cfg, prec, 1000, 2)
        assert rel_l2(gb, ob) <= tol and rel_l2(gn, on) <= tol, (prec, rel_l2(gb, ob))


def test_fused_paper_scheme_against_oracle(cx):
    # Heun with sigma redrawn every step from the triangular law, FP32 recipe
    cfg = dict(W.CONFIG0, nx=200, ny=190, chi0=1.0, scheme=1, noise_mode=1, noise_dist=1,
               noise_amp=1.0, seed=8)
    s = np.zeros((190, 200))
    b0, n0 = oracle.initial_state(200, 190, 1.0, cfg["n0"], cfg["bM"], cfg["r0sq"])
    dt = 0.2 * oracle.dt_limit(dx=1.0, Dn=1.0, theta=1.0, chi0=1.0, n0=cfg["n0"], bM=cfg["bM"],
                               sigma0=cfg["sigma0"], amp=1.0)
    ob, on, _ = oracle.run(s, b0, n0, 1000, dx=1.0, dt=dt, Dn=1.0, theta=1.0, chi0=1.0, scheme=1,
                           noise_mode=1, seed=8, sigma0=cfg["sigma0"], amp=1.0, dist=1, recipe=1)
    gb, gn, _ = run(cx, cfg, 1, 1000, 2)
    assert rel_l2(gb, ob) <= TOL32 and rel_l2(gn, on) <= TOL32


def test_time_block_defaults_and_rejects_other_depths(cx):
    for prec, default in ((0, 1), (1, 2)):
        params = dict(W.split(dict(W.CONFIG0, nx=16, ny=16))[1], precision=prec)
        with cx.Sim(16, 16, 1.0, seed=0, **params) as sim:
            assert cx.cx_get_time_block(sim.h) == default
            for bad in (0, 3, -1):
                with pytest.raises(cx.CxError) as e:
                    cx.cx_set_time_block(sim.h, bad)
                assert e.value.code == cx.CX_ERR_INVALID_ARG
            assert cx.cx_get_time_block(sim.h) == default


def test_automatic_tile_height_follows_the_depth(cx):
    # 8192^2 launches enough tiles for either cap; smaller grids get fewer
    # rows so that every SM gets its share of tiles: sixteen one-warp tiles
    # of 120 columns (two stages, static sigma), eight four-warp tiles of 480
    # columns (two stages, sigma drawn per step), four of 512 (one stage)
    params = dict(W.split(W.CONFIG0)[1], precision=1)
    sms = 152
    with cx.Sim(8192, 8192, 1.0, seed=0, **params) as sim:
        cx.cx_set_time_block(sim.h, 1)
        assert cx.cx_get_tile_rows(sim.h) == 32
        cx.cx_set_time_block(sim.h, 2)
        assert cx.cx_get_tile_rows(sim.h) == 64
    with cx.Sim(4096, 4096, 1.0, seed=0, **params) as sim:
        assert cx.cx_get_tile_rows(sim.h) == -(-4096 * 35 // (16 * sms))  # 59
        cx.cx_set_tile_rows(sim.h, 17)
        assert cx.cx_get_tile_rows(sim.h) == 17
        cx.cx_set_tile_rows(sim.h, 0)
        assert cx.cx_get_tile_rows(sim.h) == 59
        cx.cx_set_time_block(sim.h, 1)
        assert cx.cx_get_tile_rows(sim.h) == 32   # 54 rows' worth of tiles, capped
    for side, rows in ((512, 2), (1024, 4), (1536, 9), (2048, 16)):
        with cx.Sim(side, side, 1.0, seed=0, **params) as sim:
            assert cx.cx_get_tile_rows(sim.h) == rows
    ps = dict(params, noise_mode=cx.CX_NOISE_PER_STEP)
    with cx.Sim(4096, 4096, 1.0, seed=0, **ps) as sim:
        assert cx.cx_get_tile_rows(sim.h) == -(-4096 * 9 // (8 * sms))  # 31


def test_autotuner_picks_depth_and_height(cx, tmp_path, monkeypatch):
    monkeypatch.setenv("CX_TUNE_CACHE", str(tmp_path / "tune.json"))
    from paper_1301_5058_gb300 import autotune
    params = dict(W.split(W.CONFIG0)[1], precision=1)
    with cx.Sim(1024, 1024, 1.0, seed=0, **params) as sim:
        choice, res = autotune.tune_single(sim, steps=4, reps=1, use_cache=False)
        assert {d for d, _ in res} == {1, 2} and choice == min(res, key=res.get)
        assert (cx.cx_get_time_block(sim.h), cx.cx_get_tile_rows(sim.h)) == choice
        again, _ = autotune.tune_single(sim, use_cache=True)
        assert again == choice


@pytest.mark.parametrize("prec", [0, 1])
def test_create_with_caller_buffers(cx, prec):
    # the fields in device arrays a framework owns (torch tensors here): the
    # run equals a library-allocated one bit for bit, and the arrays hold it
    import torch
    nx, ny, pitch = 300, 77, 320
    cfg = dict(W.CONFIG0, nx=nx, ny=ny, chi0=1.0, seed=4)
    grid, params, seed = W.split(cfg)
    params["precision"] = prec
    dtype = torch.float64 if prec == 0 else torch.float32
    b = torch.full((2, ny, pitch), 7.0, dtype=dtype, device="cuda")
    n = torch.full((2, ny, pitch), 7.0, dtype=dtype, device="cuda")
    s = torch.full((ny, pitch), 7.0, dtype=dtype, device="cuda")
    g, p = cx.cx_grid(nx, ny, 1.0), cx.cx_params_default(**params)
    h = cx.cx_create_with_buffers(g, p, seed, [b[0].data_ptr(), b[1].data_ptr()],
                                  [n[0].data_ptr(), n[1].data_ptr()], s.data_ptr(), pitch)
    npd = np.float64 if prec == 0 else np.float32
    with cx.Sim(nx, ny, 1.0, seed=seed, handle=h, **params) as own, \
            cx.Sim(nx, ny, 1.0, seed=seed, **params) as ref:
        torch.cuda.synchronize()
        assert np.array_equal(natural(s, nx), ref.field(cx.CX_FIELD_SIGMA, npd))
        for sim in (own, ref):
            sim.step(37)
        for w in (cx.CX_FIELD_B, cx.CX_FIELD_N):
            assert np.array_equal(own.field(w, npd), ref.field(w, npd))
        cur = own.field(cx.CX_FIELD_B, npd)
        held = [natural(b[q], nx) for q in (0, 1)]
        assert any(np.array_equal(cur, x) for x in held)


def test_create_with_caller_buffers_rejects_bad_layouts(cx):
    import torch
    nx, ny, pitch = 64, 16, 64
    params = dict(W.split(dict(W.CONFIG0, nx=nx, ny=ny))[1], precision=1)
    g, p = cx.cx_grid(nx, ny, 1.0), cx.cx_params_default(**params)
    t = torch.zeros((6, ny, pitch), dtype=torch.float32, device="cuda")
    ptr = [t[i].data_ptr() for i in range(6)]
    bad = [
        ([ptr[0], ptr[1]], [ptr[2], ptr[3]], ptr[4], nx - 4),        # pitch < nx
        ([ptr[0], ptr[1]], [ptr[2], ptr[3]], ptr[4], 66),            # row not 16-byte sized
        ([ptr[0] + 4, ptr[1]], [ptr[2], ptr[3]], ptr[4], pitch),     # misaligned
        ([ptr[0], ptr[0] + 256], [ptr[2], ptr[3]], ptr[4], pitch),   # overlapping
    ]
    for b, n, s, pt in bad:
        with pytest.raises(cx.CxError) as e:
            cx.cx_create_with_buffers(g, p, 0, b, n, s, pt)
        assert e.value.code == cx.CX_ERR_INVALID_ARG
    # FP64 rows of 66 elements are 16-byte sized but not whole groups of four
    p64 = cx.cx_params_default(**dict(params, precision=0))
    t64 = torch.zeros((6, ny, 68), dtype=torch.float64, device="cuda")
    q = [t64[i].data_ptr() for i in range(6)]
    with pytest.raises(cx.CxError) as e:
        cx.cx_create_with_buffers(g, p64, 0, [q[0], q[1]], [q[2], q[3]], q[4], 66)
    assert e.value.code == cx.CX_ERR_INVALID_ARG
