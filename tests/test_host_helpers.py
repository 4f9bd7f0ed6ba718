"""Host-side helpers of the sweep, surrogate, autotuner and front-speed code:
their definitions checked on CPU against closed forms and invariants."""
import json
import math

import numpy as np
import pytest

from paper_1301_5058_gb300 import autotune, front_speed, surrogate
from paper_1301_5058_gb300 import workloads as W


def test_sweep_specs_cover_the_box_and_are_reproducible():
    a, b = W.sweep_specs(512, seed=0), W.sweep_specs(512, seed=0)
    assert a == b and len(a) == 512
    assert {s["nx"] for s in a} == set(W.SWEEP_SIDES) and all(s["nx"] == s["ny"] for s in a)
    assert [s["seed"] for s in a] == list(range(512))
    n0 = np.array([s["n0"] for s in a])
    chi0 = np.array([s["chi0"] for s in a])
    s0 = np.array([s["sigma0"] for s in a])
    assert n0.min() >= 0.1 and n0.max() <= 1.5
    assert s0.min() >= 1.0 and s0.max() <= 8.0
    assert chi0.max() <= 4.0 and (chi0 == 0).any() and ((chi0 == 0) | (chi0 >= 0.05)).all()
    # log-uniform draws: log n0 has the mean of the interval's log midpoint
    assert abs(np.log(n0).mean() - 0.5 * (np.log(0.1) + np.log(1.5))) < 0.1
    assert W.sweep_specs(512, seed=1) != a


def test_encode_maps_the_box_onto_the_cube():
    corners = [[0.1, 0.0, 1.0, 0.0], [1.5, 4.0, 8.0, 1.0], [math.sqrt(0.15), 2.0, math.sqrt(8.0), 0.5]]
    x = surrogate.encode(corners)
    assert np.allclose(x[0], -1.0) and np.allclose(x[1], 1.0) and np.allclose(x[2], 0.0, atol=1e-6)
    p = surrogate.draw_points(1000, seed=3)
    e = surrogate.encode(p)
    assert e.dtype == np.float32 and e.min() >= -1.0 - 1e-6 and e.max() <= 1.0 + 1e-6


@pytest.mark.parametrize("k", [1, 2, 5, 9])
def test_count_runs_counts_circular_arcs(k):
    th = np.linspace(0.0, 2 * np.pi, 4096, endpoint=False)
    prof = np.cos(k * th + 0.3)
    assert surrogate.count_runs(prof, 0.5) == k
    assert surrogate.count_runs(np.ones(64), 0.5) == 0       # a closed ring is no branch
    assert surrogate.count_runs(np.zeros(64), 0.5) == 0
    # an arc through the wrap-around point counts once
    assert surrogate.count_runs(np.r_[np.ones(3), np.zeros(10), np.ones(3)], 0.5) == 1


def test_slopes_recover_lines():
    t = np.linspace(0.0, 10.0, 41)
    r = 3.0 + 0.25 * t
    assert surrogate.lsq_slope(t, r) == pytest.approx(0.25, rel=1e-12)
    assert math.isnan(surrogate.lsq_slope(np.ones(5), r[:5]))
    # fit_speed keeps only lo <= r <= hi
    rr = np.where(t < 5.0, r, 100.0)
    assert front_speed.fit_speed(t, rr, 0.0, 10.0) == pytest.approx(0.25, rel=1e-12)
    assert math.isnan(front_speed.fit_speed(t, r, 50.0, 60.0))


def test_strip_spec_is_the_one_dimensional_workload():
    s = front_speed.strip_spec(0.7, 2.5)
    assert s["ny"] == 1 and s["nx"] == 400 and s["noise_amp"] == 0.0
    assert s["b_threshold"] == pytest.approx(0.35)


def test_autotune_cache_round_trip(tmp_path, monkeypatch):
    monkeypatch.setenv("CX_TUNE_CACHE", str(tmp_path / "sub" / "tune.json"))
    assert autotune._load_cache() == {}
    autotune._store("a", [1, 2])
    autotune._store("b", {"x": 3})
    assert autotune._load_cache() == {"a": [1, 2], "b": {"x": 3}}
    (tmp_path / "sub" / "tune.json").write_text("not json")
    assert autotune._load_cache() == {}                       # a damaged cache is ignored


def test_batch_key_names_the_size_mix():
    class G:
        def __init__(self, n):
            self.nx = self.ny = n

    class P:
        precision, scheme = 1, 0

    key = autotune.batch_key([G(512), G(1024), G(512)], [P()])
    assert key == "batch/p1/s0/512x512:2,1024x1024:1"          # sizes in numeric order
    assert json.dumps(key)


def test_smooth_time_step_stays_below_the_stability_limit():
    # the sweep's time step is never above the library's limit (the runs stay
    # stable), is within a factor 3 of it, and has no kink where the limit's
    # max / min switch branches (a finite-difference second derivative along
    # a line through such a switch stays bounded)
    from paper_1301_5058_gb300 import _build
    _build.build()
    import paper_1301_5058_gb300 as cx
    pts = surrogate.draw_points(400, seed=11, a_range=(0.0, 1.0))
    sd = surrogate.smooth_dt(pts)
    g = cx.cx_grid(8, 8, 1.0)
    for p, d in zip(pts, sd):
        prm = cx.cx_params_default(n0=p[0], chi0=p[1], sigma0=p[2], noise_amp=p[3], bM=0.71)
        lim = prm.cfl_frac * cx.cx_dt_limit(g, prm)
        assert 0.3 * lim <= d <= lim
    # along sigma0 the library's diffusivity switches from Dn to the cross
    # diffusivity (a kink of the limit); the smooth step's curvature stays small
    s0 = np.linspace(0.2, 3.0, 2001)
    line = np.stack([np.full_like(s0, 0.3), np.zeros_like(s0), s0, np.zeros_like(s0)], 1)
    y = np.log(surrogate.smooth_dt(line))
    d2 = np.diff(y, 2) / (s0[1] - s0[0]) ** 2
    assert np.max(np.abs(d2)) < 10.0


def test_initial_area_radius_is_the_disc_above_the_level():
    # bM exp(-r^2 / r0sq) >= 0.1 n0  <=>  r^2 <= r0sq ln(bM / (0.1 n0))
    n0 = np.array([0.1, 0.35, 1.5, 7.1])
    r = surrogate.initial_area_radius(n0, 32.0 ** 2)
    for ni, ri in zip(n0, r):
        if 0.71 > 0.1 * ni:
            assert 0.71 * math.exp(-ri ** 2 / 32.0 ** 2) == pytest.approx(0.1 * ni, rel=1e-12)
        else:
            assert ri == 0.0


def test_poly_features_span_the_monomials():
    X = np.random.default_rng(0).uniform(-1, 1, (50, 4))
    F = surrogate.poly_features(X, 3)
    assert F.shape == (50, 35)          # C(4 + 3, 3) monomials of degree <= 3
    assert np.allclose(F[:, 0], 1.0) and np.allclose(F[:, 1:5], X)
