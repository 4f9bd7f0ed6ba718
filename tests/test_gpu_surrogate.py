"""The learned part on the GPU: the network's forward pass and gradient
against the FP64 oracle (with bf16 rounding at the same operands), training
on the GPU, the polar-profile label against the oracle's bilinear sampling,
and a small end-to-end surrogate fit on solver labels."""
import numpy as np
import pytest

import oracle
from oracle import mlp as omlp
from paper_1301_5058_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cx():
    from paper_1301_5058_gb300 import _build
    _build.build()
    import paper_1301_5058_gb300 as cx
    return cx


def _theta(seed):
    rng = np.random.default_rng(seed)
    parts = {"W1": rng.normal(0, 0.5, (256, 4)), "b1": rng.normal(0, 0.1, 256),
             "W2": rng.normal(0, 1 / 16, (256, 256)), "b2": rng.normal(0, 0.1, 256),
             "W3": rng.normal(0, 1 / 16, (2, 256)), "b3": rng.normal(0, 0.1, 2)}
    return omlp.pack(parts).astype(np.float32)


def _blocks(v):
    out, o = {}, 0
    for name, shape in omlp.SHAPES:
        k = int(np.prod(shape))
        out[name] = np.asarray(v[o:o + k], np.float64)
        o += k
    return out


@pytest.mark.parametrize("batch", [50, 128, 1000])
def test_gradient_matches_oracle(cx, batch):
    theta = _theta(batch)
    rng = np.random.default_rng(batch + 1)
    X = rng.uniform(-1, 1, (batch, 4)).astype(np.float32)
    T = rng.normal(size=(batch, 2)).astype(np.float32)
    with cx.Mlp(1024, theta) as net:
        loss, g = net.gradient(X, T)
        y = net.forward(X)
    oloss, og = omlp.loss_and_grad(theta.astype(np.float64), X.astype(np.float64),
                                   T.astype(np.float64), rounding=True)
    oy, _ = omlp.forward(theta.astype(np.float64), X.astype(np.float64), rounding=True)
    assert loss == pytest.approx(oloss, rel=1e-4)
    assert np.linalg.norm(y - oy) <= 1e-4 * np.linalg.norm(oy)
    gb, ob = _blocks(g), _blocks(og)
    for name in gb:
        err = np.linalg.norm(gb[name] - ob[name]) / max(np.linalg.norm(ob[name]), 1e-30)
        assert err <= 1e-3, (name, err)


def test_members_compute_what_single_networks_compute(cx):
    # three members with their own parameters and training rows: forward,
    # gradient and 40 Adam steps equal, bit for bit, one-member networks
    # given the same parameters and rows (batch 200: two 128-row tiles, one
    # of them ragged)
    E, n, batch = 3, 600, 200
    thetas = [_theta(10 + k) for k in range(E)]
    rng = np.random.default_rng(3)
    X = rng.uniform(-1, 1, (E, n, 4)).astype(np.float32)
    T = rng.normal(size=(E, n, 2)).astype(np.float32)
    with cx.Mlp(1024, np.stack(thetas), members=E) as net:
        y = net.forward(X[0])
        loss, g = net.gradient(X[0, :batch], T[0, :batch])
        losses = net.train(X, T, batch, 40, 1e-3)
        p = net.params()
    assert y.shape == (E, n, 2) and g.shape == (E, 67586) and losses.shape == (E, 40)
    for k in range(E):
        with cx.Mlp(1024, thetas[k]) as one:
            assert np.array_equal(one.forward(X[0]), y[k])
            l1, g1 = one.gradient(X[0, :batch], T[0, :batch])
            assert l1 == loss[k] and np.array_equal(g1, g[k])
            assert np.array_equal(one.train(X[k], T[k], batch, 40, 1e-3), losses[k])
            assert np.array_equal(one.params(), p[k])


@pytest.mark.parametrize("batch,cap", [(1, 1), (128, 128), (129, 256)])
def test_gradient_edge_batches_match_oracle(cx, batch, cap):
    # one valid row in a 128-row tile; a batch at exactly the capacity; one
    # row into a second tile
    theta = _theta(batch + 7)
    rng = np.random.default_rng(batch)
    X = rng.uniform(-1, 1, (batch, 4)).astype(np.float32)
    T = rng.normal(size=(batch, 2)).astype(np.float32)
    with cx.Mlp(cap, theta) as net:
        loss, g = net.gradient(X, T)
    oloss, og = omlp.loss_and_grad(theta.astype(np.float64), X.astype(np.float64),
                                   T.astype(np.float64), rounding=True)
    assert loss == pytest.approx(oloss, rel=1e-4)
    gb, ob = _blocks(g), _blocks(og)
    for name in gb:
        err = np.linalg.norm(gb[name] - ob[name]) / max(np.linalg.norm(ob[name]), 1e-30)
        assert err <= 1e-3, (name, err)


def test_sixty_four_members(cx):
    # the largest ensemble: every member's forward equals its own one-member network
    thetas = np.stack([_theta(100 + k) for k in range(64)])
    x = np.random.default_rng(2).uniform(-1, 1, (200, 4)).astype(np.float32)
    with cx.Mlp(256, thetas, members=64) as net:
        assert cx.lib().cx_mlp_members(net.h) == 64
        y = net.forward(x)
    for k in (0, 1, 37, 63):
        with cx.Mlp(256, thetas[k]) as one:
            assert np.array_equal(one.forward(x), y[k])


def test_forward_at_the_screens_batch_matches_oracle(cx):
    # the screen evaluates candidates 8192 at a time: 64 row tiles per member
    thetas = [_theta(20 + k) for k in range(2)]
    x = np.random.default_rng(7).uniform(-1, 1, (8192, 4)).astype(np.float32)
    with cx.Mlp(8192, np.stack(thetas), members=2) as net:
        y = net.forward(x)
    for k in range(2):
        oy, _ = omlp.forward(thetas[k].astype(np.float64), x.astype(np.float64), rounding=True)
        assert np.linalg.norm(y[k] - oy) <= 1e-4 * np.linalg.norm(oy)
        assert np.max(np.abs(y[k] - oy)) <= 1e-3 * np.max(np.abs(oy))


def test_tensor_core_wait_timeout_is_reported(cx, monkeypatch):
    # failure detection without a GPU fault: a wait limit of 0 makes every
    # tile's first completion wait give up at once; the tile then waits
    # (bounded) for its products, releases its tensor memory and returns,
    # and the host reports CX_ERR_TIMEOUT
    theta = _theta(5)
    x = np.random.default_rng(0).uniform(-1, 1, (300, 4)).astype(np.float32)
    monkeypatch.setenv("CX_MMA_WAIT_LIMIT", "0")
    with cx.Mlp(512, theta) as net:
        with pytest.raises(cx.CxError) as e:
            net.forward(x)
        assert e.value.code == cx.CX_ERR_TIMEOUT
    monkeypatch.delenv("CX_MMA_WAIT_LIMIT")
    with cx.Mlp(512, theta) as net:                # the device still works
        y = net.forward(x)
    oy, _ = omlp.forward(theta.astype(np.float64), x.astype(np.float64), rounding=True)
    assert np.linalg.norm(y - oy) <= 1e-4 * np.linalg.norm(oy)


def test_training_fits_a_smooth_map(cx):
    rng = np.random.default_rng(0)
    X = rng.uniform(-1, 1, (4096, 4)).astype(np.float32)
    T = np.stack([np.sin(2 * X[:, 0]) + X[:, 1] * X[:, 2], np.cos(X[:, 3]) - X[:, 0] ** 2], 1)
    T = T.astype(np.float32)
    from paper_1301_5058_gb300 import surrogate
    with cx.Mlp(4096, surrogate.init_params(1)) as net:
        losses = net.train(X, T, 256, 3000, 2e-3)
        y = net.forward(X)
    assert losses[-20:].mean() < 0.02 * losses[:5].mean()
    assert np.sqrt(((y - T) ** 2).mean()) < 0.05


@pytest.mark.parametrize("prec", [0, 1])
def test_polar_profile_matches_oracle(cx, prec):
    cfg = dict(W.CONFIG0, nx=150, ny=120, chi0=1.0)
    grid, params, seed = W.split(cfg)
    with cx.Sim(150, 120, 0.7, seed=seed, **dict(params, precision=prec)) as sim:
        sim.step(600)
        b = sim.field(cx.CX_FIELD_B)
        r = 0.8 * sim.diagnostics()["r_env"]
        prof = cx.cx_polar_profile(sim.h, r, 4096)
        edge = cx.cx_polar_profile(sim.h, 200.0, 256)   # far outside: clamped to the walls
    ref = omlp.polar_profile(b, 0.7, r, 4096)
    assert np.max(np.abs(prof - ref)) <= 1e-12 * max(1.0, np.abs(ref).max())
    assert np.max(np.abs(edge - omlp.polar_profile(b, 0.7, 200.0, 256))) <= 1e-12


def test_batch_polar_profile_matches_single(cx):
    specs = [dict(nx=100, ny=90, dx=1.0, seed=3, n0=0.7, chi0=0.5, sigma0=4.0, noise_amp=0.5,
                  bM=0.5, r0sq=16.0, precision=1)]
    with cx.Batch(specs) as bt:
        bt.step(300)
        pb = cx.cx_batch_polar_profile(bt.h, 0, 9.5, 1000)
        b = bt.field(0, cx.CX_FIELD_B)
    assert np.max(np.abs(pb - omlp.polar_profile(b, 1.0, 9.5, 1000))) <= 1e-12


def test_validated_throughput_and_active_sweep_small(cx):
    from paper_1301_5058_gb300 import surrogate
    out = surrogate.validated_throughput(side=64, steps=400, n_train=128, n_test=64, members=2,
                                         agree=0.05, train_steps=300)
    assert out["batched_solver_points_per_hour"] > out["single_instance_points_per_hour"] > 0
    assert 0.0 <= out["accepted_fraction"] <= 1.0
    assert np.isfinite(out["heldout_rel_error_median_all"])
    assert out["campaign_points"] == 128 * 5 and out["campaign_points_per_hour"] > 0
    noise = surrogate.label_noise(side=64, steps=400, points=8, seeds=3)
    assert noise["moving_points"] <= 8 and 0.0 <= noise["runs_within_1pct_of_point_mean"] <= 1.0
    res = surrogate.active_sweep(rounds=2, per_round=16, first=32, pool=256, seed=1,
                                 label_kw=dict(side=64, steps=400, samples=8),
                                 train_kw=dict(steps=300, lr=2e-3, batch=32))
    assert len(res["points"]) == 32 + 2 * 16
    assert np.all(np.isfinite(res["labels"][:, 0]))
    assert len(res["history"]) == 2


def test_surrogate_end_to_end_small(cx):
    from paper_1301_5058_gb300 import surrogate
    pts = surrogate.draw_points(96, seed=5)
    v, br, last = surrogate.solver_labels(pts, side=96, steps=800, samples=16)
    assert np.all(np.isfinite(v)) and np.all(v >= 0)
    assert all(d["finite"] == 1 for d in last)
    model = surrogate.Surrogate(seed=2, max_batch=1024)
    losses = model.fit(pts, np.stack([v, br], 1), steps=1500, lr=2e-3, batch=96)
    pred = model.predict(pts)
    model.close()
    assert losses[-10:].mean() < 0.2 * losses[:5].mean()
    # the fit explains most of the velocity variance on its training points
    resid = ((pred[:, 0] - v) ** 2).mean() / max(v.var(), 1e-30)
    assert resid < 0.2


def test_network_gain_over_solver_only(cx):
    # What the trained network adds to the plain method: the ensemble answers
    # most held-out candidates without a solver run, at an error judged by the
    # solver (measured at this size: held-out median error 0.9 %, 96 %
    # accepted at 2 % agreement, 95th percentile error 4.3 %).
    from paper_1301_5058_gb300 import surrogate
    out = surrogate.validated_throughput(side=96, steps=3000, n_train=768, n_test=256, members=4,
                                         agree=0.02, train_steps=6000, decay=3)
    assert out["heldout_rel_error_median_all"] <= 0.02
    t = out["agreement_thresholds"]["0.02"]
    assert t["accepted"] >= 0.5 and t["p95_error"] <= 0.08
    # solver runs saved: points per hour grow by at least 1 / (1 - accepted)
    assert out["speedup_screened"] >= 2.0 * out["speedup_batched_solver_only"]


def test_validated_sweep_small(cx):
    # the validated-throughput measurement end to end on a small mix: every
    # figure present and consistent; the accepted points (if any) meet the
    # stated bar at the stated quantile on the evaluation half
    from paper_1301_5058_gb300 import surrogate
    out = surrogate.validated_sweep(train_side=128, sides=(96, 128), steps=600, n_train=256,
                                    n_test=128, members=2, train_steps=1500, decay=1,
                                    bar=0.05, campaign=1, samples=12)
    for k in ("single_instance_points_per_hour", "batched_points_per_hour",
              "screened_points_per_hour", "campaign_points_per_hour"):
        assert out[k] > 0
    assert 0.0 <= out["accepted_fraction"] <= 1.0
    batch_s = 3600.0 / out["batched_points_per_hour"]
    mixed_s = out["screen_seconds_per_point"] + (1 - out["accepted_fraction"]) * batch_s
    assert out["screened_points_per_hour"] == pytest.approx(3600.0 / mixed_s, rel=1e-9)
    if out["accepted_fraction"] > 0:
        assert out["accepted_error"]["0.5"] <= out["accepted_error"]["0.99"]
