"""Pins of the oracle's surrogate MLP and morphology labels."""

import numpy as np
import pytest

from oracle import mlp


def _theta(seed):
    rng = np.random.default_rng(seed)
    parts = {"W1": rng.normal(0, 0.5, (256, 4)), "b1": rng.normal(0, 0.1, 256),
             "W2": rng.normal(0, 1 / 16, (256, 256)), "b2": rng.normal(0, 0.1, 256),
             "W3": rng.normal(0, 1 / 16, (2, 256)), "b3": rng.normal(0, 0.1, 2)}
    return mlp.pack(parts)


def test_gradient_matches_central_differences():
    # without the bf16 rounding the loss is smooth: the backward pass must
    # equal its central differences
    theta = _theta(1)
    rng = np.random.default_rng(2)
    X = rng.normal(size=(7, 4))
    T = rng.normal(size=(7, 2))
    _, g = mlp.loss_and_grad(theta, X, T, rounding=False)
    idx = rng.choice(mlp.N_PARAMS, 60, replace=False)
    idx = np.concatenate([idx, [0, 1024, 1280 + 5, 1280 + 65536 + 3, mlp.N_PARAMS - 1]])
    h = 1e-6
    for i in idx:
        e = np.zeros_like(theta)
        e[i] = h
        fd = (mlp.loss_and_grad(theta + e, X, T, False)[0] -
              mlp.loss_and_grad(theta - e, X, T, False)[0]) / (2 * h)
        assert fd == pytest.approx(g[i], rel=1e-5, abs=1e-9), i


def test_bf16_rounding_agrees_with_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(3)
    x = np.concatenate([rng.normal(size=4000) * 10.0 ** rng.integers(-6, 6, 4000),
                        [0.0, -0.0, 1.0, 1.00390625, 1.01171875, 3.0e38]])
    ref = torch.tensor(x.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(mlp.bf16(x), ref)


def test_polar_profile_is_exact_on_linear_fields():
    ny, nx, dx = 60, 80, 0.5
    y, x = np.mgrid[0:ny, 0:nx]
    X = (x + 0.5 - nx / 2) * dx
    Y = (y + 0.5 - ny / 2) * dx
    b = 0.3 * X - 0.7 * Y + 2.0
    r = 9.3
    prof = mlp.polar_profile(b, dx, r, 360)
    ang = 2 * np.pi * np.arange(360) / 360
    assert np.allclose(prof, 0.3 * r * np.cos(ang) - 0.7 * r * np.sin(ang) + 2.0, atol=1e-12)


@pytest.mark.parametrize("k", [1, 3, 7, 12])
def test_branch_count_of_k_arm_field(k):
    n, dx = 201, 1.0
    y, x = np.mgrid[0:n, 0:n]
    X = x + 0.5 - n / 2
    Y = y + 0.5 - n / 2
    th = np.arctan2(Y, X) + 0.1
    b = (np.cos(k * th) > 0.2).astype(float)
    assert mlp.count_runs(mlp.polar_profile(b, dx, 60.0, 4096), 0.5) == k
    assert mlp.count_runs(np.ones(10), 0.5) == 0 and mlp.count_runs(np.zeros(10), 0.5) == 0


def test_velocity_fit_recovers_a_line():
    t = np.linspace(0, 50, 40)
    assert mlp.velocity_fit(t, 3.0 + 0.37 * t) == pytest.approx(0.37, rel=1e-13)
