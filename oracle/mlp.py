"""FP64 reference of the surrogate MLP (4 -> 256 -> 256 -> 2, tanh) and of
the morphology labels, in plain numpy.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Forward, for a batch X (B x 4) and targets T (B x 2):
    Z1 = X W1^T + b1,  H1 = tanh(Z1)
    Z2 = bf(H1) bf(W2)^T + b2,  H2 = tanh(Z2)
    Y  = H2 W3^T + b3
    loss = sum((Y - T)^2) / (2 B)
where bf() rounds to bfloat16 (round to nearest even): the 256 x 256 layer
runs on bf16 operands with wide accumulation, the two thin layers in full
precision.  Backward (chain rule, written out):
    dY = (Y - T) / B;  dW3 = dY^T H2;  db3 = sum_b dY
    dZ2 = (dY W3) * (1 - H2^2);  db2 = sum_b dZ2
    dW2 = bf(dZ2)^T bf(H1);  dH1 = bf(dZ2) bf(W2)
    dZ1 = dH1 * (1 - H1^2);  dW1 = dZ1^T X;  db1 = sum_b dZ1
Parameters are packed flat as W1 (256x4), b1, W2 (256x256), b2, W3 (2x256), b3.
"""
from __future__ import annotations

import numpy as np

HIDDEN = 256
N_IN = 4
N_OUT = 2
SHAPES = (("W1", (HIDDEN, N_IN)), ("b1", (HIDDEN,)), ("W2", (HIDDEN, HIDDEN)), ("b2", (HIDDEN,)),
          ("W3", (N_OUT, HIDDEN)), ("b3", (N_OUT,)))
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)


def unpack(theta):
    out, o = {}, 0
    for name, shape in SHAPES:
        k = int(np.prod(shape))
        out[name] = np.asarray(theta[o:o + k], np.float64).reshape(shape)
        o += k
    return out


def pack(parts):
    return np.concatenate([np.asarray(parts[name], np.float64).ravel() for name, _ in SHAPES])


def bf16(x):
    """Round to the nearest bfloat16 (ties to even), via float32."""
    f = np.ascontiguousarray(np.asarray(x, np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def forward(theta, X, rounding=True):
    p = unpack(theta)
    r = bf16 if rounding else (lambda a: np.asarray(a, np.float64))
    Z1 = X @ p["W1"].T + p["b1"]
    H1 = np.tanh(Z1)
    Z2 = r(H1) @ r(p["W2"]).T + p["b2"]
    H2 = np.tanh(Z2)
    Y = H2 @ p["W3"].T + p["b3"]
    return Y, (H1, H2)


def loss_and_grad(theta, X, T, rounding=True):
    X = np.asarray(X, np.float64)
    T = np.asarray(T, np.float64)
    B = X.shape[0]
    p = unpack(theta)
    r = bf16 if rounding else (lambda a: np.asarray(a, np.float64))
    Y, (H1, H2) = forward(theta, X, rounding)
    loss = float(((Y - T) ** 2).sum() / (2 * B))
    dY = (Y - T) / B
    g = {"W3": dY.T @ H2, "b3": dY.sum(0)}
    dZ2 = (dY @ p["W3"]) * (1 - H2 ** 2)
    g["b2"] = dZ2.sum(0)
    g["W2"] = r(dZ2).T @ r(H1)
    dH1 = r(dZ2) @ r(p["W2"])
    dZ1 = dH1 * (1 - H1 ** 2)
    g["W1"] = dZ1.T @ X
    g["b1"] = dZ1.sum(0)
    return loss, pack(g)


# ---------------------------------------------------------------------------
# Morphology labels

def polar_profile(b, dx, radius, nsamples):
    """b on the circle of the given radius about the domain centre, by
    bilinear interpolation of the cell-centred values (clamped at walls);
    sample k at angle 2 pi k / nsamples."""
    b = np.asarray(b, np.float64)
    ny, nx = b.shape
    ang = 2 * np.pi * np.arange(nsamples) / nsamples
    fx = radius * np.cos(ang) / dx + 0.5 * nx - 0.5
    fy = radius * np.sin(ang) / dx + 0.5 * ny - 0.5
    out = np.empty(nsamples)
    for k in range(nsamples):
        x = min(max(fx[k], 0.0), nx - 1.0)
        y = min(max(fy[k], 0.0), ny - 1.0)
        i0 = min(int(np.floor(x)), nx - 1)
        j0 = min(int(np.floor(y)), ny - 1)
        i1, j1 = min(i0 + 1, nx - 1), min(j0 + 1, ny - 1)
        wx, wy = x - i0, y - j0
        out[k] = ((1 - wy) * ((1 - wx) * b[j0, i0] + wx * b[j0, i1])
                  + wy * ((1 - wx) * b[j1, i0] + wx * b[j1, i1]))
    return out


def count_runs(profile, level):
    """Number of maximal circular runs of samples with value >= level (a full
    circle above the level counts as 0 branches: an unbroken disc)."""
    above = np.asarray(profile) >= level
    if above.all() or not above.any():
        return 0
    starts = above & ~np.roll(above, 1)
    return int(starts.sum())


def velocity_fit(t, r):
    """FP64 least-squares slope of r against t."""
    t = np.asarray(t, np.float64)
    r = np.asarray(r, np.float64)
    tm, rm = t.mean(), r.mean()
    return float(((t - tm) * (r - rm)).sum() / ((t - tm) ** 2).sum())
