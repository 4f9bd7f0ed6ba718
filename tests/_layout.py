"""The library's in-row order of device arrays, for tests that read a
caller-owned array directly: each aligned group of four cells of a row is
stored as (4g, 4g+2, 4g+1, 4g+3)."""
import numpy as np


def natural(t, nx):
    """The rows of device array t (a torch tensor, last axis = the row) in
    natural cell order, the first nx columns."""
    x = t.cpu().numpy().copy()
    w = (nx + 3) // 4 * 4
    g = x[..., :w].reshape(x.shape[:-1] + (w // 4, 4))
    g[..., [1, 2]] = g[..., [2, 1]]
    x[..., :w] = g.reshape(x.shape[:-1] + (w,))
    return x[..., :nx]
