"""Guard bands around caller-owned fields: the step kernels write only the
nx x ny cells of each array, and what lies beside them (the padding columns
of each row, and memory before and after each array) never reaches a
result.  The arrays are filled with NaN outside the grid; after the steps
that NaN must still be there, untouched, and the fields must equal, bit for
bit, a run over library-owned arrays (whose padding holds zeros)."""
import numpy as np
import pytest

from paper_1301_5058_gb300 import workloads as W

pytestmark = pytest.mark.gpu

GUARD = 4096  # elements before and after each array


@pytest.fixture(scope="module")
def cx():
    from paper_1301_5058_gb300 import _build
    _build.build()
    import paper_1301_5058_gb300 as cx
    return cx


@pytest.mark.parametrize("prec,time_block,scheme,noise", [
    (1, 2, 0, 0), (1, 1, 0, 0), (1, 2, 1, 1), (1, 2, 0, 1), (0, 1, 0, 0), (0, 2, 1, 0)])
def test_kernels_write_only_inside_the_grid(cx, prec, time_block, scheme, noise):
    torch = pytest.importorskip("torch")
    dev = torch.device("cuda", torch.cuda.current_device())
    tdt = torch.float32 if prec == cx.CX_PREC_F32 else torch.float64
    elem = 4 if prec == cx.CX_PREC_F32 else 8
    nx, ny = 1000, 77                      # ragged against every tile width
    pitch = (nx * elem + 127) // 128 * 128 // elem + 32  # rows 128-byte aligned, 32 padding columns
    cfg = dict(W.CONFIG0, nx=nx, ny=ny, chi0=1.0)
    grid, params, seed = W.split(cfg)
    params = dict(params, precision=prec, scheme=scheme, noise_mode=noise, noise_dist=1)
    bufs = [torch.full((2 * GUARD + ny * pitch,), float("nan"), dtype=tdt, device=dev)
            for _ in range(5)]
    ptr = [t.data_ptr() + GUARD * elem for t in bufs]
    g = cx.cx_grid(nx, ny, 1.0)
    h = cx.cx_create_with_buffers(g, cx.cx_params_default(**params), seed, ptr[0:2], ptr[2:4],
                                  ptr[4], pitch)
    try:
        cx.cx_set_time_block(h, time_block)
        torch.cuda.synchronize()
        for t in bufs:  # NaN in every row's padding columns, after the initialisation
            t[GUARD:GUARD + ny * pitch].view(ny, pitch)[:, nx:] = float("nan")
        torch.cuda.synchronize()
        cx.cx_step(h, 50)
        cx.cx_synchronize(h)
        dtype = np.float32 if prec == cx.CX_PREC_F32 else np.float64
        gb = cx.cx_get_field(h, cx.CX_FIELD_B, np.empty((ny, nx), dtype))
        gn = cx.cx_get_field(h, cx.CX_FIELD_N, np.empty((ny, nx), dtype))
    finally:
        cx.cx_destroy(h)
    for t in bufs:
        assert bool(torch.isnan(t[:GUARD]).all()) and bool(torch.isnan(t[-GUARD:]).all())
        assert bool(torch.isnan(t[GUARD:GUARD + ny * pitch].view(ny, pitch)[:, nx:]).all())
    assert np.isfinite(gb).all() and np.isfinite(gn).all()
    with cx.Sim(nx, ny, 1.0, seed=seed, **params) as sim:
        cx.cx_set_time_block(sim.h, time_block)
        sim.step(50)
        rb, rn = sim.field(cx.CX_FIELD_B, dtype), sim.field(cx.CX_FIELD_N, dtype)
    assert np.array_equal(gb, rb) and np.array_equal(gn, rn)
