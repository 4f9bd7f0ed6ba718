"""cx_diagnostics_noalloc: the diagnostics reduction for callers that may not
allocate device memory themselves (for example a framework whose caching
allocator owns every device buffer, so that a stray cudaMalloc/cudaFree would
synchronise the device and fragment its pool).  The call keeps its scratch
in a static device array; the test owns every buffer it passes (allocated
here through PyTorch, playing the role of such a framework) and checks the
result against cx_diagnostics on a library handle, on two calls in a row.

This file is named so that pytest collects it last.
"""
import numpy as np
import pytest

from paper_1301_5058_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cx():
    from paper_1301_5058_gb300 import _build
    _build.build()
    import paper_1301_5058_gb300 as cx
    return cx


def _state(cx, nx, ny, prec, steps, seed):
    cfg = dict(W.CONFIG0, nx=nx, ny=ny, chi0=1.0, seed=seed)
    grid, params, s = W.split(cfg)
    sim = cx.Sim(nx, ny, 1.0, seed=s, **dict(params, precision=prec))
    sim.step(steps)
    ref = sim.diagnostics()
    dt = np.float64 if prec == cx.CX_PREC_F64 else np.float32
    b, n = sim.field(cx.CX_FIELD_B, dt), sim.field(cx.CX_FIELD_N, dt)
    sim.close()
    return ref, b, n


def _compare(d, ref):
    for k in ("mass_b", "mass_n", "invariant"):
        assert d[k] == pytest.approx(ref[k], rel=1e-13), k
    for k in ("min_b", "min_n", "max_b", "finite", "status"):
        assert d[k] == ref[k], k
    assert d["r_env"] == pytest.approx(ref["r_env"], rel=1e-14)
    assert d["area_env"] == ref["area_env"]


@pytest.mark.parametrize("prec", [0, 1])
def test_noalloc_matches_cx_diagnostics_on_two_calls_in_a_row(cx, prec):
    torch = pytest.importorskip("torch")
    dev = torch.device("cuda", torch.cuda.current_device())
    tdt = torch.float64 if prec == cx.CX_PREC_F64 else torch.float32
    stream = torch.cuda.current_stream(dev).cuda_stream
    result = torch.full((8,), float("nan"), dtype=torch.float64, device=dev)
    # a larger grid first (more partial records), then a smaller one: the
    # second call must not see the first call's records
    for nx, ny, steps, seed in ((700, 1500, 300, 1), (300, 200, 400, 2)):
        ref, b, n = _state(cx, nx, ny, prec, steps, seed)
        # pitched device copies owned by the caller (pitch > nx)
        pitch = nx + 13
        bd = torch.zeros((ny, pitch), dtype=tdt, device=dev)
        nd = torch.zeros((ny, pitch), dtype=tdt, device=dev)
        bd[:, :nx] = torch.from_numpy(b).to(dev)
        nd[:, :nx] = torch.from_numpy(n).to(dev)
        torch.cuda.synchronize()
        d = cx.cx_diagnostics_noalloc(bd.data_ptr(), nd.data_ptr(), nx, ny, pitch, prec, 1.0, 1.0,
                                      0.1 * W.CONFIG0["n0"], stream, result.data_ptr()).as_dict()
        _compare(d, ref)
        # the raw record in the caller's device buffer agrees with the host struct
        rec = result.cpu().numpy()
        assert rec[0] + rec[1] == pytest.approx(ref["invariant"], rel=1e-13)
        assert rec[2] == ref["min_b"] and rec[4] == ref["max_b"]


@pytest.mark.parametrize("prec", [0, 1])
def test_noalloc_calls_after_the_first_allocate_no_device_memory(cx, prec):
    # The property the entry point exists for: once the first call on the
    # device has set its scratch array up, further calls leave both the
    # caller's allocator and the device's free memory exactly as they were.
    torch = pytest.importorskip("torch")
    dev = torch.device("cuda", torch.cuda.current_device())
    tdt = torch.float64 if prec == cx.CX_PREC_F64 else torch.float32
    stream = torch.cuda.current_stream(dev).cuda_stream
    nx, ny = 1000, 777
    ref, b, n = _state(cx, nx, ny, prec, 200, 3)
    bd = torch.from_numpy(b).to(dev)
    nd = torch.from_numpy(n).to(dev)
    result = torch.zeros(8, dtype=torch.float64, device=dev)
    torch.cuda.synchronize()
    args = (bd.data_ptr(), nd.data_ptr(), nx, ny, nx, prec, 1.0, 1.0, 0.1 * W.CONFIG0["n0"], stream,
            result.data_ptr())
    cx.cx_diagnostics_noalloc(*args)  # warm-up: the first call may set the array up
    torch.cuda.synchronize()
    before = (torch.cuda.memory_allocated(dev), torch.cuda.mem_get_info(dev)[0])
    for _ in range(2):
        d = cx.cx_diagnostics_noalloc(*args).as_dict()
        _compare(d, ref)
    torch.cuda.synchronize()
    after = (torch.cuda.memory_allocated(dev), torch.cuda.mem_get_info(dev)[0])
    assert after == before


def test_noalloc_rejects_bad_sizes(cx):
    torch = pytest.importorskip("torch")
    dev = torch.device("cuda", torch.cuda.current_device())
    buf = torch.zeros(64, dtype=torch.float64, device=dev)
    p = buf.data_ptr()
    # the last case: wider than 2^26 columns, where the squared envelope radius
    # in record slot 5 would no longer be exact
    for nx, ny, pitch in ((0, 4, 4), (4, 0, 4), (8, 4, 7), (70000, 70000, 70000), (1, 3000000, 1),
                          ((1 << 26) + 1, 1, (1 << 26) + 1)):
        with pytest.raises(cx.CxError) as e:
            cx.cx_diagnostics_noalloc(p, p, nx, ny, pitch, 0, 1.0, 1.0, 0.1, None, p)
        assert e.value.code == cx.CX_ERR_INVALID_ARG
        assert "cx_diagnostics_noalloc" in cx.cx_last_error()
