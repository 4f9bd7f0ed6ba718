"""Staged uploads (cx_stage_state / cx_commit_state): a state uploaded
asynchronously and committed must equal the same state written with
cx_set_field, bit for bit, and a pipeline that stages the next state while the
current one steps must match the sequential run."""
import numpy as np
import pytest

from paper_1301_5058_gb300 import workloads as W

from _layout import natural

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cx():
    from paper_1301_5058_gb300 import _build
    _build.build()
    import paper_1301_5058_gb300 as cx
    return cx


def setup(cx, prec, nx=300, ny=77, seed=4):
    cfg = dict(W.CONFIG0, nx=nx, ny=ny, chi0=1.0, seed=seed)
    grid, params, seed = W.split(cfg)
    params["precision"] = prec
    npd = np.float64 if prec == cx.CX_PREC_F64 else np.float32
    return grid, params, seed, npd


def fields(sim, npd, cx):
    return sim.field(cx.CX_FIELD_B, npd), sim.field(cx.CX_FIELD_N, npd)


@pytest.mark.parametrize("prec", [0, 1])
def test_staged_state_equals_set_field(cx, prec):
    grid, params, seed, npd = setup(cx, prec)
    with cx.Sim(grid["nx"], grid["ny"], 1.0, seed=seed, **params) as a, \
            cx.Sim(grid["nx"], grid["ny"], 1.0, seed=seed, **params) as b, \
            cx.Sim(grid["nx"], grid["ny"], 1.0, seed=seed, **params) as c:
        a.step(25)
        fb, fn = fields(a, npd, cx)
        b.step(11)
        c.step(11)
        b.stage_state(fb, fn)
        b.step(3)                      # queued before the commit: acts on the old state
        b.commit_state()
        c.step(3)
        c.set_field(cx.CX_FIELD_B, fb)
        c.set_field(cx.CX_FIELD_N, fn)
        for x, y in zip(fields(b, npd, cx), fields(c, npd, cx)):
            assert np.array_equal(x, y)
        assert cx.cx_get_time(b.h)[0] == cx.cx_get_time(c.h)[0] == 14
        for s in (a, b):
            s.step(20)
        for x, y in zip(fields(a, npd, cx), fields(b, npd, cx)):
            assert np.array_equal(x, y)


@pytest.mark.parametrize("prec", [0, 1])
def test_staged_pipeline_matches_sequential_uploads(cx, prec):
    # every round uploads a different state from pinned memory while the
    # previous round steps; the staging arrays are reused every other round
    import torch
    grid, params, seed, npd = setup(cx, prec, nx=256, ny=96)
    tdt = torch.float64 if npd == np.float64 else torch.float32
    rounds = 5
    with cx.Sim(grid["nx"], grid["ny"], 1.0, seed=seed, **params) as src:
        states = []
        for _ in range(rounds):
            src.step(7)
            fb, fn = fields(src, npd, cx)
            states.append((torch.from_numpy(fb).pin_memory(), torch.from_numpy(fn).pin_memory()))
    with cx.Sim(grid["nx"], grid["ny"], 1.0, seed=seed, **params) as pipe, \
            cx.Sim(grid["nx"], grid["ny"], 1.0, seed=seed, **params) as seq:
        pipe.stage_state(*states[0])
        outs = []
        for k in range(rounds):
            pipe.commit_state()
            pipe.step(9)
            if k + 1 < rounds:
                pipe.stage_state(*states[k + 1])
            pipe.diagnostics()
            outs.append(fields(pipe, npd, cx))
        for k in range(rounds):
            seq.set_field(cx.CX_FIELD_B, states[k][0].numpy())
            seq.set_field(cx.CX_FIELD_N, states[k][1].numpy())
            seq.step(9)
            for x, y in zip(outs[k], fields(seq, npd, cx)):
                assert np.array_equal(x, y)
        assert all(t.dtype == tdt for t in states[0])


def test_staged_state_into_caller_buffers(cx):
    # caller-owned state arrays keep their addresses: the commit copies
    import torch
    nx, ny, pitch = 300, 77, 320
    grid, params, seed, npd = setup(cx, 1, nx=nx, ny=ny)
    b = torch.zeros((2, ny, pitch), dtype=torch.float32, device="cuda")
    n = torch.zeros((2, ny, pitch), dtype=torch.float32, device="cuda")
    s = torch.zeros((ny, pitch), dtype=torch.float32, device="cuda")
    g, p = cx.cx_grid(nx, ny, 1.0), cx.cx_params_default(**params)
    h = cx.cx_create_with_buffers(g, p, seed, [b[0].data_ptr(), b[1].data_ptr()],
                                  [n[0].data_ptr(), n[1].data_ptr()], s.data_ptr(), pitch)
    with cx.Sim(nx, ny, 1.0, seed=seed, handle=h, **params) as own, \
            cx.Sim(nx, ny, 1.0, seed=seed, **params) as ref:
        ref.step(30)
        fb, fn = fields(ref, npd, cx)
        own.stage_state(fb, fn)
        own.commit_state()
        cx.cx_synchronize(own.h)
        held = [natural(b[q], nx) for q in (0, 1)]
        assert any(np.array_equal(fb, x) for x in held)
        for sim in (own, ref):
            sim.step(10)
        for x, y in zip(fields(own, npd, cx), fields(ref, npd, cx)):
            assert np.array_equal(x, y)


def test_staged_state_rejects_misuse(cx):
    grid, params, seed, npd = setup(cx, 1, nx=64, ny=16)
    with cx.Sim(64, 16, 1.0, seed=seed, **params) as sim:
        fb, fn = fields(sim, npd, cx)
        for bad in (lambda: sim.commit_state(),                                  # nothing staged
                    lambda: sim.stage_state(fb.astype(np.float64), fn.astype(np.float64)),  # dtype
                    lambda: sim.stage_state(fb[:8], fn[:8])):                     # count
            with pytest.raises(cx.CxError) as e:
                bad()
            assert e.value.code == cx.CX_ERR_INVALID_ARG
        sim.stage_state(fb, fn)
        with pytest.raises(cx.CxError) as e:
            sim.stage_state(fb, fn)                                              # staged twice
        assert e.value.code == cx.CX_ERR_INVALID_ARG
        sim.commit_state()
        sim.step(2)
        assert sim.diagnostics()["finite"] == 1
