"""Host-side checks of the C ABI that need no GPU: the library builds and
loads, exports every function that include/*.h declares, and rejects bad
arguments before touching the device."""
import glob
import os
import re

import numpy as np
import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def cx():
    from paper_1301_5058_gb300 import _build
    _build.build()
    import paper_1301_5058_gb300 as cx
    cx.lib()
    return cx


def declared_functions():
    names = set()
    pat = re.compile(r"^\s*(?:const\s+)?(?:int|void|double|int32_t|int64_t|size_t|char)\s*\*?\s*"
                     r"(cx_\w+)\s*\(", re.M)
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        names |= set(pat.findall(open(h).read()))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("cx_create", "cx_step", "cx_diagnostics", "cx_get_field", "cx_set_field",
                     "cx_destroy", "cx_save", "cx_load", "cx_set_stream"):
        assert required in names


def test_library_exports_every_declared_symbol(cx):
    L = cx.lib()
    missing = [n for n in declared_functions() if not hasattr(L, n)]
    assert not missing, missing


def test_binding_wraps_every_declared_symbol(cx):
    missing = [n for n in declared_functions() if n not in cx._SIGNATURES]
    assert not missing, missing


def test_version_and_strings(cx):
    assert cx.cx_version() >= 1
    assert cx.cx_strerror(cx.CX_ERR_DT_UNSTABLE).startswith("time step")
    assert cx.cx_strerror(12345) == "unknown status code"


def test_params_default_is_the_normalised_model(cx):
    p = cx.cx_params_default()
    assert (p.Dn, p.theta, p.precision, p.scheme) == (1.0, 1.0, cx.CX_PREC_F32, cx.CX_SCHEME_EULER)
    assert (p.bM, p.r0sq) == (0.71, 6.25)


@pytest.mark.parametrize("chi0,sigma0,amp,n0,bM,dx", [(0.5, 4.0, 0.5, 0.7, 0.5, 1.0),
                                                       (1.0, 4.0, 0.8, 0.35, 0.71, 1.0),
                                                       (5.0, 1.0, 1.0, 1.07, 0.71, 0.332),
                                                       # reaction branch 1/(4 Dn/dx^2 + B) = 1/17 decides
                                                       (0.0, 0.5, 0.0, 0.5, 0.5, 0.5)])
def test_dt_limit_matches_oracle(cx, chi0, sigma0, amp, n0, bM, dx):
    p = cx.cx_params_default(chi0=chi0, sigma0=sigma0, noise_amp=amp, n0=n0, bM=bM)
    lim = cx.cx_dt_limit(cx.cx_grid(8, 8, dx), p)
    ref = oracle.dt_limit(dx=dx, Dn=1.0, theta=1.0, chi0=chi0, n0=n0, bM=bM, sigma0=sigma0, amp=amp)
    assert lim == pytest.approx(ref, rel=1e-15)
    if dx == 0.5:
        assert lim == pytest.approx(1.0 / 17.0, rel=1e-15)


def test_config0_time_step(cx):
    # 256^2, sigma0 = 4, a = 0.5, n0 = 0.7, bM = 0.5, chi0 = 0.5 -> Dmax = 8.064
    p = cx.cx_params_default(chi0=0.5, sigma0=4.0, noise_amp=0.5, n0=0.7, bM=0.5, r0sq=16.0)
    assert 0.2 * cx.cx_dt_limit(cx.cx_grid(256, 256, 1.0), p) == pytest.approx(0.2 / (4 * 8.064), rel=1e-14)


BAD = [
    (dict(), dict(nx=0)),
    (dict(), dict(ny=-3)),
    (dict(), dict(dx=0.0)),
    (dict(), dict(dx=float("nan"))),
    (dict(n0=-1.0), dict()),
    (dict(chi0=float("inf")), dict()),
    (dict(noise_amp=1.5), dict()),
    (dict(r0sq=0.0), dict()),
    (dict(cfl_frac=0.0), dict()),
    (dict(cfl_frac=1.5), dict()),
    (dict(chemo_law=7), dict()),
    (dict(mobility=-1), dict()),
    (dict(noise_dist=2), dict()),
    (dict(noise_mode=3), dict()),
    (dict(scheme=9), dict()),
    (dict(precision=2), dict()),
    (dict(b_threshold=float("nan")), dict()),
]


@pytest.mark.parametrize("pover,gover", BAD)
def test_create_rejects_bad_arguments_before_any_device_call(cx, pover, gover):
    g = dict(nx=16, ny=16, dx=1.0)
    g.update(gover)
    p = cx.cx_params_default(**pover)
    with pytest.raises(cx.CxError) as e:
        cx.cx_create(cx.cx_grid(g["nx"], g["ny"], g["dx"]), p, 0)
    assert e.value.code == cx.CX_ERR_INVALID_ARG
    assert cx.cx_last_error()


def test_create_rejects_unstable_dt(cx):
    g = cx.cx_grid(16, 16, 1.0)
    p = cx.cx_params_default(sigma0=4.0)
    lim = cx.cx_dt_limit(g, p)
    p.dt = lim * 1.0001
    with pytest.raises(cx.CxError) as e:
        cx.cx_create(g, p, 0)
    assert e.value.code == cx.CX_ERR_DT_UNSTABLE
    assert "stability limit" in cx.cx_last_error()


def test_create_with_buffers_checks_pointers_before_device_work(cx):
    g = cx.cx_grid(64, 16, 1.0)
    p = cx.cx_params_default(sigma0=4.0)
    for b, n, s in (([0, 0], [0, 0], 0), ([16, 32], [48, 64], 0), ([17, 4096], [8192, 12288], 16384)):
        with pytest.raises(cx.CxError) as e:
            cx.cx_create_with_buffers(g, p, 0, b, n, s, 64)
        assert e.value.code == cx.CX_ERR_INVALID_ARG


def test_null_handles_are_rejected(cx):
    for f, args in ((cx.lib().cx_step, (None, 1)), (cx.lib().cx_synchronize, (None,)),
                    (cx.lib().cx_set_tile_rows, (None, 2)), (cx.lib().cx_set_step, (None, 0)),
                    (cx.lib().cx_set_time_block, (None, 2)), (cx.lib().cx_get_time_block, (None, None)),
                    (cx.lib().cx_stage_state, (None, None, None, cx.CX_F32, 0)),
                    (cx.lib().cx_commit_state, (None,))):
        assert f(*args) == cx.CX_ERR_INVALID_ARG
    cx.lib().cx_destroy(None)  # no-op


def test_load_rejects_missing_and_foreign_files(cx, tmp_path):
    with pytest.raises(cx.CxError) as e:
        cx.cx_load(str(tmp_path / "nope.ckpt"))
    assert e.value.code == cx.CX_ERR_IO
    bad = tmp_path / "bad.ckpt"
    bad.write_bytes(b"not a checkpoint at all" * 10)
    with pytest.raises(cx.CxError) as e:
        cx.cx_load(str(bad))
    assert e.value.code == cx.CX_ERR_IO


def test_binding_refuses_non_float_host_arrays(cx):
    with pytest.raises(TypeError):
        cx._host_view(np.zeros(4, np.int32))


def test_batch_create_validates_before_any_device_call(cx):
    g = [cx.cx_grid(16, 16, 1.0), cx.cx_grid(8, 8, 1.0)]
    p32 = cx.cx_params_default()
    p64 = cx.cx_params_default(precision=cx.CX_PREC_F64)
    with pytest.raises(cx.CxError) as e:
        cx.cx_batch_create(g, [p32, p64], [0, 1])
    assert e.value.code == cx.CX_ERR_INVALID_ARG
    with pytest.raises(cx.CxError) as e:
        cx.cx_batch_create(g, [p32, cx.cx_params_default(noise_amp=2.0)], [0, 1])
    assert e.value.code == cx.CX_ERR_INVALID_ARG
    # instances must share the noise mode (per-step noise itself is supported)
    ps = cx.cx_params_default(noise_mode=cx.CX_NOISE_PER_STEP)
    with pytest.raises(cx.CxError) as e:
        cx.cx_batch_create(g, [p32, ps], [0, 1])
    assert e.value.code == cx.CX_ERR_INVALID_ARG
    bad = cx.cx_params_default(dt=10.0)
    with pytest.raises(cx.CxError) as e:
        cx.cx_batch_create(g, [p32, bad], [0, 1])
    assert e.value.code == cx.CX_ERR_DT_UNSTABLE
    with pytest.raises(cx.CxError) as e:
        cx.cx_batch_create([], [], [])
    assert e.value.code == cx.CX_ERR_INVALID_ARG
    for f, args in ((cx.lib().cx_batch_step, (None, 1)), (cx.lib().cx_batch_synchronize, (None,)),
                    (cx.lib().cx_batch_set_tuning, (None, 32, 0, 0, 0))):
        assert f(*args) == cx.CX_ERR_INVALID_ARG
    cx.lib().cx_batch_destroy(None)


def test_network_create_and_calls_validate_before_any_device_call(cx):
    import ctypes
    L = cx.lib()
    h = ctypes.c_void_p()
    for max_batch, members in ((0, 1), (1 << 20 | 1, 1), (64, 0), (64, 65)):
        assert L.cx_mlp_create_members(max_batch, members, ctypes.byref(h)) == cx.CX_ERR_INVALID_ARG
        assert h.value is None
    assert L.cx_mlp_create(0, ctypes.byref(h)) == cx.CX_ERR_INVALID_ARG
    assert L.cx_mlp_create_members(64, 2, None) == cx.CX_ERR_INVALID_ARG
    assert L.cx_mlp_members(None) == 0
    buf = (ctypes.c_float * 8)()
    assert L.cx_mlp_forward(None, buf, 1, buf) == cx.CX_ERR_INVALID_ARG
    assert L.cx_mlp_gradient(None, buf, buf, 1, buf, None) == cx.CX_ERR_INVALID_ARG
    assert L.cx_mlp_train(None, buf, buf, 1, 1, 1, 1e-3, None) == cx.CX_ERR_INVALID_ARG
    assert L.cx_mlp_set_params(None, buf, 8) == cx.CX_ERR_INVALID_ARG
    assert L.cx_mlp_get_params(None, buf, 8) == cx.CX_ERR_INVALID_ARG
    L.cx_mlp_destroy(None)
