"""Python binding of libcx.so, the GB300 time-stepper for the bacteria /
nutrient chemotaxis system with degenerate cross diffusion (Leyva, Malaga &
Plaza, Eq. ka-chem-model).

This module only marshals arguments: every step of the method runs in the
library's CUDA kernels.  The functions keep the C names of include/cx.h and
raise ``CxError`` on a non-zero status.  ``Sim`` is a small convenience
wrapper over one handle.  There is no CPU fallback: if libcx.so is missing,
importing the binding's functions raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libcx.so")

# status codes, field selectors and options (include/cx.h)
CX_OK = 0
CX_ERR_INVALID_ARG = -1
CX_ERR_DT_UNSTABLE = -2
CX_ERR_OOM = -3
CX_ERR_CUDA = -4
CX_ERR_NONFINITE = -5
CX_ERR_NEGATIVE = -6
CX_ERR_TIMEOUT = -7
CX_ERR_IO = -8
CX_ERR_UNSUPPORTED = -9
CX_FIELD_B, CX_FIELD_N, CX_FIELD_SIGMA = 0, 1, 2
CX_F64, CX_F32 = 0, 1
CX_CHEMO_RECEPTOR, CX_CHEMO_CONSTANT = 0, 1
CX_MOBILITY_CENTRAL, CX_MOBILITY_UPWIND = 0, 1
CX_NOISE_UNIFORM, CX_NOISE_TRIANGULAR = 0, 1
CX_NOISE_STATIC, CX_NOISE_PER_STEP = 0, 1
CX_SCHEME_EULER, CX_SCHEME_HEUN = 0, 1
CX_PREC_F64, CX_PREC_F32 = 0, 1


class cx_grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("dx", ctypes.c_double)]


class cx_params(ctypes.Structure):
    _fields_ = [(k, ctypes.c_double) for k in
                ("n0", "chi0", "sigma0", "noise_amp", "Dn", "theta", "bM", "r0sq", "dt",
                 "cfl_frac", "b_threshold")] + \
               [(k, ctypes.c_int32) for k in
                ("chemo_law", "mobility", "noise_dist", "noise_mode", "scheme", "precision")]


class cx_diag(ctypes.Structure):
    _fields_ = [("step", ctypes.c_int64)] + \
               [(k, ctypes.c_double) for k in
                ("t", "dt", "mass_b", "mass_n", "invariant", "min_b", "min_n", "max_b", "r_env")] + \
               [("finite", ctypes.c_int32), ("status", ctypes.c_int32),
                ("area_env", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class CxError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{msg} (status {code})")
        self.code = code


# every entry point of include/cx.h with its ctypes signature
_P = ctypes.c_void_p
_SIGNATURES = {
    "cx_version": (ctypes.c_int, []),
    "cx_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "cx_last_error": (ctypes.c_char_p, []),
    "cx_params_default": (ctypes.c_int, [ctypes.POINTER(cx_params)]),
    "cx_dt_limit": (ctypes.c_int, [ctypes.POINTER(cx_grid), ctypes.POINTER(cx_params),
                                   ctypes.POINTER(ctypes.c_double)]),
    "cx_create": (ctypes.c_int, [ctypes.POINTER(cx_grid), ctypes.POINTER(cx_params),
                                 ctypes.c_uint64, ctypes.POINTER(_P)]),
    "cx_create_with_buffers": (ctypes.c_int, [ctypes.POINTER(cx_grid), ctypes.POINTER(cx_params),
                                               ctypes.c_uint64, ctypes.POINTER(_P),
                                               ctypes.POINTER(_P), _P, ctypes.c_int64,
                                               ctypes.POINTER(_P)]),
    "cx_set_stream": (ctypes.c_int, [_P, _P]),
    "cx_step": (ctypes.c_int, [_P, ctypes.c_int64]),
    "cx_synchronize": (ctypes.c_int, [_P]),
    "cx_diagnostics": (ctypes.c_int, [_P, ctypes.POINTER(cx_diag)]),
    "cx_get_field": (ctypes.c_int, [_P, ctypes.c_int32, _P, ctypes.c_int32, ctypes.c_size_t]),
    "cx_set_field": (ctypes.c_int, [_P, ctypes.c_int32, _P, ctypes.c_int32, ctypes.c_size_t]),
    "cx_stage_state": (ctypes.c_int, [_P, _P, _P, ctypes.c_int32, ctypes.c_size_t]),
    "cx_commit_state": (ctypes.c_int, [_P]),
    "cx_get_config": (ctypes.c_int, [_P, ctypes.POINTER(cx_grid), ctypes.POINTER(cx_params),
                                     ctypes.POINTER(ctypes.c_uint64)]),
    "cx_get_time": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int64),
                                   ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]),
    "cx_set_step": (ctypes.c_int, [_P, ctypes.c_int64]),
    "cx_save": (ctypes.c_int, [_P, ctypes.c_char_p]),
    "cx_load": (ctypes.c_int, [ctypes.c_char_p, ctypes.POINTER(_P)]),
    "cx_destroy": (None, [_P]),
    "cx_set_tile_rows": (ctypes.c_int, [_P, ctypes.c_int32]),
    "cx_get_tile_rows": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int32)]),
    "cx_set_time_block": (ctypes.c_int, [_P, ctypes.c_int32]),
    "cx_batch_set_time_block": (ctypes.c_int, [_P, ctypes.c_int32]),
    "cx_batch_get_time_block": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int32)]),
    "cx_get_time_block": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int32)]),
    "cx_batch_create": (ctypes.c_int, [ctypes.c_int32, ctypes.POINTER(cx_grid),
                                       ctypes.POINTER(cx_params), ctypes.POINTER(ctypes.c_uint64),
                                       ctypes.POINTER(_P)]),
    "cx_batch_set_stream": (ctypes.c_int, [_P, _P]),
    "cx_batch_set_tuning": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int64,
                                           ctypes.c_int32]),
    "cx_batch_get_tuning": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int32),
                                           ctypes.POINTER(ctypes.c_int32),
                                           ctypes.POINTER(ctypes.c_int64),
                                           ctypes.POINTER(ctypes.c_int32)]),
    "cx_batch_step": (ctypes.c_int, [_P, ctypes.c_int64]),
    "cx_batch_synchronize": (ctypes.c_int, [_P]),
    "cx_batch_diagnostics": (ctypes.c_int, [_P, ctypes.POINTER(cx_diag)]),
    "cx_batch_get_field": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_int32, _P, ctypes.c_int32,
                                          ctypes.c_size_t]),
    "cx_batch_set_field": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_int32, _P, ctypes.c_int32,
                                          ctypes.c_size_t]),
    "cx_batch_get_time": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int32),
                                         ctypes.POINTER(ctypes.c_int64)]),
    "cx_batch_destroy": (None, [_P]),
    "cx_polar_profile": (ctypes.c_int, [_P, ctypes.c_double, ctypes.c_int32, _P]),
    "cx_batch_polar_profile": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_double, ctypes.c_int32,
                                              _P]),
    "cx_mlp_create": (ctypes.c_int, [ctypes.c_int32, ctypes.POINTER(_P)]),
    "cx_mlp_create_members": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(_P)]),
    "cx_mlp_members": (ctypes.c_int32, [_P]),
    "cx_mlp_set_params": (ctypes.c_int, [_P, _P, ctypes.c_size_t]),
    "cx_mlp_get_params": (ctypes.c_int, [_P, _P, ctypes.c_size_t]),
    "cx_mlp_forward": (ctypes.c_int, [_P, _P, ctypes.c_int32, _P]),
    "cx_mlp_gradient": (ctypes.c_int, [_P, _P, _P, ctypes.c_int32, _P, _P]),
    "cx_mlp_train": (ctypes.c_int, [_P, _P, _P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                    ctypes.c_float, _P]),
    "cx_mlp_destroy": (None, [_P]),
    "cx_diagnostics_noalloc": (ctypes.c_int, [_P, _P, ctypes.c_int32, ctypes.c_int32,
                                              ctypes.c_int64, ctypes.c_int32, ctypes.c_double,
                                              ctypes.c_double, ctypes.c_double, _P, _P,
                                              ctypes.POINTER(cx_diag)]),
    "cx_alu_peak": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32,
                                   ctypes.POINTER(ctypes.c_double)]),
}

_lib = None


def lib():
    """Load libcx.so (raises if it has not been built: there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing; build it with "
                          "paper_1301_5058_gb300._build.build() (needs nvcc)")
    L = ctypes.CDLL(LIB_PATH)
    for name, (res, args) in _SIGNATURES.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def _check(rc):
    if rc != CX_OK:
        raise CxError(rc, lib().cx_last_error().decode() or lib().cx_strerror(rc).decode())
    return rc


# ---- thin wrappers with the C names ------------------------------------------

def cx_version() -> int:
    return lib().cx_version()


def cx_strerror(code: int) -> str:
    return lib().cx_strerror(code).decode()


def cx_last_error() -> str:
    return lib().cx_last_error().decode()


def cx_params_default(**overrides) -> cx_params:
    p = cx_params()
    _check(lib().cx_params_default(ctypes.byref(p)))
    for k, v in overrides.items():
        if not hasattr(p, k):
            raise AttributeError(f"cx_params has no field {k}")
        setattr(p, k, v)
    return p


def cx_dt_limit(grid: cx_grid, params: cx_params) -> float:
    v = ctypes.c_double()
    _check(lib().cx_dt_limit(ctypes.byref(grid), ctypes.byref(params), ctypes.byref(v)))
    return v.value


def cx_create(grid: cx_grid, params: cx_params, seed: int) -> int:
    h = _P()
    _check(lib().cx_create(ctypes.byref(grid), ctypes.byref(params), seed, ctypes.byref(h)))
    return h.value


def cx_create_with_buffers(grid: cx_grid, params: cx_params, seed: int, b, n, sigma,
                           pitch: int) -> int:
    """b, n: two device addresses each (the ping-pong state); sigma: one;
    every array ny rows of `pitch` elements, owned by the caller."""
    bb = (_P * 2)(*[int(x) for x in b])
    nn = (_P * 2)(*[int(x) for x in n])
    h = _P()
    _check(lib().cx_create_with_buffers(ctypes.byref(grid), ctypes.byref(params), seed, bb, nn,
                                        _P(int(sigma)), pitch, ctypes.byref(h)))
    return h.value


def cx_set_stream(h, stream: int):
    _check(lib().cx_set_stream(h, stream))


def cx_step(h, n_steps: int):
    _check(lib().cx_step(h, n_steps))


def cx_synchronize(h):
    _check(lib().cx_synchronize(h))


def cx_diagnostics(h, check: bool = True) -> cx_diag:
    d = cx_diag()
    rc = lib().cx_diagnostics(h, ctypes.byref(d))
    if check:
        _check(rc)
    elif rc not in (CX_OK, CX_ERR_NONFINITE, CX_ERR_NEGATIVE):
        _check(rc)
    return d


def _host_view(arr: np.ndarray):
    if arr.dtype == np.float64:
        return CX_F64
    if arr.dtype == np.float32:
        return CX_F32
    raise TypeError("host arrays must be float64 or float32")


def cx_get_field(h, which: int, out: np.ndarray) -> np.ndarray:
    """Copy a field into the C-contiguous host array `out` (float64/float32)."""
    if not out.flags["C_CONTIGUOUS"]:
        raise ValueError("out must be C-contiguous")
    _check(lib().cx_get_field(h, which, out.ctypes.data, _host_view(out), out.size))
    return out


def cx_set_field(h, which: int, src: np.ndarray):
    src = np.ascontiguousarray(src)
    _check(lib().cx_set_field(h, which, src.ctypes.data, _host_view(src), src.size))


def _host_buffer(a):
    """(address, CX_F32/CX_F64, elements) of a C-contiguous host array: a
    numpy array or a CPU torch tensor (pinned, for copies that overlap queued
    work)."""
    if hasattr(a, "data_ptr"):
        if a.device.type != "cpu" or not a.is_contiguous():
            raise ValueError("host tensors must be contiguous CPU tensors")
        kind = {4: CX_F32, 8: CX_F64}.get(a.element_size()) if a.is_floating_point() else None
        if kind is None:
            raise TypeError("host arrays must be float64 or float32")
        return a.data_ptr(), kind, a.numel()
    if not a.flags["C_CONTIGUOUS"]:
        raise ValueError("host arrays must be C-contiguous")
    return a.ctypes.data, _host_view(a), a.size


def cx_stage_state(h, b, n):
    """Start asynchronous uploads of b and n (host arrays of the state's
    type) into the handle's staging arrays; cx_commit_state makes them the
    current state.  Both arrays must stay alive and unchanged until that
    commit has been followed by a synchronising call."""
    pb, kb, cb = _host_buffer(b)
    pn, kn, cn = _host_buffer(n)
    if kb != kn or cb != cn:
        raise ValueError("b and n must have the same type and size")
    _check(lib().cx_stage_state(h, pb, pn, kb, cb))


def cx_commit_state(h):
    _check(lib().cx_commit_state(h))


def cx_get_config(h):
    g, p, seed = cx_grid(), cx_params(), ctypes.c_uint64()
    _check(lib().cx_get_config(h, ctypes.byref(g), ctypes.byref(p), ctypes.byref(seed)))
    return g, p, seed.value


def cx_get_time(h):
    s, t, dt = ctypes.c_int64(), ctypes.c_double(), ctypes.c_double()
    _check(lib().cx_get_time(h, ctypes.byref(s), ctypes.byref(t), ctypes.byref(dt)))
    return s.value, t.value, dt.value


def cx_set_step(h, step: int):
    _check(lib().cx_set_step(h, step))


def cx_set_tile_rows(h, rows: int):
    _check(lib().cx_set_tile_rows(h, rows))


def cx_get_tile_rows(h) -> int:
    r = ctypes.c_int32()
    _check(lib().cx_get_tile_rows(h, ctypes.byref(r)))
    return r.value


def cx_set_time_block(h, stages: int):
    _check(lib().cx_set_time_block(h, stages))


def cx_get_time_block(h) -> int:
    r = ctypes.c_int32()
    _check(lib().cx_get_time_block(h, ctypes.byref(r)))
    return r.value


def cx_batch_set_time_block(h, stages: int):
    _check(lib().cx_batch_set_time_block(h, stages))


def cx_batch_get_time_block(h) -> int:
    r = ctypes.c_int32()
    _check(lib().cx_batch_get_time_block(h, ctypes.byref(r)))
    return r.value


def cx_batch_create(grids, params, seeds) -> int:
    n = len(grids)
    if not (len(params) == len(seeds) == n):
        raise ValueError("grids, params and seeds must have the same length")
    G = (cx_grid * n)(*grids)
    Pm = (cx_params * n)(*params)
    S = (ctypes.c_uint64 * n)(*[int(s) for s in seeds])
    h = _P()
    _check(lib().cx_batch_create(n, G, Pm, S, ctypes.byref(h)))
    return h.value


def cx_batch_set_stream(h, stream: int):
    _check(lib().cx_batch_set_stream(h, stream))


def cx_batch_set_tuning(h, tile_rows: int, graph_steps: int, group_bytes: int,
                        resident_steps: int = 0):
    _check(lib().cx_batch_set_tuning(h, tile_rows, graph_steps, group_bytes, resident_steps))


def cx_batch_get_tuning(h):
    r, g, b, s = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int64(), ctypes.c_int32()
    _check(lib().cx_batch_get_tuning(h, ctypes.byref(r), ctypes.byref(g), ctypes.byref(b),
                                     ctypes.byref(s)))
    return r.value, g.value, b.value, s.value


def cx_batch_step(h, n_steps: int):
    _check(lib().cx_batch_step(h, n_steps))


def cx_batch_synchronize(h):
    _check(lib().cx_batch_synchronize(h))


def cx_batch_get_time(h):
    c, s = ctypes.c_int32(), ctypes.c_int64()
    _check(lib().cx_batch_get_time(h, ctypes.byref(c), ctypes.byref(s)))
    return c.value, s.value


def cx_batch_diagnostics(h, check: bool = True):
    count, _ = cx_batch_get_time(h)
    out = (cx_diag * count)()
    rc = lib().cx_batch_diagnostics(h, out)
    if check or rc not in (CX_OK, CX_ERR_NONFINITE, CX_ERR_NEGATIVE):
        _check(rc)
    return [d.as_dict() for d in out]


def cx_batch_get_field(h, index: int, which: int, out: np.ndarray) -> np.ndarray:
    if not out.flags["C_CONTIGUOUS"]:
        raise ValueError("out must be C-contiguous")
    _check(lib().cx_batch_get_field(h, index, which, out.ctypes.data, _host_view(out), out.size))
    return out


def cx_batch_set_field(h, index: int, which: int, src: np.ndarray):
    src = np.ascontiguousarray(src)
    _check(lib().cx_batch_set_field(h, index, which, src.ctypes.data, _host_view(src), src.size))


def cx_batch_destroy(h):
    if h:
        lib().cx_batch_destroy(h)


def cx_polar_profile(h, radius: float, nsamples: int) -> np.ndarray:
    out = np.empty(nsamples, np.float64)
    _check(lib().cx_polar_profile(h, radius, nsamples, out.ctypes.data))
    return out


def cx_batch_polar_profile(h, index: int, radius: float, nsamples: int) -> np.ndarray:
    out = np.empty(nsamples, np.float64)
    _check(lib().cx_batch_polar_profile(h, index, radius, nsamples, out.ctypes.data))
    return out


CX_MLP_PARAMS = 67586


def _f32(a, cols):
    a = np.ascontiguousarray(a, np.float32)
    if a.ndim != 2 or a.shape[1] != cols:
        raise ValueError(f"expected an (n, {cols}) array")
    return a


class Mlp:
    """The surrogate network (include/cx.h, cx_mlp_*): `members` independent
    networks trained and evaluated together.  With one member the arrays
    have no member axis."""

    def __init__(self, max_batch: int, params=None, members: int = 1):
        h = _P()
        _check(lib().cx_mlp_create_members(max_batch, members, ctypes.byref(h)))
        self.h = h.value
        self.members = members
        if params is not None:
            self.set_params(params)

    def _squeeze(self, a):
        return a[0] if self.members == 1 else a

    def set_params(self, theta):
        theta = np.ascontiguousarray(theta, np.float32).reshape(-1)
        _check(lib().cx_mlp_set_params(self.h, theta.ctypes.data, theta.size))

    def params(self) -> np.ndarray:
        out = np.empty((self.members, CX_MLP_PARAMS), np.float32)
        _check(lib().cx_mlp_get_params(self.h, out.ctypes.data, out.size))
        return self._squeeze(out)

    def forward(self, x) -> np.ndarray:
        """(n, 2) outputs, or (members, n, 2); x (n, 4) is shared."""
        x = _f32(x, 4)
        y = np.empty((self.members, x.shape[0], 2), np.float32)
        _check(lib().cx_mlp_forward(self.h, x.ctypes.data, x.shape[0], y.ctypes.data))
        return self._squeeze(y)

    def gradient(self, x, t):
        """(loss, gradient) of every member on the shared batch (x, t)."""
        x, t = _f32(x, 4), _f32(t, 2)
        g = np.empty((self.members, CX_MLP_PARAMS), np.float32)
        loss = np.empty(self.members, np.float64)
        _check(lib().cx_mlp_gradient(self.h, x.ctypes.data, t.ctypes.data, x.shape[0],
                                     g.ctypes.data, loss.ctypes.data))
        return (float(loss[0]), g[0]) if self.members == 1 else (loss, g)

    def train(self, x, t, batch: int, steps: int, lr: float) -> np.ndarray:
        """x (n, 4) and t (n, 2), or one set per member ((members, n, 4) and
        (members, n, 2)); returns the step losses, (steps,) or (members, steps)."""
        x = np.ascontiguousarray(x, np.float32)
        t = np.ascontiguousarray(t, np.float32)
        if x.ndim == 2:
            x = np.broadcast_to(x, (self.members,) + x.shape).copy()
            t = np.broadcast_to(t, (self.members,) + t.shape).copy()
        if x.shape[0] != self.members or x.shape[2] != 4 or t.shape != x.shape[:2] + (2,):
            raise ValueError("expected (members, n, 4) inputs and (members, n, 2) targets")
        losses = np.empty((self.members, steps), np.float64)
        _check(lib().cx_mlp_train(self.h, x.ctypes.data, t.ctypes.data, x.shape[1], batch, steps,
                                  lr, losses.ctypes.data))
        return self._squeeze(losses)

    def close(self):
        if getattr(self, "h", None):
            lib().cx_mlp_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def cx_save(h, path: str):
    _check(lib().cx_save(h, os.fsencode(path)))


def cx_load(path: str) -> int:
    h = _P()
    _check(lib().cx_load(os.fsencode(path), ctypes.byref(h)))
    return h.value


def cx_destroy(h):
    if h:
        lib().cx_destroy(h)


def cx_diagnostics_noalloc(b_ptr, n_ptr, nx, ny, pitch, precision, dx, theta, b_threshold,
                           stream, result_ptr, want_host=True):
    """Diagnostics over caller-owned device fields (raw device pointers),
    with no allocation by the library; returns a cx_diag when want_host,
    else None after queueing the work on `stream`."""
    d = cx_diag() if want_host else None
    rc = lib().cx_diagnostics_noalloc(b_ptr, n_ptr, nx, ny, pitch, precision, dx, theta,
                                      b_threshold, stream, result_ptr,
                                      ctypes.byref(d) if want_host else None)
    if rc not in (CX_OK, CX_ERR_NONFINITE, CX_ERR_NEGATIVE) or not want_host:
        _check(rc)
    return d


def cx_alu_peak(precision, repeats=5) -> float:
    """Measured multiply-add rate (FLOP/s, a multiply-add counting two) of
    the current device in CX_PREC_F64 or CX_PREC_F32."""
    v = ctypes.c_double()
    _check(lib().cx_alu_peak(precision, repeats, ctypes.byref(v)))
    return v.value


# ---- convenience wrapper -----------------------------------------------------

class Sim:
    """One simulation handle.  ``Sim(nx, ny, dx=1.0, seed=0, **params)``."""

    def __init__(self, nx, ny, dx=1.0, seed=0, handle=None, **params):
        self.grid = cx_grid(nx, ny, dx)
        self.params = cx_params_default(**params)
        self.h = handle if handle is not None else cx_create(self.grid, self.params, seed)

    @classmethod
    def load(cls, path):
        h = cx_load(path)
        obj = cls.__new__(cls)
        obj.h = h
        obj.grid, obj.params, _ = cx_get_config(h)
        return obj

    def step(self, n):
        cx_step(self.h, n)

    def diagnostics(self, check=True) -> dict:
        return cx_diagnostics(self.h, check=check).as_dict()

    def field(self, which, dtype=np.float64):
        ny, nx = self.shape
        return cx_get_field(self.h, which, np.empty((ny, nx), dtype))

    def set_field(self, which, arr):
        cx_set_field(self.h, which, arr)

    def stage_state(self, b, n):
        cx_stage_state(self.h, b, n)

    def commit_state(self):
        cx_commit_state(self.h)

    @property
    def shape(self):
        return (self.grid.ny, self.grid.nx)

    def close(self):
        if getattr(self, "h", None):
            cx_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Many independent simulations stepped together.  ``specs`` is a list of
    dicts with keys nx, ny, dx, seed and any cx_params field."""

    def __init__(self, specs):
        self.grids = [cx_grid(s["nx"], s["ny"], s.get("dx", 1.0)) for s in specs]
        self.params = [cx_params_default(**{k: v for k, v in s.items()
                                            if k not in ("nx", "ny", "dx", "seed")}) for s in specs]
        self.h = cx_batch_create(self.grids, self.params, [s.get("seed", 0) for s in specs])

    def __len__(self):
        return len(self.grids)

    def step(self, n):
        cx_batch_step(self.h, n)

    def diagnostics(self, check=True):
        return cx_batch_diagnostics(self.h, check=check)

    def field(self, index, which, dtype=np.float64):
        g = self.grids[index]
        return cx_batch_get_field(self.h, index, which, np.empty((g.ny, g.nx), dtype))

    def set_field(self, index, which, arr):
        cx_batch_set_field(self.h, index, which, arr)

    def tune(self, tile_rows, graph_steps, group_bytes, resident_steps=0, time_block=None):
        cx_batch_set_tuning(self.h, tile_rows, graph_steps, group_bytes, resident_steps)
        if time_block is not None:
            cx_batch_set_time_block(self.h, time_block)

    def close(self):
        if getattr(self, "h", None):
            cx_batch_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
