"""FP64 CPU oracle for the nutrient-chemotaxis / degenerate cross-diffusion
system (Leyva, Malaga & Plaza, Eq. ka-chem-model and its general form
Eq. ka-model-dim).

TEST INFRASTRUCTURE ONLY: tests, the package smoke check and the benchmark's
CPU-baseline leg are the only callers.  The product path (the CUDA library
and its Python binding) never imports this package, and this package never
imports the product.

The arithmetic lives in ``cx_oracle.c`` (plain C, FP64, no fused
multiply-add); this module compiles it with gcc on first use and wraps it with
ctypes and numpy.  Arrays are row-major ``(ny, nx)`` float64.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cx_oracle.c")
_LIB_PATH = os.path.join(_HERE, "libcx_oracle.so")
_OMP_LIB_PATH = os.path.join(_HERE, "libcx_oracle_omp.so")
_lock = threading.Lock()
_lib = None
_omp_lib = None

_D = ctypes.c_double
_I = ctypes.c_int
_U64 = ctypes.c_uint64
_I64 = ctypes.c_int64
_PD = ctypes.POINTER(ctypes.c_double)
_PU32 = ctypes.POINTER(ctypes.c_uint32)


def build(force: bool = False, omp: bool = False) -> str:
    """Compile cx_oracle.c into libcx_oracle.so next to it (gcc, -O2,
    -ffp-contract=off so no multiply-add is fused on any host); with omp,
    the threaded build libcx_oracle_omp.so (-fopenmp: the row loop of the
    right-hand side and the update loops on several host threads, the same
    arithmetic per cell)."""
    path = _OMP_LIB_PATH if omp else _LIB_PATH
    with _lock:
        if (not force and os.path.exists(path)
                and os.path.getmtime(path) >= os.path.getmtime(_SRC)):
            return path
        tmp = path + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fno-fast-math",
               "-fPIC", "-shared"] + (["-fopenmp"] if omp else []) + ["-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, path)
        return path


def _load(omp: bool = False):
    global _lib, _omp_lib
    if omp and _omp_lib is not None:
        return _omp_lib
    if not omp and _lib is not None:
        return _lib
    lib = ctypes.CDLL(build(omp=omp))
    lib.orc_philox4x32_10.argtypes = [_PU32, _PU32, _PU32]
    lib.orc_philox4x32_10.restype = None
    lib.orc_noise_delta.argtypes = [_U64, _U64, _U64, _I]
    lib.orc_noise_delta.restype = _D
    lib.orc_sigma_field.argtypes = [_I, _I, _U64, _U64, _D, _D, _I, _PD]
    lib.orc_sigma_field.restype = None
    lib.orc_sigma_field_f32.argtypes = [_I, _I, _U64, _U64, _D, _D, _I, _PD]
    lib.orc_sigma_field_f32.restype = None
    lib.orc_initial_state.argtypes = [_I, _I, _D, _D, _D, _D, _PD, _PD]
    lib.orc_initial_state.restype = None
    lib.orc_rhs.argtypes = [_I, _I, _D, _D, _D, _D, _I, _I, _PD, _PD, _PD, _PD, _PD]
    lib.orc_rhs.restype = None
    for name in ("orc_step_euler", "orc_step_heun"):
        f = getattr(lib, name)
        f.argtypes = [_I, _I, _D, _D, _D, _D, _D, _I, _I, _PD, _PD, _PD, _PD, _PD]
        f.restype = _I
    lib.orc_run.argtypes = [_I, _I, _D, _D, _D, _D, _D, _I, _I, _I, _I, _I, _U64, _D, _D, _I,
                            _I64, _I64, _PD, _PD, _PD]
    lib.orc_run.restype = _I
    lib.orc_diagnostics.argtypes = [_I, _I, _D, _D, _D, _PD, _PD, _PD]
    lib.orc_diagnostics.restype = _I
    lib.orc_dt_limit.argtypes = [_D, _D, _D, _D, _D, _D, _D, _D]
    lib.orc_dt_limit.restype = _D
    lib.orc_threads.argtypes = []
    lib.orc_threads.restype = _I
    lib.orc_set_threads.argtypes = [_I]
    lib.orc_set_threads.restype = None
    if omp:
        _omp_lib = lib
    else:
        _lib = lib
    return lib


def _ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_PD)


# --------------------------------------------------------------------------
# Random perturbation of sigma (Sec. 3; Eq. CoefCrsDif)

def philox4x32_10(ctr, key):
    """Philox4x32-10 block (Salmon et al., SC'11): 4 counter words, 2 key
    words -> 4 output words."""
    lib = _load()
    c = (ctypes.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    k = (ctypes.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    o = (ctypes.c_uint32 * 4)()
    lib.orc_philox4x32_10(c, k, o)
    return [int(v) for v in o]


def noise_delta(seed: int, idx: int, step: int, dist: int) -> float:
    """Delta of one cell: uniform on [-1,1) (dist 0) or triangular on (-1,1)
    (dist 1), keyed by (seed, cell index, time step)."""
    return float(_load().orc_noise_delta(seed, idx, step, dist))


def sigma_field(nx, ny, seed, sigma0, amp, dist=0, step=0) -> np.ndarray:
    """sigma = sigma0 (1 + a Delta) on every cell (Eq. CoefCrsDif)."""
    s = np.empty((ny, nx), np.float64)
    _load().orc_sigma_field(nx, ny, seed, step, sigma0, amp, dist, _ptr(s))
    return s


def sigma_field_f32(nx, ny, seed, sigma0, amp, dist=0, step=0) -> np.ndarray:
    """The FP32 recipe (two 16-bit uniforms per cell from one Philox word,
    four cells per block, float arithmetic), used by FP32-state runs whose
    sigma is redrawn every step; returned as float64 (exactly the float
    values)."""
    s = np.empty((ny, nx), np.float64)
    _load().orc_sigma_field_f32(nx, ny, seed, step, sigma0, amp, dist, _ptr(s))
    return s


def initial_state(nx, ny, dx, n0, bM, r0sq):
    """n = n0, b = bM exp(-r^2/r0sq) (Eq. inicond, Eq. inibacexp)."""
    b = np.empty((ny, nx), np.float64)
    n = np.empty((ny, nx), np.float64)
    _load().orc_initial_state(nx, ny, dx, n0, bM, r0sq, _ptr(b), _ptr(n))
    return b, n


def rhs(sigma, b, n, *, dx, Dn, theta, chi0, chemo_law=0, mobility=0):
    """Semi-discrete right-hand side (r_b, r_n) of Eq. ka-model-dim with the
    chemotactic flux of Eq. chemflux."""
    ny, nx = b.shape
    rb = np.empty_like(b)
    rn = np.empty_like(n)
    _load().orc_rhs(nx, ny, dx, Dn, theta, chi0, chemo_law, mobility,
                    _ptr(np.ascontiguousarray(sigma)), _ptr(np.ascontiguousarray(b)),
                    _ptr(np.ascontiguousarray(n)), _ptr(rb), _ptr(rn))
    return rb, rn


def step(sigma, b, n, *, dx, dt, Dn, theta, chi0, chemo_law=0, mobility=0, scheme=0):
    """One time step (scheme 0 forward Euler, 1 Heun); returns new (b, n)."""
    ny, nx = b.shape
    bo = np.empty_like(b)
    no = np.empty_like(n)
    f = _load().orc_step_euler if scheme == 0 else _load().orc_step_heun
    rc = f(nx, ny, dx, dt, Dn, theta, chi0, chemo_law, mobility,
           _ptr(np.ascontiguousarray(sigma)), _ptr(np.ascontiguousarray(b)),
           _ptr(np.ascontiguousarray(n)), _ptr(bo), _ptr(no))
    if rc != 0:
        raise MemoryError("oracle step: allocation failed")
    return bo, no


def run(sigma, b, n, nsteps, *, dx, dt, Dn, theta, chi0, chemo_law=0, mobility=0,
        scheme=0, noise_mode=0, seed=0, sigma0=0.0, amp=0.0, dist=0, step0=0, recipe=0,
        threads=0):
    """Advance (b, n) by `nsteps` steps in place (copies are returned).  With
    noise_mode 1 sigma is redrawn from (seed, cell, m) before every step m,
    by the FP64 recipe (recipe 0) or the FP32 recipe (recipe 1).  threads >
    0 runs the threaded build on that many host threads (same bits)."""
    s = np.array(sigma, np.float64, order="C", copy=True)
    bb = np.array(b, np.float64, order="C", copy=True)
    nn = np.array(n, np.float64, order="C", copy=True)
    ny, nx = bb.shape
    lib = _load(omp=threads > 0)
    if threads > 0:
        lib.orc_set_threads(int(threads))
    rc = lib.orc_run(nx, ny, dx, dt, Dn, theta, chi0, chemo_law, mobility, scheme,
                         noise_mode, recipe, seed, sigma0, amp, dist, step0, nsteps,
                         _ptr(s), _ptr(bb), _ptr(nn))
    if rc != 0:
        raise MemoryError("oracle run: allocation failed")
    return bb, nn, s


DIAG_KEYS = ("mass_b", "mass_n", "invariant", "min_b", "min_n", "max_b", "r_env", "finite",
             "area_env")


def omp_threads() -> int:
    """Threads the threaded build uses by default (the host's cores, or
    OMP_NUM_THREADS)."""
    return int(_load(omp=True).orc_threads())


def diagnostics(b, n, *, dx, theta, b_th) -> dict:
    """Masses, the conserved invariant dx^2 sum(b + theta n), extrema, the
    envelope radius, a finiteness flag and the colony's area (cells with
    b >= b_th times dx^2)."""
    ny, nx = b.shape
    out = np.zeros(9, np.float64)
    rc = _load().orc_diagnostics(nx, ny, dx, theta, b_th,
                                 _ptr(np.ascontiguousarray(b, np.float64)),
                                 _ptr(np.ascontiguousarray(n, np.float64)), _ptr(out))
    if rc != 0:
        raise MemoryError("oracle diagnostics: allocation failed")
    d = dict(zip(DIAG_KEYS, (float(v) for v in out)))
    d["finite"] = int(d["finite"])
    return d


def dt_limit(*, dx, Dn, theta, chi0, n0, bM, sigma0, amp) -> float:
    """Explicit stability limit under this project's reading of Sec. 3."""
    return float(_load().orc_dt_limit(dx, Dn, theta, chi0, n0, bM, sigma0, amp))


def default_b_threshold(theta: float, n0: float) -> float:
    """Envelope level: one tenth of the plateau theta*n0 left behind the front."""
    return 0.1 * theta * n0
