"""Radial colony runs (the 2D workload of Sec. 3) over the full 50000 steps
of the 16384^2 configuration, on a 1024^2 grid: the colony's envelope stays
inside radius 400 by then, far from the walls.  The envelope velocity has no
printed value in the paper; it is checked against the speed bound of the
scalar reduction (Sec. 4.1), which the constant-chi law gives and the
receptor law (chi(n) <= chi0) can only lower, together with conservation,
positivity and a growing envelope.  Beyond 1000 steps round-off grows with
the colony, so the FP32 run is compared with the FP64 run (itself pinned to
the oracle) on envelope radius and velocity, within 1 %."""
import numpy as np
import pytest

from oracle import speed
from paper_1301_5058_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cx():
    from paper_1301_5058_gb300 import _build
    _build.build()
    import paper_1301_5058_gb300 as cx
    return cx


@pytest.mark.parametrize("chi0", [0.0, 1.0])
def test_radial_run_full_length(cx, chi0):
    from paper_1301_5058_gb300 import radial
    cfg = dict(W.CONFIG1, nx=1024, ny=1024, chi0=chi0)
    out = radial.radial_run(cfg, steps=50000, samples=40)
    ref = radial.radial_run(cfg, steps=50000, samples=40, precision=cx.CX_PREC_F64)
    r = np.asarray(out["r_env"])
    r64 = np.asarray(ref["r_env"])
    assert ref["invariant_rel_drift"] <= 1e-11 and ref["min_b"] >= 0.0 and ref["min_n"] >= 0.0
    assert np.max(np.abs(r - r64) / r64) <= 0.01
    for key in ("velocity_second_half", "velocity_last_quarter"):
        assert abs(out[key] - ref[key]) <= 0.01 * ref[key]
    assert out["finite"] == 1 and out["min_b"] >= 0.0 and out["min_n"] >= 0.0
    # FP32 state: at the leading edge b's growth theta n b dt is representable
    # while the matching loss n b dt is below half an ulp of n, so the
    # invariant grows slowly (FP64 keeps it to 1e-12; measured here 2e-5)
    assert out["invariant_rel_drift"] <= 1e-4
    assert np.all(np.diff(r) >= 0.0) and r[-1] > 2 * r[0]
    assert r[-1] < 0.45 * 1024                           # still clear of the walls
    cbar = speed.c_bar(cfg["n0"], chi0, cfg["sigma0"])
    assert 0.0 < out["velocity_last_quarter"] <= cbar
    print(f"\nchi0={chi0}: R_env {r[0]:.1f} -> {r[-1]:.1f}, v(last quarter) = "
          f"{out['velocity_last_quarter']:.4f} (FP64 {ref['velocity_last_quarter']:.4f}), "
          f"c_bar = {cbar:.4f}, max rel R_env diff {np.max(np.abs(r - r64) / r64):.1e}, "
          f"invariant drift FP32 {out['invariant_rel_drift']:.2e} FP64 "
          f"{ref['invariant_rel_drift']:.1e}")
