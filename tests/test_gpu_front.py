"""The one-dimensional front-speed study of Sec. 4.2 on the GPU path.

Checks: the strip set-up (ny = 1, constant chemotactic law, no noise)
matches the oracle step for step; the measured front speeds respect the
bound cbar of Eq. c-bar-chi0 (within 5%: the full system is not exactly the
scalar reduction the bound is derived for), grow with chi0 (Prop. 1), and are
of the order of the threshold speed c* of the scalar reduction (Appendix).
"""
import numpy as np
import pytest

import oracle
from oracle import speed

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fs():
    from paper_1301_5058_gb300 import _build
    _build.build()
    from paper_1301_5058_gb300 import front_speed
    return front_speed


def test_strip_matches_oracle(fs):
    import paper_1301_5058_gb300 as cx
    spec = fs.strip_spec(1.07, 5.0, half_length=20.0, dx=0.1)
    kw = {k: v for k, v in spec.items() if k not in ("nx", "ny", "dx", "seed")}
    with cx.Sim(spec["nx"], 1, spec["dx"], seed=0, **kw) as sim:
        dt = cx.cx_get_time(sim.h)[2]
        sim.step(3000)
        gb, gn = sim.field(cx.CX_FIELD_B), sim.field(cx.CX_FIELD_N)
    b, n = oracle.initial_state(spec["nx"], 1, 0.1, 1.07, 0.71, 6.25)
    s = np.ones_like(b)
    ob, on, _ = oracle.run(s, b, n, 3000, dx=0.1, dt=dt, Dn=1.0, theta=1.0, chi0=5.0, chemo_law=1)
    assert np.linalg.norm(gb - ob) <= 1e-12 * np.linalg.norm(ob)
    assert np.linalg.norm(gn - on) <= 1e-12 * np.linalg.norm(on)


def test_front_speeds_against_the_bounds(fs):
    # the regime where the scalar reduction n + b = n0 behind cbar holds:
    # fronts fast against nutrient diffusion (n0 >= 2) and chi0 n0 moderate
    cases = [(2.0, 0.0), (2.0, 1.0), (3.0, 0.0), (3.0, 1.0)]
    res = fs.measure(cases)
    by = {(r["n0"], r["chi0"]): r["speed"] for r in res}
    for (n0, chi0), c in by.items():
        cbar = speed.c_bar(n0, chi0, 1.0)
        assert np.isfinite(c)
        assert c <= 1.05 * cbar, (n0, chi0, c, cbar)
        assert c >= 0.5 * cbar, (n0, chi0, c, cbar)
    for n0 in (2.0, 3.0):
        assert by[(n0, 1.0)] > by[(n0, 0.0)]
    assert all(r["min_b"] >= 0.0 for r in res)
