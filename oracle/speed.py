"""Front-speed bounds of Sec. 4.1 (Eqs. D-tilde, reac-term, c-bar-chi0,
c-bar-0) in plain FP64 Python.

TEST INFRASTRUCTURE ONLY (see the package docstring).

For the scalar reduction b_t = sigma0 div(D~(b) grad b) + g(b) with
  D~(b, chi0) = n0 b (1 - b/n0) (1 + chi0 b)        (Eq. D-tilde)
  g(b)        = n0 b (1 - b/n0)                     (Eq. reac-term)
the threshold speed is bounded by
  cbar = 2 sqrt( sup_b sigma0 D~ g / b ) = 2 n0 sqrt(sigma0) sqrt(max psi),
  psi(b) = b (1 - b/n0)^2 (1 + chi0 b).
"""
from __future__ import annotations

import math


def D_tilde(b: float, n0: float, chi0: float) -> float:
    """Effective diffusivity of the scalar reduction (Eq. D-tilde)."""
    return n0 * b * (1.0 - b / n0) * (1.0 + chi0 * b)


def g_reaction(b: float, n0: float) -> float:
    """Fisher-KPP reaction of the scalar reduction (Eq. reac-term)."""
    return n0 * b * (1.0 - b / n0)


def psi(b: float, n0: float, chi0: float) -> float:
    """psi(b) = b (1 - b/n0)^2 (1 + chi0 b)."""
    return b * (1.0 - b / n0) ** 2 * (1.0 + chi0 * b)


def b_star(n0: float, chi0: float) -> float:
    """Maximiser of psi on (0, n0) (closed form of Sec. 4.1 for chi0 > 0;
    n0/3 for chi0 = 0)."""
    if chi0 == 0.0:
        return n0 / 3.0
    a = 0.5 * n0 - 0.75 / chi0
    return 0.5 * a + 0.5 * math.sqrt(a * a + n0 / chi0)


def c_bar(n0: float, chi0: float, sigma0: float) -> float:
    """Upper bound on the threshold front speed (Eq. c-bar-chi0)."""
    return 2.0 * n0 * math.sqrt(sigma0) * math.sqrt(psi(b_star(n0, chi0), n0, chi0))


def c_bar_no_chemotaxis(n0: float, sigma0: float) -> float:
    """chi0 = 0 closed form 4/(3 sqrt 3) n0^(3/2) sigma0^(1/2) (Eq. c-bar-0,
    reading the printed sigma^(1/2) as sigma0^(1/2))."""
    return 4.0 / (3.0 * math.sqrt(3.0)) * n0 ** 1.5 * math.sqrt(sigma0)


# ---------------------------------------------------------------------------
# Threshold speed c* of the Malaguti-Marcelli problem (Appendix, Eqs.
# scalar-mm, problemstar): travelling fronts of u_t = (D(u) u_x)_x + g(u)
# on [0, 1] exist for c >= c*, where c* is the least c for which
#     dz/du = -c - D(u) g(u) / z,   z(0+) = z(1-) = 0,   z < 0 on (0, 1)
# has a solution (z = D u' along the front).
#
# Bisection on c: the trajectory leaving (1, 0) is followed backwards to
# u = eps.  Below c* it ends at z(0+) < 0, so z(eps)/eps is large and
# negative; from c* on it enters the origin, with z(eps)/eps ~ -c at c*
# and ~ 0 above it.

def _trajectory_end(c, h, eps):
    from scipy.integrate import solve_ivp
    d = 1e-7
    hp1 = -h(1.0 - d) / d                  # h'(1) <= 0
    k = 0.5 * (-c + math.sqrt(c * c + 4.0 * abs(hp1)))
    u0 = 1.0 - eps
    z0 = -k * eps if k > 1e-12 else -h(u0) / c
    if z0 >= 0.0:
        z0 = -1e-300
    event = lambda u, z: z[0]
    event.terminal = True
    # z is tiny at both ends, so without a step cap the error control can
    # jump straight across the interval
    sol = solve_ivp(lambda u, z: [-c - h(u) / z[0]], [u0, eps], [z0], method="Radau",
                    rtol=1e-10, atol=1e-16, max_step=1e-3, events=event)
    if sol.status == -1:
        raise RuntimeError(f"threshold_speed: integration failed at c = {c}: {sol.message}")
    return sol.t[-1], sol.y[0][-1]


def threshold_speed(D, g, c_hi: float, eps: float = 1e-7, tol: float = 1e-9) -> float:
    """c* for u_t = (D(u) u_x)_x + g(u) with D, g >= 0 on [0, 1] vanishing
    as in the Appendix; c_hi must be an upper bound (e.g. the bound of
    Eq. threshold)."""
    h = lambda u: D(u) * g(u)
    lo, hi = 0.0, c_hi
    while hi - lo > tol * max(hi, 1e-12):
        c = 0.5 * (lo + hi)
        u, z = _trajectory_end(c, h, eps)
        below = (u > 2 * eps) or (z / u < -0.5 * c)
        if below:
            lo = c
        else:
            hi = c
    return 0.5 * (lo + hi)


def mm_bound(D, g, n: int = 200001) -> float:
    """2 sqrt(sup_u D(u) g(u) / u) (Eq. threshold), on a fine grid."""
    u = [(k + 0.5) / n for k in range(n)]
    return 2.0 * math.sqrt(max(D(x) * g(x) / x for x in u))


def c_star(n0: float, chi0: float, sigma0: float) -> float:
    """Threshold speed of the scalar reduction of Sec. 4.1
    b_t = sigma0 div(D~(b) grad b) + g(b) (Eqs. scalar-eq-b-re, D-tilde,
    reac-term), written for u = b/n0 in [0, 1]:
    u_t = (sigma0 n0^2 u(1-u)(1+chi0 n0 u) u_x)_x + n0 u (1-u)."""
    D = lambda u: sigma0 * n0 * n0 * u * (1.0 - u) * (1.0 + chi0 * n0 * u)
    g = lambda u: n0 * u * (1.0 - u)
    return threshold_speed(D, g, c_hi=1.01 * c_bar(n0, chi0, sigma0))
