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
