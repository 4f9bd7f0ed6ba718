"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test pins the oracle to something other than itself: published
known-answer vectors, closed forms, exact invariants, exact symmetries,
the continuous operator of Eq. ka-chem-model (manufactured solutions with a
measured convergence order), and the speed bounds of Sec. 4.1.
"""
import math
import os

import numpy as np
import pytest

import oracle
from oracle import speed

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

CFG0 = dict(nx=256, ny=256, dx=1.0, Dn=1.0, theta=1.0, chi0=0.5, n0=0.7,
            sigma0=4.0, amp=0.5, bM=0.5, r0sq=16.0, cfl=0.2, seed=0)


def cfg0_dt(c=CFG0):
    return c["cfl"] * oracle.dt_limit(dx=c["dx"], Dn=c["Dn"], theta=c["theta"], chi0=c["chi0"],
                                      n0=c["n0"], bM=c["bM"], sigma0=c["sigma0"], amp=c["amp"])


# ---------------------------------------------------------------------------
# Random perturbation of sigma (Sec. 3)

def _kat_rows():
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            lhs, rhs = line.split(":")
            w = [int(t, 16) for t in lhs.split()]
            rows.append((w[:4], w[4:6], [int(t, 16) for t in rhs.split()]))
    return rows


@pytest.mark.parametrize("ctr,key,expect", _kat_rows())
def test_philox_known_answers(ctr, key, expect):
    assert oracle.philox4x32_10(ctr, key) == expect


def test_uniform_noise_moments():
    # Delta ~ U[-1,1): mean 0, variance 1/3; sigma = sigma0 (1 + a Delta)
    s = oracle.sigma_field(512, 512, 7, 4.0, 0.5, dist=0)
    d = (s / 4.0 - 1.0) / 0.5
    n = d.size
    assert abs(d.mean()) < 5 * math.sqrt(1 / 3 / n)
    assert abs(d.var() - 1 / 3) < 5 * math.sqrt(4 / 45 / n)
    assert d.min() >= -1.0 and d.max() < 1.0
    assert d.min() < -0.999 and d.max() > 0.999


def test_triangular_noise_distribution():
    # Delta = U_a + U_b - 1 is triangular on (-1,1): CDF F(x) = (1+x)^2/2 for
    # x <= 0 and 1 - (1-x)^2/2 for x >= 0; variance 1/6.  Kolmogorov-Smirnov.
    s = oracle.sigma_field(400, 400, 3, 1.0, 1.0, dist=1)
    d = np.sort((s - 1.0).ravel())
    n = d.size
    F = np.where(d <= 0, 0.5 * (1 + d) ** 2, 1 - 0.5 * (1 - d) ** 2)
    ks = np.max(np.maximum(np.arange(1, n + 1) / n - F, F - np.arange(n) / n))
    assert ks < 1.63 / math.sqrt(n)          # 1% KS critical value
    assert abs(d.var() - 1 / 6) < 0.01
    assert d.min() > -1.0 and d.max() < 1.0


def test_noise_redraw_differs_per_step_and_seed():
    a = oracle.sigma_field(64, 64, 1, 1.0, 1.0, dist=1, step=0)
    b = oracle.sigma_field(64, 64, 1, 1.0, 1.0, dist=1, step=1)
    c = oracle.sigma_field(64, 64, 2, 1.0, 1.0, dist=1, step=0)
    assert not np.any(a == b) or np.mean(a == b) < 1e-3
    assert np.mean(a == c) < 1e-3
    # a cell's value depends only on (seed, global index, step): a 64x64 field
    # and a 64x32 field share their first 32 rows' indices only where j*nx+i
    # agree, i.e. the whole of the smaller one when nx is equal
    d = oracle.sigma_field(64, 32, 1, 1.0, 1.0, dist=1, step=0)
    assert np.array_equal(a[:32], d)


# ---------------------------------------------------------------------------
# Initial state and diagnostics

def test_initial_mass_is_gaussian_integral():
    # the midpoint rule integrates a well-resolved Gaussian to round-off:
    # int bM exp(-r^2/r0sq) dA = pi r0sq bM   (Eq. inibacexp)
    b, n = oracle.initial_state(256, 256, 1.0, 0.7, 0.5, 16.0)
    d = oracle.diagnostics(b, n, dx=1.0, theta=1.0, b_th=0.07)
    assert d["mass_b"] == pytest.approx(math.pi * 16.0 * 0.5, rel=1e-13)
    assert d["mass_n"] == pytest.approx(0.7 * 256 * 256, rel=1e-14)
    assert d["invariant"] == pytest.approx(d["mass_b"] + d["mass_n"], rel=1e-14)
    assert d["min_n"] == 0.7 and d["max_b"] < 0.5


def test_envelope_radius_of_gaussian():
    # b >= b_th  <=>  r^2 <= r0sq ln(bM/b_th); the envelope radius is the
    # largest cell-centre distance inside that disc (enumerated directly).
    nx, ny, dx, bM, r0sq, bth = 101, 80, 0.5, 0.71, 30.0, 0.1
    b, n = oracle.initial_state(nx, ny, dx, 0.35, bM, r0sq)
    d = oracle.diagnostics(b, n, dx=dx, theta=1.0, b_th=bth)
    x = (np.arange(nx) + 0.5 - nx / 2) * dx
    y = (np.arange(ny) + 0.5 - ny / 2) * dx
    r2 = x[None, :] ** 2 + y[:, None] ** 2
    inside = r2 <= r0sq * math.log(bM / bth) * (1 + 1e-12)
    assert d["r_env"] == pytest.approx(math.sqrt(r2[inside].max()), rel=1e-14)
    # the colony's area: the cells of that disc, dx^2 each (enumerated), which
    # approaches the disc's area pi r0sq ln(bM/b_th) as the cells shrink
    assert d["area_env"] == inside.sum() * dx * dx
    assert d["area_env"] == pytest.approx(math.pi * r0sq * math.log(bM / bth), rel=0.02)


def test_diagnostics_flags_nonfinite():
    b, n = oracle.initial_state(16, 16, 1.0, 0.5, 0.5, 4.0)
    b[3, 4] = np.nan
    assert oracle.diagnostics(b, n, dx=1.0, theta=1.0, b_th=0.05)["finite"] == 0


# ---------------------------------------------------------------------------
# Exact discrete solutions

@pytest.mark.parametrize("scheme", [0, 1])
def test_heat_mode_decay_when_b_is_zero(scheme):
    # b = 0: the b-equation is frozen and n obeys the discrete heat equation
    # with no-flux walls.  The Neumann cosine mode cos(pi k (i+1/2)/nx) *
    # cos(pi l (j+1/2)/ny) is an eigenvector with eigenvalue
    # lam = -(4/dx^2)(sin^2(pi k/2nx) + sin^2(pi l/2ny)); forward Euler scales
    # its amplitude by (1 + dt Dn lam) per step, Heun by 1 + z + z^2/2.
    nx, ny, dx, Dn, dt, k, l, A, n0 = 40, 24, 0.7, 1.3, 0.05, 3, 2, 0.2, 1.0
    i = np.arange(nx) + 0.5
    j = np.arange(ny) + 0.5
    phi = np.outer(np.cos(math.pi * l * j / ny), np.cos(math.pi * k * i / nx))
    n = n0 + A * phi
    b = np.zeros_like(n)
    sigma = oracle.sigma_field(nx, ny, 5, 2.0, 0.5)
    lam = -(4 / dx ** 2) * (math.sin(math.pi * k / (2 * nx)) ** 2 + math.sin(math.pi * l / (2 * ny)) ** 2)
    z = dt * Dn * lam
    g = 1 + z if scheme == 0 else 1 + z + 0.5 * z * z
    m = 50
    bb, nn, _ = oracle.run(sigma, b, n, m, dx=dx, dt=dt, Dn=Dn, theta=1.0, chi0=2.0, scheme=scheme)
    assert np.all(bb == 0.0)
    expect = n0 + A * g ** m * phi
    assert np.max(np.abs(nn - expect)) < 1e-13 * n0


@pytest.mark.parametrize("theta", [1.0, 0.6])
def test_reaction_only_is_discrete_logistic_map(theta):
    # Dn = 0 and sigma = 0: each cell keeps C = b + theta n, and with
    # theta n = C - b the Euler step is b <- b + dt b (C - b) (Eq. mass-conser
    # and the logistic equation that follows it).
    nx, ny, dt = 7, 5, 0.03
    rng = np.random.default_rng(0)
    b0 = rng.uniform(0.01, 0.5, (ny, nx))
    n0 = rng.uniform(0.2, 1.0, (ny, nx))
    sigma = np.zeros((ny, nx))
    m = 200
    bb, nn, _ = oracle.run(sigma, b0, n0, m, dx=1.0, dt=dt, Dn=0.0, theta=theta, chi0=1.0)
    C = b0 + theta * n0
    b = b0.copy()
    for _ in range(m):
        b = b + dt * b * (C - b)  # theta n b = b (C - b)
    assert np.max(np.abs(bb - b)) < 1e-12
    assert np.max(np.abs(bb + theta * nn - C)) < 1e-13


@pytest.mark.parametrize("scheme,order", [(0, 1), (1, 2)])
def test_time_integrator_order_on_logistic(scheme, order):
    # Continuous limit of the reaction-only system: b(t) = C / (1 + (C/b0 - 1)
    # e^{-C t}) with theta = 1 (Eq. mass-conser).  Halving dt divides the error
    # by 2^order: 2 for forward Euler, 4 for Heun (second-order Runge-Kutta).
    C, b0, T = 1.0, 0.05, 4.0
    exact = C / (1 + (C / b0 - 1) * math.exp(-C * T))
    errs = []
    for m in (100, 200, 400):
        dt = T / m
        bb, nn, _ = oracle.run(np.zeros((1, 1)), np.full((1, 1), b0), np.full((1, 1), C - b0), m,
                               dx=1.0, dt=dt, Dn=0.0, theta=1.0, chi0=0.0, scheme=scheme)
        errs.append(abs(bb[0, 0] - exact))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert abs(math.log2(r1) - order) < 0.1 and abs(math.log2(r2) - order) < 0.1


# ---------------------------------------------------------------------------
# Manufactured solutions: the discrete right-hand side converges, at second
# order for the central scheme, to the continuous operator of Eq. ka-chem-model
# (general form with Dn, theta) evaluated symbolically.

def _mms_operator(chemo_law):
    sp = pytest.importorskip("sympy")
    X, Y = sp.symbols("X Y")
    Lx, Ly = 3.0, 2.0
    b = 0.3 + 0.2 * sp.cos(sp.pi * X / Lx) * sp.cos(2 * sp.pi * Y / Ly)
    n = 0.6 + 0.3 * sp.cos(2 * sp.pi * X / Lx) * sp.cos(sp.pi * Y / Ly)
    s = 2.0 + 0.5 * sp.cos(sp.pi * X / Lx) + 0.3 * sp.cos(sp.pi * Y / Ly)
    Dn, theta, chi0 = 1.7, 0.8, 2.5
    chi = chi0 / (1 + n) ** 2 if chemo_law == 0 else chi0
    fx = s * n * b * sp.diff(b, X) - chi * s * n * b ** 2 * sp.diff(n, X)
    fy = s * n * b * sp.diff(b, Y) - chi * s * n * b ** 2 * sp.diff(n, Y)
    rb = sp.diff(fx, X) + sp.diff(fy, Y) + theta * n * b
    rn = Dn * (sp.diff(n, X, 2) + sp.diff(n, Y, 2)) - n * b
    f = {k: sp.lambdify((X, Y), e, "numpy") for k, e in
         dict(b=b, n=n, s=s, rb=rb, rn=rn).items()}
    return f, Lx, Ly, dict(Dn=Dn, theta=theta, chi0=chi0)


@pytest.mark.parametrize("chemo_law", [0, 1])
@pytest.mark.parametrize("mobility,order", [(0, 2.0), (1, 1.0)])
def test_rhs_converges_to_continuous_operator(chemo_law, mobility, order):
    f, Lx, Ly, par = _mms_operator(chemo_law)
    errs = []
    for N in (48, 96, 192):
        nx, ny = N, int(N * Ly / Lx)
        dx = Lx / nx
        Xc = (np.arange(nx) + 0.5) * dx
        Yc = (np.arange(ny) + 0.5) * dx
        XX, YY = np.meshgrid(Xc, Yc)
        fb, fn, fs = (np.asarray(f[k](XX, YY), np.float64) * np.ones_like(XX) for k in "bns")
        rb, rn = oracle.rhs(fs, fb, fn, dx=dx, chemo_law=chemo_law, mobility=mobility, **par)
        # every cell, wall cells included: the walls carry the exact (zero)
        # flux because the manufactured fields have zero normal derivative
        eb = np.abs(rb - f["rb"](XX, YY)).max()
        en = np.abs(rn - f["rn"](XX, YY)).max()
        errs.append(max(eb, en))
    rates = [math.log2(errs[k] / errs[k + 1]) for k in range(2)]
    assert min(rates) > order - 0.25, (errs, rates)
    assert errs[-1] < (2e-3 if order == 2.0 else 3e-2)


# ---------------------------------------------------------------------------
# Invariants and symmetries of the full iteration

def _brute_force_step(s, b, n, dx, dt, Dn, theta, chi0, mobility=0):
    """One forward-Euler step of Eq. ka-chem-model on a tiny grid, cell by
    cell, each face flux written out from the face means (reading of the
    discretisation), walls carrying no flux.  Indexing is [y][x].  With
    mobility 1 the b^2 of the chemotactic flux is the donor cell's: the cell
    of the pair with the lower nutrient, the one bacteria leave when they
    climb the nutrient gradient."""
    ny, nx = b.shape
    bo, no = np.empty_like(b), np.empty_like(n)

    def flux(P, Q):  # from cell Q into cell P across their shared face
        sf = 0.5 * (s[P] + s[Q])
        nf = 0.5 * (n[P] + n[Q])
        bf = 0.5 * (b[P] + b[Q])
        chi = chi0 / (1.0 + nf) ** 2
        if mobility == 0:
            m = bf * bf
        else:
            donor = P if n[P] < n[Q] else Q     # equal n: no chemotactic flux either way
            m = b[donor] ** 2
        Fd = sf * nf * bf * (b[Q] - b[P]) / dx          # Kawasaki cross diffusion
        Fc = chi * sf * nf * m * (n[Q] - n[P]) / dx     # nutrient chemotaxis
        G = Dn * (n[Q] - n[P]) / dx                     # nutrient diffusion
        return Fd - Fc, G

    for j in range(ny):
        for i in range(nx):
            db = dn = 0.0
            for dj, di in ((0, 1), (0, -1), (1, 0), (-1, 0)):
                jj, ii = j + dj, i + di
                if 0 <= jj < ny and 0 <= ii < nx:
                    F, G = flux((j, i), (jj, ii))
                    db += F
                    dn += G
            r = n[j, i] * b[j, i]
            bo[j, i] = b[j, i] + dt * (db / dx + theta * r)
            no[j, i] = n[j, i] + dt * (dn / dx - r)
    return bo, no


@pytest.mark.parametrize("mobility", [0, 1])
@pytest.mark.parametrize("nx,ny", [(3, 3), (4, 5), (5, 2)])
def test_one_step_against_brute_force(nx, ny, mobility):
    # tiny non-square grids: every cell touches a wall, so index order (x
    # fastest), the walls on each side and each face mean are all exercised;
    # random n makes the donor fall on either side of the faces
    rng = np.random.default_rng(nx * 10 + ny)
    s = rng.uniform(1.0, 6.0, (ny, nx))
    b = rng.uniform(0.05, 0.9, (ny, nx))
    n = rng.uniform(0.05, 0.9, (ny, nx))
    kw = dict(dx=0.7, dt=0.013, Dn=1.3, theta=0.8, chi0=1.7)
    ob, on = oracle.step(s, b, n, mobility=mobility, **kw)
    bb, bn = _brute_force_step(s, b, n, mobility=mobility, **kw)
    assert np.allclose(ob, bb, rtol=1e-14, atol=0) and np.allclose(on, bn, rtol=1e-14, atol=0)
    # the two mobilities really differ on these fields, so each is pinned apart
    cb, _ = _brute_force_step(s, b, n, mobility=1 - mobility, **kw)
    assert np.max(np.abs(cb - bb)) > 1e-6


@pytest.mark.parametrize("axis", [0, 1])
@pytest.mark.parametrize("empty_side", [0, 1])
@pytest.mark.parametrize("law", [0, 1])
def test_donor_cell_keeps_an_empty_lower_nutrient_cell_nonnegative(axis, empty_side, law):
    # Two cells, one empty of bacteria.  Chemotaxis carries bacteria up the
    # nutrient gradient (Eq. chemflux), so across the face it moves them out
    # of the lower-n cell into the higher-n one.  Reading c3: the donor-cell
    # mobility takes b^2 of the lower-n cell.
    #   (a) empty cell has the LOWER n: it is the donor and holds nothing, so
    #       no chemotactic flux crosses the face at any chi0 -- its update is
    #       the chi0 = 0 update bit for bit and it stays >= 0, while the central
    #       b_f^2 drives it negative once chi0 is large;
    #   (b) empty cell has the HIGHER n: the full cell is the donor, so the
    #       chemotactic flux is chi(n_f) s_f n_f b_full^2 dn / dx, computed here
    #       by hand.  A donor taken from the wrong side would give 0 in (b) and
    #       a negative cell in (a).
    dx, dt, theta, Dn = 0.5, 1e-3, 1.0, 1.0
    s0 = np.array([2.0, 3.0])
    bfull, nlo, nhi = 0.6, 0.2, 0.9
    for empty_is_low in (True, False):
        b = np.array([0.0, bfull]) if empty_side == 0 else np.array([bfull, 0.0])
        ne = nlo if empty_is_low else nhi
        nf_ = nhi if empty_is_low else nlo
        n = np.array([ne, nf_]) if empty_side == 0 else np.array([nf_, ne])
        shape = (1, 2) if axis == 0 else (2, 1)
        S, B, N = (a.reshape(shape) for a in (s0, b, n))
        e = empty_side
        chi0 = 200.0
        kw = dict(dx=dx, Dn=Dn, theta=theta, chemo_law=law)
        rb, _ = oracle.rhs(S, B, N, chi0=chi0, mobility=1, **kw)
        rb0, _ = oracle.rhs(S, B, N, chi0=0.0, mobility=1, **kw)
        rbc, _ = oracle.rhs(S, B, N, chi0=chi0, mobility=0, **kw)
        rb, rb0, rbc = rb.ravel(), rb0.ravel(), rbc.ravel()
        if empty_is_low:
            assert rb[e] == rb0[e] and rb[e] > 0.0
            assert rbc[e] < 0.0                   # central mobility: negative after one step
            bb, _ = oracle.step(S, B, N, dt=dt, chi0=chi0, mobility=1, **kw)
            assert bb.ravel()[e] >= 0.0
        else:
            sf, nfc = 0.5 * (s0[0] + s0[1]), 0.5 * (nlo + nhi)
            chi = chi0 / (1 + nfc) ** 2 if law == 0 else chi0
            Fc = chi * sf * nfc * bfull ** 2 * (nhi - nlo) / dx
            # the chemotactic part of the empty cell's rate: Fc / dx into it
            assert rb[e] - rb0[e] == pytest.approx(Fc / dx, rel=1e-13)


@pytest.mark.parametrize("theta,Dn", [(1.0, 1.0), (0.7, 1.3)])
def test_conservation_of_b_plus_theta_n(theta, Dn):
    # d/dt int (b + theta n) = 0 for Eq. ka-model-dim with no-flux walls; the
    # discrete fluxes telescope and the reaction terms cancel, so the sum
    # changes only by round-off.
    c = dict(CFG0, nx=96, ny=80, theta=theta, Dn=Dn)
    dt = cfg0_dt(c)
    s = oracle.sigma_field(c["nx"], c["ny"], 0, c["sigma0"], c["amp"])
    b, n = oracle.initial_state(c["nx"], c["ny"], c["dx"], c["n0"], c["bM"], c["r0sq"])
    d0 = oracle.diagnostics(b, n, dx=1.0, theta=theta, b_th=0.07)
    bb, nn, _ = oracle.run(s, b, n, 2000, dx=1.0, dt=dt, Dn=Dn, theta=theta, chi0=c["chi0"])
    d1 = oracle.diagnostics(bb, nn, dx=1.0, theta=theta, b_th=0.07)
    assert abs(d1["invariant"] - d0["invariant"]) <= 1e-12 * d0["invariant"]
    assert d1["mass_b"] > 5 * d0["mass_b"]      # the colony grew


def test_positivity_config0():
    c = CFG0
    dt = cfg0_dt()
    s = oracle.sigma_field(c["nx"], c["ny"], c["seed"], c["sigma0"], c["amp"])
    b, n = oracle.initial_state(c["nx"], c["ny"], c["dx"], c["n0"], c["bM"], c["r0sq"])
    bb, nn, _ = oracle.run(s, b, n, 2000, dx=1.0, dt=dt, Dn=1.0, theta=1.0, chi0=c["chi0"])
    d = oracle.diagnostics(bb, nn, dx=1.0, theta=1.0, b_th=0.07)
    assert d["finite"] == 1 and d["min_b"] >= 0.0 and d["min_n"] >= 0.0


@pytest.mark.parametrize("N", [48, 47])
def test_eightfold_symmetry_with_uniform_sigma(N):
    # a = 0 (uniform sigma) and a centred inoculum on a square grid: the
    # scheme commutes with the dihedral group of the square, exactly.
    b, n = oracle.initial_state(N, N, 1.0, 0.7, 0.5, 16.0)
    s = np.full((N, N), 4.0)
    bb, nn, _ = oracle.run(s, b, n, 300, dx=1.0, dt=0.006, Dn=1.0, theta=1.0, chi0=0.5)
    for f in (bb, nn):
        assert np.array_equal(f, f.T)
        assert np.array_equal(f, f[::-1, :])
        assert np.array_equal(f, f[:, ::-1])


def test_chi_zero_ignores_chemotaxis_options():
    # chi0 = 0 is the Kawasaki model (Eq. ka-model-dim): the chemotactic law
    # and the face mobility must not matter, bit for bit.
    s = oracle.sigma_field(30, 20, 1, 4.0, 0.5)
    b, n = oracle.initial_state(30, 20, 1.0, 0.7, 0.5, 16.0)
    outs = [oracle.run(s, b, n, 50, dx=1.0, dt=0.006, Dn=1.0, theta=1.0, chi0=0.0,
                       chemo_law=law, mobility=mob)[0] for law in (0, 1) for mob in (0, 1)]
    for o in outs[1:]:
        assert np.array_equal(o, outs[0])


def test_chemotaxis_speeds_up_the_colony():
    # Prop. 1 / Sec. 3: switching the chemotactic flux on moves the envelope
    # faster.
    c = dict(CFG0, nx=128, ny=128)
    s = oracle.sigma_field(128, 128, 0, c["sigma0"], c["amp"])
    b, n = oracle.initial_state(128, 128, 1.0, c["n0"], c["bM"], c["r0sq"])
    r = []
    for chi0 in (0.0, 2.0):
        bb, nn, _ = oracle.run(s, b, n, 1500, dx=1.0, dt=0.006, Dn=1.0, theta=1.0, chi0=chi0)
        r.append(oracle.diagnostics(bb, nn, dx=1.0, theta=1.0, b_th=0.07)["r_env"])
    assert r[1] > r[0]


def test_per_step_noise_uses_step_index():
    # noise_mode 1 redraws sigma from (seed, cell, m) before step m.
    nx, ny = 20, 12
    b, n = oracle.initial_state(nx, ny, 1.0, 0.7, 0.5, 9.0)
    bb, nn, s_last = oracle.run(np.zeros((ny, nx)), b, n, 3, dx=1.0, dt=0.005, Dn=1.0,
                                theta=1.0, chi0=0.5, noise_mode=1, seed=9, sigma0=4.0,
                                amp=1.0, dist=1, step0=10)
    assert np.array_equal(s_last, oracle.sigma_field(nx, ny, 9, 4.0, 1.0, dist=1, step=12))
    b1, n1 = b, n
    for m in (10, 11, 12):
        s = oracle.sigma_field(nx, ny, 9, 4.0, 1.0, dist=1, step=m)
        b1, n1 = oracle.step(s, b1, n1, dx=1.0, dt=0.005, Dn=1.0, theta=1.0, chi0=0.5)
    assert np.array_equal(bb, b1) and np.array_equal(nn, n1)


# ---------------------------------------------------------------------------
# Stability limit (reading c7), both branches by hand

def test_dt_limit_diffusive_branch_by_hand():
    # config 0: B = bM + theta n0 = 1.2, sigma_max = 4 (1 + 0.5) = 6,
    # D = 6 * 0.7 * 1.2 * (1 + 0.5 * 1.2) = 8.064 > Dn, so the limit is
    # dx^2 / (4 D) = 1 / 32.256 (the reaction branch is 1 / 5.2)
    lim = oracle.dt_limit(dx=1.0, Dn=1.0, theta=1.0, chi0=0.5, n0=0.7, bM=0.5, sigma0=4.0, amp=0.5)
    assert lim == pytest.approx(1.0 / 32.256, rel=1e-15)


def test_dt_limit_reaction_branch_by_hand():
    # Dn = 10 dominates the cross diffusion (sigma_max n0 B (1 + chi0 B) =
    # 0.5 * 0.5 * 1.0 * 1 = 0.25), so Dmax = Dn and the diffusive branch is
    # dx^2 / (4 Dn) = 0.25 / 40 = 1/160; the branch that keeps n >= 0 under
    # Euler, 1 / (4 Dn / dx^2 + B) = 1 / (160 + 1), is smaller and decides
    lim = oracle.dt_limit(dx=0.5, Dn=10.0, theta=1.0, chi0=0.0, n0=0.5, bM=0.5, sigma0=0.5, amp=0.0)
    assert lim == pytest.approx(1.0 / 161.0, rel=1e-15)
    # and that branch is what it says: with b = B everywhere (the largest b the
    # reading allows) and an n checkerboard, one Euler step at the limit takes
    # the low cells to exactly 0 and no lower
    nx = ny = 6
    n = np.where((np.add.outer(np.arange(ny), np.arange(nx)) % 2) == 0, 1.0, 0.0)
    b = np.full((ny, nx), 1.0)
    s = np.zeros((ny, nx))
    _, nn = oracle.step(s, b, n, dx=0.5, dt=lim, Dn=10.0, theta=1.0, chi0=0.0)
    interior = (slice(1, -1), slice(1, -1))
    assert nn[interior].min() >= -1e-15


# ---------------------------------------------------------------------------
# Speed bounds (Sec. 4.1, Prop. 1)

@pytest.mark.parametrize("n0", [0.35, 0.71, 1.07, 2.0, 3.0, 4.0])
def test_psi_maximum_without_chemotaxis(n0):
    assert speed.psi(n0 / 3, n0, 0.0) == pytest.approx(4 * n0 / 27, rel=1e-14)
    bs = np.linspace(0, n0, 200001)
    assert np.max(speed.psi(bs, n0, 0.0)) <= 4 * n0 / 27 * (1 + 1e-14)
    assert speed.c_bar(n0, 0.0, 1.0) == pytest.approx(speed.c_bar_no_chemotaxis(n0, 1.0), rel=1e-14)


@pytest.mark.parametrize("n0", [0.35, 0.71, 1.07, 2.0, 4.0])
@pytest.mark.parametrize("chi0", [0.1, 1.0, 2.5, 5.0, 10.0])
def test_b_star_maximises_psi(n0, chi0):
    scipy_opt = pytest.importorskip("scipy.optimize")
    res = scipy_opt.minimize_scalar(lambda b: -speed.psi(b, n0, chi0), bounds=(0, n0),
                                    method="bounded", options=dict(xatol=1e-12))
    assert speed.b_star(n0, chi0) == pytest.approx(res.x, rel=1e-6, abs=1e-9)
    assert 0 < speed.b_star(n0, chi0) < n0


@pytest.mark.parametrize("n0", [0.35, 1.07, 3.0])
def test_c_bar_against_direct_supremum(n0):
    # cbar = 2 sqrt(sup_b sigma0 D~(b) g(b) / b), evaluated by brute force.
    sigma0 = 4.0
    for chi0 in (0.0, 1.0, 5.0):
        bs = np.linspace(1e-9, n0, 400001)
        sup = max(sigma0 * speed.D_tilde(b, n0, chi0) * speed.g_reaction(b, n0) / b for b in bs[::97])
        sup = max(sup, float(np.max(sigma0 * speed.D_tilde(bs, n0, chi0) * speed.g_reaction(bs, n0) / bs)))
        assert speed.c_bar(n0, chi0, sigma0) == pytest.approx(2 * math.sqrt(sup), rel=1e-8)


def test_c_bar_monotone_in_chi0():
    # Prop. 1 (i)
    for n0 in (0.35, 0.71, 2.0):
        v = [speed.c_bar(n0, chi0, 1.0) for chi0 in np.linspace(0, 10, 101)]
        assert all(b >= a for a, b in zip(v, v[1:]))
    assert speed.b_star(1.0, 1e-9) == pytest.approx(1 / 3, rel=1e-6)


# ---------------------------------------------------------------------------
# FP32 recipe of the per-step noise

@pytest.mark.parametrize("dist", [0, 1])
def test_fp32_noise_recipe_laws_and_pairing(dist):
    # the FP32 recipe draws four cells from one Philox block (a 32-bit word
    # each, split into two 16-bit integers): the values lie on the exact
    # 2^-16 lattice, the law is uniform / triangular (KS), the cells of a
    # block are uncorrelated, and a cell's value follows from word h of its
    # block (the known-answer-pinned generator)
    s0, a = 4.0, 0.8
    s32 = oracle.sigma_field_f32(300, 200, 11, s0, a, dist=dist, step=5)
    assert np.all(s32 == s32.astype(np.float32))
    flat = ((s32 / s0 - 1) / a).ravel()
    lattice = flat * 2.0 ** 16
    assert np.max(np.abs(lattice - np.round(lattice))) < 1e-2   # float rounding of a and s0
    quads = flat[: flat.size // 4 * 4].reshape(-1, 4)
    for u in range(4):
        for v in range(u + 1, 4):
            rho = np.corrcoef(quads[:, u], quads[:, v])[0, 1]
            assert abs(rho) < 5 / math.sqrt(len(quads))
    for idx in (0, 1, 2, 3, 12345, 59999):
        w = oracle.philox4x32_10([idx >> 2, 0, 5, 0], [11, 0])
        h = idx & 3
        ja, jb = w[h] >> 16, w[h] & 0xFFFF
        num = 2 * ja - (1 << 16) if dist == 0 else ja + jb - (1 << 16)
        d = np.float32(num) * np.float32(2.0 ** -16)
        ref = np.float32(s0) * (np.float32(1.0) + np.float32(a) * d)
        assert s32.ravel()[idx] == np.float64(ref)
    d = np.sort(flat)
    if dist == 1:
        F = np.where(d <= 0, 0.5 * (1 + d) ** 2, 1 - 0.5 * (1 - d) ** 2)
    else:
        F = 0.5 * (1 + d)
    m = d.size
    ks = np.max(np.maximum(np.arange(1, m + 1) / m - F, F - np.arange(m) / m))
    assert ks < 1.63 / math.sqrt(m) + 2.0 ** -15


# ---------------------------------------------------------------------------
# Threshold speed c* of the travelling-front problem (Appendix)

def test_threshold_speed_of_the_porous_fisher_equation():
    # u_t = (u u_x)_x + u (1 - u) has a sharp front moving at exactly
    # 1/sqrt(2) (Newman 1980; Aronson 1980); with g = 4 u (1 - u) the speed
    # scales by sqrt(4).
    assert speed.threshold_speed(lambda u: u, lambda u: u * (1 - u), 2.0, tol=1e-6) == \
        pytest.approx(1 / math.sqrt(2), rel=1e-5)
    assert speed.threshold_speed(lambda u: u, lambda u: 4 * u * (1 - u), 4.0, tol=1e-6) == \
        pytest.approx(math.sqrt(2), rel=1e-5)


def test_c_star_below_c_bar_and_increasing_in_chi0():
    # Eq. threshold: c* <= cbar; Prop. 1 (ii): c*(chi0) >= c*(0)
    n0, sigma0 = 0.71, 1.0
    cs = []
    for chi0 in (0.0, 2.5):
        D = lambda u, c=chi0: sigma0 * n0 * n0 * u * (1 - u) * (1 + c * n0 * u)
        g = lambda u: n0 * u * (1 - u)
        cs.append(speed.threshold_speed(D, g, 1.01 * speed.c_bar(n0, chi0, sigma0), tol=1e-5))
        assert cs[-1] < speed.c_bar(n0, chi0, sigma0)
        assert speed.mm_bound(D, g, 20001) == pytest.approx(speed.c_bar(n0, chi0, sigma0), rel=1e-6)
    assert cs[1] > cs[0]


# ---------------------------------------------------------------------------
# Threaded build of the oracle (timed as the all-cores CPU baseline)

@pytest.mark.parametrize("scheme", [0, 1])
def test_threaded_oracle_gives_the_same_bits(scheme):
    # only the row loop of the right-hand side and the update loops are split
    # across threads; each cell's arithmetic is unchanged, so the results are
    # identical to the serial build's
    nx, ny = 97, 61
    s = oracle.sigma_field(nx, ny, 4, 4.0, 0.5)
    b, n = oracle.initial_state(nx, ny, 1.0, 0.7, 0.5, 16.0)
    kw = dict(dx=1.0, dt=0.006, Dn=1.0, theta=1.0, chi0=1.5, scheme=scheme)
    b1, n1, _ = oracle.run(s, b, n, 40, **kw)
    b4, n4, _ = oracle.run(s, b, n, 40, threads=4, **kw)
    assert np.array_equal(b1, b4) and np.array_equal(n1, n4)
    assert oracle.omp_threads() >= 1
