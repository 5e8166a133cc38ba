"""Pins of the oracle parts that the transform, mask and Krylov tests leave
open: the amplitude and periodic wrap of the Gaussian vortex of the initial
condition (Sec. 3.1), the absolute scale of the diagnostics (Sec. 3.3, the
energy, enstrophy and palinstrophy of the budget identities, and the
circulation), and the collocation operator on a non-uniform adaptive grid
(Sec. 2.5: derivatives at each point's stencil level with ghost values from
the DD reconstruction), whose error must fall at fourth order where the
stencils read active values and at second order where they read ghosts."""

import numpy as np

from oracle import wrc_oracle as O


def _lattice(NJ):
    h = 2 * np.pi / NJ
    x = -np.pi + h * np.arange(NJ)
    X, Y = np.meshgrid(x, x)
    return h, X, Y


# --------------------------------------------------------------------------
# vortex_field: omega = Gamma / (pi s^2) exp(-r^2 / s^2)
# --------------------------------------------------------------------------

def test_vortex_peak_is_gamma_over_pi_s2():
    NJ = 128
    h, X, Y = _lattice(NJ)
    i0, k0 = 70, 41                      # centre on a lattice point
    xc, yc = -np.pi + h * i0, -np.pi + h * k0
    for gam, s in ((1.0, 0.3), (-0.7, 0.25), (2.5, 0.5)):
        om = O.vortex_field(NJ, [xc], [yc], [gam], [s])
        assert abs(om[k0, i0] - gam / (np.pi * s * s)) <= 1e-14 * abs(gam) / (np.pi * s * s)
        # one lattice cell away along x: exp(-h^2 / s^2) of the peak
        assert abs(om[k0, i0 + 1] / om[k0, i0] - np.exp(-h * h / (s * s))) <= 1e-14


def test_vortex_lattice_integral_is_the_circulation():
    """h^2 sum omega = sum Gamma: the lattice sum of a Gaussian equals its
    integral up to exp(-(pi s / h)^2) (Poisson summation), and the periodic
    images add exp(-pi^2 / s^2).  A wrong normalisation (Gamma / (2 pi s^2),
    exp(-r^2 / (2 s^2))) is off by a factor 2."""
    NJ = 256
    h, _, _ = _lattice(NJ)
    xc, yc = [-0.6, 0.55, 1.7], [0.1, -0.3, 1.2]
    gam, s = [1.0, -0.45, 0.8], [0.3, 0.22, 0.4]
    om = O.vortex_field(NJ, xc, yc, gam, s)
    assert abs(h * h * om.sum() - sum(gam)) <= 1e-12
    for q in range(3):
        one = O.vortex_field(NJ, [xc[q]], [yc[q]], [gam[q]], [s[q]])
        assert abs(h * h * one.sum() - gam[q]) <= 1e-12


def test_vortex_wraps_by_minimum_image():
    """A vortex centred next to the seam x = pi: the part across the seam
    sits at x near -pi with the wrapped distance, and the integral is still
    Gamma (without the wrap half of the vortex would be missing)."""
    NJ = 256
    h, X, Y = _lattice(NJ)
    xc, yc, gam, s = np.pi - 0.05, -np.pi + 0.02, 1.3, 0.3
    om = O.vortex_field(NJ, [xc], [yc], [gam], [s])
    assert abs(h * h * om.sum() - gam) <= 1e-12
    # the point (x, y) = (-pi + 2h, -pi) lies 0.05 + 2h across the x seam
    dx = (-np.pi + 2 * h) + 2 * np.pi - xc
    dy = -np.pi - yc
    expect = gam / (np.pi * s * s) * np.exp(-(dx * dx + dy * dy) / (s * s))
    assert abs(om[0, 2] - expect) <= 1e-14 * expect
    # and the point (x, y) = (pi - h, pi - h) lies across the y seam
    dx = (np.pi - h) - xc
    dy = (np.pi - h) - 2 * np.pi - yc
    expect = gam / (np.pi * s * s) * np.exp(-(dx * dx + dy * dy) / (s * s))
    assert abs(om[NJ - 1, NJ - 1] - expect) <= 1e-14 * expect


# --------------------------------------------------------------------------
# diagnostics: Taylor-Green closed forms with the stencils' own symbols
# --------------------------------------------------------------------------

def test_diagnostics_taylor_green_closed_forms():
    """omega = 2 sin x sin y + c on the full lattice.  The first-derivative
    stencil multiplies sin by d = (8 sin h - sin 2h) / (6h), the Laplacian
    symbol is -2 sigma with sigma = (30 - 32 cos h + 2 cos 2h) / (12 h^2), so
    psi = sin x sin y / sigma and, with sums of sin^2 over the lattice equal to
    NJ / 2 and h NJ = 2 pi,
        E = pi^2 (d / sigma)^2,  Z = 2 pi^2 (1 + c^2),  P = 4 pi^2 d^2,
        circulation = 4 pi^2 c.
    (Continuum: E = pi^2, P = 4 pi^2.)"""
    for n0, J in ((8, 2), (16, 1), (4, 3)):
        cfg = O.Config(n0=n0, J=J, eps=0.0, re=100.0)
        NJ = cfg.NJ
        h, X, Y = _lattice(NJ)
        for c in (0.0, 0.37):
            om = 2 * np.sin(X) * np.sin(Y) + c
            st = O.State(np.ones((NJ, NJ), dtype=bool), om)
            dg = O.diagnostics(cfg, st)
            d = (8 * np.sin(h) - np.sin(2 * h)) / (6 * h)
            sig = (30 - 32 * np.cos(h) + 2 * np.cos(2 * h)) / (12 * h * h)
            assert abs(dg["E"] - np.pi ** 2 * (d / sig) ** 2) <= 1e-12 * np.pi ** 2
            assert abs(dg["Z"] - 2 * np.pi ** 2 * (1 + c * c)) <= 1e-12 * np.pi ** 2
            assert abs(dg["P"] - 4 * np.pi ** 2 * d * d) <= 1e-12 * np.pi ** 2
            assert abs(dg["circulation"] - 4 * np.pi ** 2 * c) <= 1e-12 * np.pi ** 2
        # the discrete values differ from the continuum ones at O(h^4) only
        assert abs(np.pi ** 2 * (d / sig) ** 2 - np.pi ** 2) <= 0.1 * h ** 4 * np.pi ** 2


def test_diagnostics_read_the_reconstruction_on_an_adaptive_grid():
    """On a thresholded grid the diagnostics are those of R(omega): the same
    numbers as for the full-lattice field R(omega) itself."""
    cfg = O.Config(n0=16, J=3, eps=1e-3, re=100.0)
    st = O.initial_state(cfg, [-0.6, 0.6], [0.0, 0.1], [1.0, 0.8], [0.3, 0.3])
    assert st.active.sum() < 0.5 * cfg.NJ ** 2
    R = O.reconstruct(st.omega, st.active, cfg.J)
    full = O.diagnostics(cfg, O.State(np.ones_like(st.active), R))
    ad = O.diagnostics(cfg, st)
    for key in ("E", "Z", "P", "circulation"):
        assert abs(ad[key] - full[key]) <= 1e-13 * abs(full[key])


# --------------------------------------------------------------------------
# apply_operator on a fixed non-uniform closed grid: convergence rates
# --------------------------------------------------------------------------

def _three_zone_grid(n0, J):
    """Level 0 everywhere, every point inside r < 1.1, the level <= 1 points in
    1.1 <= r < 2.0, then the DD closure: a grid with coarse-fine interfaces
    of both kinds whose shape in [-pi, pi)^2 does not change with n0."""
    NJ = n0 << J
    _, X, Y = _lattice(NJ)
    lev = O.levels(n0, J)
    r = np.hypot(X - 0.2, Y + 0.1)
    A = (lev == 0) | (r < 1.1) | ((r < 2.0) & (lev <= 1))
    return O.closure(A, J), lev


def _fields(X, Y):
    U = 0.7 * np.cos(Y) + 0.3 * np.sin(X + Y)
    V = 0.5 * np.sin(X) - 0.3 * np.sin(X + Y)
    q = np.sin(X) * np.cos(Y) + 0.5 * np.sin(2 * X + Y)
    qx = np.cos(X) * np.cos(Y) + np.cos(2 * X + Y)
    qy = -np.sin(X) * np.sin(Y) + 0.5 * np.cos(2 * X + Y)
    lap = -2 * np.sin(X) * np.cos(Y) - 2.5 * np.sin(2 * X + Y)
    return U, V, q, qx, qy, lap


def _reads_ghost(A, jx, jy, J):
    """Active points whose x or y stencil (offsets +-1, +-2 at the stencil
    level's spacing) reads a point outside the grid, i.e. a ghost value."""
    reads = np.zeros_like(A)
    for j in range(J + 1):
        s = 1 << (J - j)
        for d in (-2, -1, 1, 2):
            reads |= A & (jx == j) & ~np.roll(A, -d * s, axis=1)
            reads |= A & (jy == j) & ~np.roll(A, -d * s, axis=0)
    return reads


def test_operator_convergence_on_nonuniform_grid():
    """A_n q = -U q_x - V q_y + nu (q_xx + q_yy) - r q for analytic U, V, q on
    the three-zone grid, n0 = 32, 64, 128 (J = 2).  At points whose stencils
    read only active values the error falls at fourth order (16 per
    halving).  At points whose stencils read ghost values it falls at second
    order (4 per halving): a ghost value is the DD4 interpolant, exact for
    cubics and so off by O(h^4), and the second-derivative stencil divides
    that by 12 h^2.  A ghost fill that is not the DD4 interpolant (zero, the
    nearest value, linear interpolation), a stencil at the wrong spacing or
    a wrong sign leaves an O(1) error at one of the two kinds of points and
    fails."""
    nu, rr = 0.05, 0.3
    e_act, e_gho = [], []
    for n0 in (32, 64, 128):
        J = 2
        cfg = O.Config(n0=n0, J=J, eps=0.0, re=1.0 / nu, rayleigh_r=rr)
        NJ = cfg.NJ
        h, X, Y = _lattice(NJ)
        A, lev = _three_zone_grid(n0, J)
        assert 0.1 < A.mean() < 0.6
        jx, jy = O.stencil_levels(A, lev, J)
        U, V, q, qx, qy, lap = _fields(X, Y)
        Z = np.zeros_like(q)
        fz = O.Frozen(A, jx, jy, U, V, Z, Z, Z, nu, rr)
        got = O.apply_operator(cfg, fz, q[A])
        exact = (-U * qx - V * qy + nu * lap - rr * q)[A]
        err = np.abs(got - exact)
        sel = _reads_ghost(A, jx, jy, J)[A]
        assert 100 < sel.sum() < 0.5 * sel.size
        e_gho.append(err[sel].max())
        e_act.append(err[~sel].max())
    for a, b in zip(e_act, e_act[1:]):
        assert 14.0 < a / b < 18.0, e_act
    for a, b in zip(e_gho, e_gho[1:]):
        assert 3.5 < a / b < 5.0, e_gho
    assert e_act[-1] < 1e-5 and e_gho[-1] < 1e-3


def test_ghost_values_are_fourth_order_interpolants():
    """R(q) at the ghost points of the three-zone grid is the DD4 interpolant
    of the active values: its error against the analytic q falls at fourth
    order (a linear or nearest-point fill would fall at second order or not
    at all)."""
    errs = []
    for n0 in (16, 32, 64):
        J = 2
        NJ = n0 << J
        _, X, Y = _lattice(NJ)
        A, lev = _three_zone_grid(n0, J)
        jx, jy = O.stencil_levels(A, lev, J)
        G = O.ghost_set(A, jx, jy, J)
        assert G.sum() > 0
        q = _fields(X, Y)[2]
        R = O.reconstruct(q, A, J)
        assert np.array_equal(R[A], q[A])
        errs.append(np.abs(R - q)[G].max())
    for a, b in zip(errs, errs[1:]):
        assert 13.0 < a / b < 19.0, errs
