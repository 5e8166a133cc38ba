"""Pins of the velocity-Exner oracle (oracle/exner.py; Eqs. 1-2 with the
f-plane Coriolis term and Rayleigh friction): the right-hand side against
closed forms built from the 4th-order stencils' Fourier symbols, a discrete
geostrophic jet and a uniform geostrophic wind that are exact steady states,
the acoustic standing wave of the linearised system (frequency
sigma_1 sqrt(C pi_0)), the Jacobian against the exact central difference of
the quadratic right-hand side, the Krylov step against the dense matrix
exponential, second order in time of the Rosenbrock form (first of the
frozen one), and the joint grid against the single-field grids."""

import numpy as np
import pytest
import scipy.linalg

from oracle import exner as E
from oracle import wrc_oracle as W


def _lattice(NJ):
    h = 2.0 * np.pi / NJ
    x = -np.pi + h * np.arange(NJ)
    return h, x[None, :], x[:, None]


def _symbols(h):
    """Fourier symbols of the 2p = 4 collocation stencils at wavenumber 1:
    D1 sin = s1 cos, D1 cos = -s1 sin, D2 cos = s2 cos (s2 < 0)."""
    s1 = (8.0 * np.sin(h) - np.sin(2.0 * h)) / (6.0 * h)
    s2 = (-2.0 * np.cos(2.0 * h) + 32.0 * np.cos(h) - 30.0) / (12.0 * h * h)
    return s1, s2


def _full(cfg, u, v, p):
    return E.ExnerState(np.ones(u.shape, dtype=bool), u, v, p)


def test_rhs_matches_closed_form_on_trigonometric_fields():
    cfg = E.ExnerConfig(n0=16, J=1, eps=0.0, re=50.0, rayleigh_r=0.05, cpt=3.0, coriolis=0.7, gx=0.3, gy=-0.2)
    h, X, Y = _lattice(cfg.NJ)
    s1, s2 = _symbols(h)
    a, b, c, d, e, p0 = 0.9, -0.6, 0.04, 0.35, -0.03, 1.7
    one = np.ones_like(X + Y)
    u = a * np.cos(Y) + d * np.sin(X)
    v = b * np.cos(X) * one
    p = p0 + c * np.sin(X) + e * np.sin(Y)
    ux, uy = d * s1 * np.cos(X) * one, -a * s1 * np.sin(Y) * one
    vx, vy = -b * s1 * np.sin(X) * one, 0.0 * one
    px, py = c * s1 * np.cos(X) * one, e * s1 * np.cos(Y) * one
    lu, lv = s2 * u, s2 * v
    C, f, r, nu = cfg.cpt, cfg.coriolis, cfg.rayleigh_r, cfg.nu_eff
    Fu = -(u * ux + v * uy) - C * px + f * (v - cfg.gy) - r * u + nu * lu
    Fv = -(u * vx + v * vy) - C * py - f * (u - cfg.gx) - r * v + nu * lv
    Fp = -(u * px + v * py) - p * (ux + vy)
    got = E.exner_rhs(cfg, E.freeze_exner(cfg, _full(cfg, u, v, p)))
    want = E.stack(Fu.ravel(), Fv.ravel(), Fp.ravel())
    assert np.max(np.abs(got - want)) <= 1e-12 * np.max(np.abs(want))


def _vortex_state(cfg, amp=1.0, pi0=1.0, pert=0.0):
    om = W.vortex_field(cfg.NJ, [-0.7, 0.6], [0.1, -0.2], [2.0 * amp, 1.2 * amp], [0.45, 0.5])
    psi = W.streamfunction(om, cfg.h, cfg.p)
    u, v = W.velocity(psi, cfg.h, cfg.p)
    h, X, Y = _lattice(cfg.NJ)
    p = pi0 + pert * np.exp(-((X - 0.3) ** 2 + (Y + 0.4) ** 2) / 0.3) + 0.0 * X * Y
    return u, v, p


def test_frozen_operator_reproduces_the_rhs_on_an_adaptive_grid():
    cfg = E.ExnerConfig(n0=16, J=3, eps=2e-3, re=800.0, cpt=5.0, coriolis=0.6, gx=0.2, gy=0.1, rayleigh_r=0.02)
    st = E.exner_initial_state(cfg, *_vortex_state(cfg, pert=0.01))
    assert 0.05 < st.active.mean() < 0.6
    b = E.freeze_exner(cfg, st)
    n = b.u.size
    g = E.stack(np.full(n, -cfg.coriolis * cfg.gy), np.full(n, cfg.coriolis * cfg.gx), np.zeros(n))
    F = E.exner_rhs(cfg, b)
    AU = E.exner_linear(cfg, b, E.stack(b.u, b.v, b.pi), full=False) + g
    assert np.max(np.abs(AU - F)) <= 1e-12 * np.max(np.abs(F))


@pytest.mark.parametrize("p", [2, 3])
def test_jacobian_is_the_exact_derivative_of_the_quadratic_rhs(p):
    cfg = E.ExnerConfig(n0=16, J=3, eps=2e-3, re=800.0, cpt=5.0, coriolis=0.6, gx=0.2, rayleigh_r=0.02, p=p)
    st = E.exner_initial_state(cfg, *_vortex_state(cfg, pert=0.01))
    A = st.active
    b = E.freeze_exner(cfg, st)
    rng = np.random.default_rng(7)
    q = rng.standard_normal(3 * int(A.sum()))
    jq = E.exner_linear(cfg, b, q, full=True)
    aq = E.exner_linear(cfg, b, q, full=False)
    eps = 1e-3
    Fs = []
    for sgn in (1.0, -1.0):
        du, dv, dp = E.unstack(sgn * eps * q)
        fields = []
        for F, d in zip((st.u, st.v, st.pi), (du, dv, dp)):
            G = F.copy()
            G[A] = F[A] + d
            fields.append(G)
        Fs.append(E.exner_rhs(cfg, E.freeze_exner(cfg, E.ExnerState(A, *fields))))
    cd = (Fs[0] - Fs[1]) / (2.0 * eps)
    assert np.max(np.abs(cd - jq)) <= 1e-8 * np.max(np.abs(jq))
    # the frozen operator misses the terms of the base state's gradients
    assert np.max(np.abs(cd - aq)) > 1e-3 * np.max(np.abs(jq))


def test_discrete_geostrophic_jet_and_uniform_wind_are_steady():
    cfg = E.ExnerConfig(n0=16, J=1, eps=0.0, re=float("inf"), cpt=2.0, coriolis=0.8, gx=0.25,
                        scheme="rosenbrock", m=10, dt=0.1)
    h, X, Y = _lattice(cfg.NJ)
    s1, _ = _symbols(h)
    a, p0 = 0.6, 1.3
    one = np.ones_like(X + Y)
    # a zonal jet on the mean wind G_x, in discrete geostrophic balance:
    # C D_y pi = -f (u - G_x) with the stencil's own derivative of sin y
    u = cfg.gx + a * np.cos(Y) * one
    v = 0.0 * one
    p = p0 - cfg.coriolis * a / (cfg.cpt * s1) * np.sin(Y) * one
    st = _full(cfg, u, v, p)
    F = E.exner_rhs(cfg, E.freeze_exner(cfg, st))
    assert np.max(np.abs(F)) <= 1e-13
    st2, info = E.exner_step(cfg, st)
    for x, y in zip((st.u, st.v, st.pi), (st2.u, st2.v, st2.pi)):
        assert np.max(np.abs(x - y)) <= 1e-13
    # a uniform wind equal to G, with uniform pi, is steady too
    cfg2 = E.ExnerConfig(n0=16, J=1, eps=0.0, re=float("inf"), cpt=2.0, coriolis=0.8, gx=0.25, gy=-0.4)
    st3 = _full(cfg2, cfg2.gx * one, cfg2.gy * one, p0 * one)
    assert np.max(np.abs(E.exner_rhs(cfg2, E.freeze_exner(cfg2, st3)))) == 0.0


@pytest.mark.parametrize("scheme", ["rosenbrock", "frozen"])
def test_acoustic_standing_wave(scheme):
    cfg = E.ExnerConfig(n0=16, J=1, eps=0.0, re=float("inf"), cpt=3.0, scheme=scheme, m=30, dt=0.05)
    h, X, Y = _lattice(cfg.NJ)
    s1, _ = _symbols(h)
    pi0, amp = 2.0, 1e-7
    one = np.ones_like(X + Y)
    st = _full(cfg, 0.0 * one, 0.0 * one, pi0 + amp * np.cos(X) * one)
    nsteps = 12
    for _ in range(nsteps):
        st, _ = E.exner_step(cfg, st)
    t = nsteps * cfg.dt
    w = s1 * np.sqrt(cfg.cpt * pi0)
    want_p = amp * np.cos(w * t) * np.cos(X) * one
    want_u = amp * w / (pi0 * s1) * np.sin(w * t) * np.sin(X) * one
    assert np.max(np.abs((st.pi - pi0) - want_p)) <= 1e-5 * amp
    assert np.max(np.abs(st.u - want_u)) <= 1e-5 * amp * w / (pi0 * s1)
    assert np.max(np.abs(st.v)) <= 1e-12 * amp


def test_krylov_step_matches_dense_matrix_exponential():
    cfg = E.ExnerConfig(n0=4, J=1, eps=0.0, re=40.0, cpt=2.5, coriolis=0.4, rayleigh_r=0.1, scheme="rosenbrock",
                        m=192, dt=0.08)
    h, X, Y = _lattice(cfg.NJ)
    one = np.ones_like(X + Y)
    u = 0.4 * np.sin(Y + 0.3) * one + 0.1 * np.cos(2 * X)
    v = -0.3 * np.cos(X - 0.2) * one
    p = 1.1 + 0.05 * np.sin(X + Y)
    st = _full(cfg, u, v, p)
    b = E.freeze_exner(cfg, st)
    N = 3 * cfg.NJ * cfg.NJ
    Jm = np.zeros((N, N))
    for c in range(N):
        e = np.zeros(N)
        e[c] = 1.0
        Jm[:, c] = E.exner_linear(cfg, b, e, full=True)
    F = E.exner_rhs(cfg, b)
    M = np.zeros((N + 1, N + 1))
    M[:N, :N] = cfg.dt * Jm
    M[:N, N] = F
    inc = cfg.dt * scipy.linalg.expm(M)[:N, N]      # dt phi_1(dt J) F
    st2, info = E.exner_step(cfg, st)
    got = E.stack(st2.u.ravel(), st2.v.ravel(), st2.pi.ravel())
    want = E.stack(u.ravel(), v.ravel(), p.ravel()) + inc
    assert np.max(np.abs(got - want)) <= 1e-10 * np.max(np.abs(inc))


def _advance(cfg, st, T):
    n = int(round(T / cfg.dt))
    for _ in range(n):
        st, _ = E.exner_step(cfg, st)
    return st


def _err(a, b):
    return np.sqrt(sum(np.sum((x - y) ** 2) for x, y in zip((a.u, a.v, a.pi), (b.u, b.v, b.pi))))


def test_rosenbrock_is_second_order_and_frozen_first_order():
    """Self-convergence: |U(dt) - U(dt/2)| / |U(dt/2) - U(dt/4)| tends to 2^order."""
    base = dict(n0=8, J=1, eps=0.0, re=200.0, cpt=4.0, coriolis=0.5, m=30)
    cfg0 = E.ExnerConfig(**base, dt=0.1)
    st0 = _full(cfg0, *_vortex_state(cfg0, amp=0.6, pert=0.02))
    T = 0.2
    for scheme, lo, hi in (("rosenbrock", 3.4, 4.7), ("frozen", 1.7, 2.4)):
        runs = [_advance(E.ExnerConfig(**base, dt=dt, scheme=scheme), st0, T) for dt in (0.1, 0.05, 0.025)]
        ratio = _err(runs[0], runs[1]) / _err(runs[1], runs[2])
        assert lo <= ratio <= hi, (scheme, ratio)


def test_joint_grid_is_the_union_of_the_single_field_grids():
    cfg = E.ExnerConfig(n0=16, J=3, eps=2e-3, re=800.0)
    u, v, p = _vortex_state(cfg, pert=0.05, pi0=1.0)
    one = np.ones_like(u)
    # a single field drives the same grid as the vorticity form's thresholding of it
    Au = E.exner_initial_state(cfg, u, 0.0 * one, one).active
    assert np.array_equal(Au, W.state_from_field(cfg, u).active)
    Ap = E.exner_initial_state(cfg, 0.0 * one, 0.0 * one, p).active
    assert np.array_equal(Ap, W.state_from_field(cfg, p - 1.0).active)
    A = E.exner_initial_state(cfg, u, v, p).active
    Av = W.state_from_field(cfg, v).active
    assert (A >= Au).all() and (A >= Av).all() and (A >= Ap).all()
    lev = W.levels(cfg.n0, cfg.J)
    full = np.ones_like(A)
    S = np.zeros_like(A)
    for F in (u, v, p):
        S |= W.significant(W.details(F, full, cfg.J, cfg.p), full, lev, cfg.eps)
    assert np.array_equal(A, W.closure(W.adjacent_zone(S, lev, cfg.J), cfg.J, cfg.p))
