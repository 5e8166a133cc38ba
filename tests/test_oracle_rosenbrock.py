"""Pins of the full-Jacobian exponential Rosenbrock step (Sec. 1 and 2.1:
the Krylov projection with the Jacobian of the discrete right-hand side,
JFNK-style; §8(f) f1): the Jacobian against the exact central difference of
the quadratic right-hand side, the Krylov step against the dense matrix
exponential, and second-order convergence in time (the frozen step is first
order)."""

import numpy as np
import pytest
import scipy.linalg

from oracle import wrc_oracle as O


def _rhs(cfg, A, omega):
    """F(omega) = -U(omega) . grad omega + nu lap omega - r omega at the active
    points of the fixed grid A (no subgrid forcing)."""
    fz = O.freeze(cfg, A, omega)
    return O.apply_operator(cfg, fz, omega[A])


@pytest.mark.parametrize("p,eps", [(2, 0.0), (2, 2e-3), (3, 2e-3)])
def test_jacobian_is_the_exact_derivative_of_the_quadratic_rhs(p, eps):
    """Without subgrid forcing F is quadratic in omega (the velocity is linear
    in omega), so (F(omega + e q) - F(omega - e q)) / (2e) equals J q up to
    rounding, for any e.  Leaving out U[q] . grad omega, or taking the
    velocity of omega for that of q, fails by O(1)."""
    cfg = O.Config(n0=8, J=2, eps=eps, re=200.0, rayleigh_r=0.1, p=p)
    st = O.initial_state(cfg, [-0.6, 0.7], [0.2, -0.4], [1.0, -0.6], [0.45, 0.4])
    A = st.active
    rng = np.random.default_rng(7)
    q = np.zeros_like(st.omega)
    q[A] = rng.standard_normal(int(A.sum()))
    fz = O.freeze(cfg, A, st.omega)
    dwx, dwy = O.vorticity_gradient(cfg, fz, st.omega)
    Jq = O.jacobian_operator(cfg, fz, dwx, dwy, q[A])
    for e in (0.5, 1e-2):
        fd = (_rhs(cfg, A, st.omega + e * q) - _rhs(cfg, A, st.omega - e * q)) / (2 * e)
        assert np.linalg.norm(fd - Jq) <= 1e-10 / e * np.linalg.norm(Jq)
    # the extra term is not negligible: J differs from the frozen operator
    assert np.linalg.norm(Jq - O.apply_operator(cfg, fz, q[A])) > 1e-2 * np.linalg.norm(Jq)


@pytest.mark.parametrize("eps", [0.0, 3e-3])
def test_rosenbrock_krylov_matches_dense_exponential(eps):
    cfg = O.Config(n0=8, J=1, eps=eps, re=50.0, dt=0.05, m=20, scheme="rosenbrock")
    st = O.initial_state(cfg, [-0.7, 0.8], [0.2, -0.5], [1.0, -0.7], [0.6, 0.5])
    fz = O.freeze(cfg, st.active, st.omega)
    om = st.omega[st.active]
    n = om.size
    dwx, dwy = O.vorticity_gradient(cfg, fz, st.omega)
    Jd = np.stack([O.jacobian_operator(cfg, fz, dwx, dwy, e) for e in np.eye(n)], axis=1)
    b = O.apply_operator(cfg, fz, om)
    M = np.zeros((n + 1, n + 1))
    M[:n, :n] = cfg.dt * Jd
    M[:n, n] = cfg.dt * b
    exact = scipy.linalg.expm(M)[:n, n]
    inc, _ = O.arnoldi_phi1(lambda q: O.jacobian_operator(cfg, fz, dwx, dwy, q), b, n, cfg.dt)
    assert np.linalg.norm(inc - exact) <= 1e-10 * np.linalg.norm(exact)
    st1, _ = O.step_rosenbrock(cfg, st)
    new = np.zeros_like(st.omega)
    new[st.active] = om + exact
    A2, om2, _ = O.adapt(cfg, st.active, new)
    assert np.array_equal(st1.active, A2)
    assert np.abs(st1.omega - om2).max() <= 1e-10 * np.abs(om2).max()


def _run(cfg, st, T):
    n = int(round(T / cfg.dt))
    for _ in range(n):
        st, _ = O.advance(cfg, st)
    return st


def test_second_order_in_time_frozen_first_order():
    """A Lamb-Oseen-type vortex advecting a weaker one (uniform 32^2 grid,
    Re = 100, T = 0.4): against the same scheme at dt = 1/160, the Rosenbrock
    error falls by ~4 per halving of dt, the frozen step's by ~2."""
    T = 0.4
    errs = {}
    for scheme in ("rosenbrock", "frozen"):
        base = O.Config(n0=8, J=2, eps=0.0, re=100.0, m=24, scheme=scheme)
        st0 = O.initial_state(base, [0.0, 1.0], [0.0, 0.3], [1.0, 0.4], [0.5, 0.4])
        ref = _run(O.Config(**{**base.__dict__, "dt": T / 64}), st0, T)
        errs[scheme] = []
        for dt in (T / 4, T / 8, T / 16):
            got = _run(O.Config(**{**base.__dict__, "dt": dt}), st0, T)
            errs[scheme].append(np.abs(got.omega - ref.omega).max())
    r = errs["rosenbrock"]
    f = errs["frozen"]
    assert all(3.2 < a / b < 4.8 for a, b in zip(r, r[1:])), r
    assert all(1.6 < a / b < 2.6 for a, b in zip(f, f[1:])), f
    assert r[-1] < 0.2 * f[-1]
