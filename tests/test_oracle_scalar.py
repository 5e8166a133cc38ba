"""Pins of the passive scalar (the vapour mixing ratio with diffusion only,
the paper's section on the transport of water vapor): exact discrete decay of
a Fourier mode without flow, invariance of a constant under any flow, the
reduction to the vorticity equation, brute force against the dense matrix
exponential, and the joint grid adaptation."""

import numpy as np
import scipy.linalg

from oracle import wrc_oracle as O


def _lattice(cfg):
    x = -np.pi + cfg.h * np.arange(cfg.NJ)
    return np.meshgrid(x, x)   # X[k, i] = x_i, Y[k, i] = y_k


def test_fourier_mode_decays_exactly_without_flow():
    # omega = 0: no flow and only the level-0 lattice (eps above every
    # detail).  sin x sin y is an eigenvector of the level-0 operator
    # kappa (Dxx + Dyy) (4th-order 5-point stencils, spacing h0 = 2 pi / N0),
    # so each step multiplies it by exp(2 kappa sigma dt) exactly.
    cfg = O.Config(n0=8, J=2, eps=10.0, re=100.0, dt=0.05, m=10)
    kappa = 0.05
    X, Y = _lattice(cfg)
    st = O.state_from_field(cfg, np.zeros((cfg.NJ, cfg.NJ)))
    r0 = np.sin(X) * np.sin(Y)
    st, rv = O.scalar_init(cfg, st, r0)
    lev = O.levels(cfg.n0, cfg.J)
    assert np.array_equal(st.active, lev == 0)
    h0 = 2.0 * np.pi / cfg.n0
    sigma = (32.0 * np.cos(h0) - 2.0 * np.cos(2.0 * h0) - 30.0) / (12.0 * h0 * h0)
    nsteps = 4
    for _ in range(nsteps):
        st, rv, info, info_r = O.step_with_scalar(cfg, st, rv, kappa)
        assert info_r.k == 1                       # happy breakdown: an eigenvector
    assert np.array_equal(st.active, lev == 0)
    exact = r0 * np.exp(2.0 * kappa * sigma * nsteps * cfg.dt)
    a = st.active
    assert np.abs(rv[a] - exact[a]).max() <= 1e-14


def test_constant_scalar_is_invariant_under_the_flow():
    cfg = O.Config(n0=8, J=2, eps=2e-3, re=200.0, dt=0.05, m=12, sgs="dynamic", cs=0.17)
    st = O.initial_state(cfg, [-0.6, 0.6], [0.0, 0.1], [1.0, 0.8], [0.4, 0.4])
    st, rv = O.scalar_init(cfg, st, np.full((cfg.NJ, cfg.NJ), 0.7))
    for _ in range(3):
        st, rv, _, info_r = O.step_with_scalar(cfg, st, rv, 0.02)
        assert info_r.beta <= 1e-12               # A_r c = 0: nothing to project
    assert np.abs(rv[st.active] - 0.7).max() <= 1e-14


def test_scalar_started_from_omega_follows_omega():
    # No subgrid forcing, no Rayleigh friction, kappa = 1 / Re: A_r is A_n,
    # so r_v started from omega stays equal to it, and the joint grid is
    # omega's own.
    cfg = O.Config(n0=8, J=2, eps=1e-3, re=300.0, dt=0.05, m=14)
    xc, yc, gam, s = [-0.6, 0.6], [0.0, 0.0], [1.0, 0.7], [0.45, 0.45]
    st = O.initial_state(cfg, xc, yc, gam, s)
    ref = O.initial_state(cfg, xc, yc, gam, s)
    st, rv = O.scalar_init(cfg, st, O.vortex_field(cfg.NJ, xc, yc, gam, s))
    assert np.array_equal(st.active, ref.active)
    for _ in range(3):
        st, rv, _, _ = O.step_with_scalar(cfg, st, rv, 1.0 / cfg.re)
        ref, _ = O.step(cfg, ref)
        assert np.array_equal(st.active, ref.active)
        assert np.array_equal(st.omega, ref.omega)
        assert np.array_equal(rv[st.active], st.omega[st.active])


def test_scalar_step_matches_dense_exponential():
    # All points active (eps = 0, J = 1): the Krylov increment of r_v with
    # m = N is dt phi_1(dt A_r) A_r r to rounding, A_r built column by column.
    cfg = O.Config(n0=8, J=1, eps=0.0, re=50.0, dt=0.05, m=20)
    st = O.initial_state(cfg, [-0.7, 0.8], [0.2, -0.5], [1.0, -0.7], [0.6, 0.5])
    X, Y = _lattice(cfg)
    rv = np.tanh(3.0 * Y) + 0.2 * np.cos(X)
    st, rv = O.scalar_init(cfg, st, rv)
    fz = O.freeze(cfg, st.active, st.omega)
    r = rv[st.active]
    n = r.size
    kappa = 0.03
    Ad = np.stack([O.scalar_operator(cfg, fz, kappa, e) for e in np.eye(n)], axis=1)
    b = Ad @ r
    M = np.zeros((n + 1, n + 1))
    M[:n, :n] = cfg.dt * Ad
    M[:n, n] = cfg.dt * b
    exact = scipy.linalg.expm(M)[:n, n]
    inc, info = O.arnoldi_phi1(lambda q: O.scalar_operator(cfg, fz, kappa, q), b, n, cfg.dt)
    assert np.linalg.norm(inc - exact) <= 1e-10 * np.linalg.norm(exact)
    # the operator itself: A_r = A_n with nu -> kappa, r -> 0, against a
    # direct evaluation on a constant-velocity-free part (kappa only)
    fz0 = O.Frozen(fz.A, fz.jx, fz.jy, 0.0 * fz.U, 0.0 * fz.V, fz.g, fz.R, fz.psi, kappa, 0.0)
    assert np.allclose(O.scalar_operator(cfg, fz0, kappa, r), O.apply_operator(cfg, fz0, r), rtol=0, atol=0)


def test_front_refines_the_joint_grid():
    # A sharp r_v front along y = 0 away from the vortices adds points that
    # omega alone would not keep; omega's values are unchanged there and r_v
    # is sampled at the new points.
    cfg = O.Config(n0=8, J=3, eps=1e-3, re=300.0, dt=0.05, m=10)
    st = O.initial_state(cfg, [0.0], [1.5], [1.0], [0.3])
    X, Y = _lattice(cfg)
    front = 0.5 * (1.0 + np.tanh(Y / 0.15))
    st2, rv = O.scalar_init(cfg, st, front)
    assert (st2.active & ~st.active).any()
    assert not (st.active & ~st2.active).any()    # omega's own grid is kept
    R = O.reconstruct(st.omega, st.active, cfg.J)
    assert np.array_equal(st2.omega[st2.active], R[st2.active])
    assert np.array_equal(rv[st2.active], front[st2.active])
