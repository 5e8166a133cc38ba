"""Pins of the higher DD orders 2p = 6, 8, 10 (Sec. 2.4 predictor, Sec. 2.5
collocation derivatives, Sec. 2.6.2 Table 1 convergence study): the
predictor's polynomial reproduction and its leading error term, the
derivative of the DD scaling function at the integers against the limit of
the subdivision scheme itself (an independent route to the same numbers),
the stencils' exactness and convergence orders, Table 1's rows, the
adaptive transform, and the Krylov step on order-2p grids (dense brute
force, exact Taylor-Green decay with the order-2p symbol)."""

import os
from fractions import Fraction

import numpy as np
import pytest
import scipy.linalg

from oracle import wrc_oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
ORDERS = (2, 3, 4, 5)


def _dfact2(n):
    r = 1
    while n > 1:
        r *= n
        n -= 2
    return r


@pytest.mark.parametrize("p", ORDERS)
def test_predictor_reproduces_polynomials_of_degree_2p_minus_1(p):
    """Details vanish for polynomials of degree <= 2p - 1 (non-periodic
    harness: interior points only); for x^(2p) the detail at spacing h is
    (-1)^p ((2p - 1)!!)^2 h^(2p) (the Lagrange remainder at 0 with nodes
    +-1, +-3, ..)."""
    h = 0.1
    x = h * (np.arange(41) - 20)
    F = np.tile(x, (3, 1))
    cut = 2 * p
    for deg in range(2 * p):
        f = F ** deg
        pred = O.dd_x(f, p)
        assert np.abs(pred - f)[:, cut:-cut].max() <= 1e-13 * max(1.0, np.abs(f).max())
    f = F ** (2 * p)
    det = (f - O.dd_x(f, p))[:, cut:-cut]
    expect = (-1) ** p * _dfact2(2 * p - 1) ** 2 * h ** (2 * p)
    np.testing.assert_allclose(det, expect, rtol=1e-6)


@pytest.mark.parametrize("p", ORDERS)
def test_predictor_weights_are_powers_of_two_denominators_summing_to_one(p):
    w = O.dd_predictor_weights(p)
    assert 2 * sum(w) == 1
    c, q = O.dd_predictor_integers(p)
    assert all(Fraction(ci, 1 << q) == wi for ci, wi in zip(c, w))


def _cascade_phi(p, K):
    """The DD scaling function on the grid 2^-K Z by K rounds of the
    subdivision scheme itself, started from the unit impulse (an
    independent route: no eigenproblem)."""
    w = [float(x) for x in O.dd_predictor_weights(p)]
    L = 2 * p - 1
    v = np.zeros(2 * L + 1)
    v[L] = 1.0                         # values at the integers -L..L
    pad = 4 * p
    for _ in range(K):
        a = np.concatenate([np.zeros(pad), v, np.zeros(pad)])
        n = a.size
        out = np.zeros(2 * n - 1)
        out[0::2] = a
        for i in range(n - 1):         # midpoint between a[i] and a[i+1]
            acc = 0.0
            for k in range(1, p + 1):
                lo, hi = i - (k - 1), i + k
                if lo >= 0 and hi < n:
                    acc += w[k - 1] * (a[lo] + a[hi])
            out[2 * i + 1] = acc
        v = out
    return v


@pytest.mark.parametrize("p", (2, 3, 4))
def test_phi_prime_at_integers_matches_the_subdivision_limit(p):
    """phi'(n) from the refinement eigenvector against a centred difference
    of the subdivision limit sampled at spacing 2^-K (K = 9): agreement to
    the difference's own O(2^-2K) error plus the limit's approximation
    error."""
    K = 9
    v = _cascade_phi(p, K)
    c = v.size // 2                    # x = 0
    hh = 2.0 ** -K
    dphi = O.dd_scaling_derivative(p)
    for n, exact in enumerate(dphi, start=1):
        i = c + n * (1 << K)
        num = (v[i + 1] - v[i - 1]) / (2 * hh)
        assert abs(num - float(exact)) < 2e-4, (p, n, num, float(exact))
    # and phi' vanishes at the integers beyond 2p - 2
    i = c + (2 * p - 1) * (1 << K)
    assert abs((v[i + 1] - v[i - 1]) / (2 * hh)) < 2e-4


@pytest.mark.parametrize("p", (2, 3, 4))
def test_first_derivative_is_the_derivative_of_the_interpolant(p):
    """Sec. 2.5: the first derivative at a collocation point is the
    derivative there of the DD interpolant of the data.  Random periodic
    data on 16 points are refined K = 9 times by the subdivision scheme
    (periodically, with the predictor weights alone); a centred difference
    of the refined values at the coarse points matches d1 of the data to
    the difference's O(4^-K) error.  Any other first-derivative stencil of
    the same order (e.g. the central difference of order 2p) differs by
    O(1) on such data."""
    rng = np.random.default_rng(p)
    u = rng.standard_normal(16)
    w = [float(x) for x in O.dd_predictor_weights(p)]
    v = u.copy()
    K = 9
    for _ in range(K):
        mid = np.zeros_like(v)
        for k in range(1, p + 1):
            mid += w[k - 1] * (np.roll(v, k - 1) + np.roll(v, -k))
        out = np.empty(2 * v.size)
        out[0::2] = v
        out[1::2] = mid
        v = out
    hh = 1.0 / (1 << K)                # coarse spacing 1
    num = (np.roll(v, -1) - np.roll(v, 1))[0::(1 << K)] / (2 * hh)
    ours = O.d1(u[None, :], 1, 1.0, p)[0]
    assert np.abs(num - ours).max() < 1e-3 * np.abs(ours).max()


@pytest.mark.parametrize("p", ORDERS)
def test_stencils_exact_on_polynomials(p):
    """The first-derivative stencil is exact for degree <= 2p (the
    interpolant reproduces degree 2p - 1, the odd stencil kills the next
    even term), the second-derivative stencil for degree <= 2p + 1."""
    h = 0.05
    x = h * (np.arange(80) - 40)
    F = np.tile(x, (3, 1))
    cut = 2 * p
    for deg in range(2 * p + 1):
        f = F ** deg
        df = deg * F ** (deg - 1) if deg else 0 * F
        assert np.abs(O.d1(f, 1, h, p) - df)[:, cut:-cut].max() <= 1e-8 * max(1.0, np.abs(f).max())
    for deg in range(2 * p + 2):
        f = F ** deg
        d2f = deg * (deg - 1) * F ** (deg - 2) if deg >= 2 else 0 * F
        assert np.abs(O.d2(f, 1, h, p) - d2f)[:, cut:-cut].max() <= 1e-6 * max(1.0, np.abs(f).max())
    # and not beyond: degree 2p + 1 for the first derivative
    f = F ** (2 * p + 1)
    assert np.abs(O.d1(f, 1, h, p) - (2 * p + 1) * F ** (2 * p))[:, cut:-cut].max() > 1e-10


@pytest.mark.parametrize("p", (3, 4))
def test_periodic_convergence_order_2p(p):
    errs = []
    for NJ in (32, 64):
        h = 2 * np.pi / NJ
        x = -np.pi + h * np.arange(NJ)
        X, Y = np.meshgrid(x, x)
        f = np.sin(2 * X) * np.cos(3 * Y)
        e1 = np.abs(O.d1(f, 1, h, p) - 2 * np.cos(2 * X) * np.cos(3 * Y)).max()
        e2 = np.abs(O.d2(f, 0, h, p) + 9 * f).max()
        errs.append((e1, e2))
    r = 2.0 ** (2 * p)
    assert 0.8 * r < errs[0][0] / errs[1][0] < 1.2 * r
    assert 0.8 * r < errs[0][1] / errs[1][1] < 1.2 * r


def _table1():
    rows = {}
    with open(os.path.join(GOLDEN, "table1_dd.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                tp, n, e = line.split()
                rows.setdefault(int(tp), []).append((int(n), float(e)))
    return rows


def _table1_ours(p, ns):
    def uv(X, Y):
        r2 = X * X + Y * Y
        f = np.where(r2 > 0, (1 - np.exp(-r2)) / (2 * np.pi * np.where(r2 > 0, r2, 1.0)), 1 / (2 * np.pi))
        return -Y * f, X * f
    out = []
    cut = 2 * O.stencil_reach(p)
    for n in ns:
        x = np.linspace(-4.0, 4.0, n)
        h = x[1] - x[0]
        X, Y = np.meshgrid(x, x)
        u, v = uv(X, Y)
        om = O.d1(v, 1, h, p) - O.d1(u, 0, h, p)
        lap = O.d2(om, 1, h, p) + O.d2(om, 0, h, p)
        r2 = X * X + Y * Y
        exact = (4 * r2 - 4) * np.exp(-r2) / np.pi
        out.append(np.abs(lap - exact)[cut:-cut, cut:-cut].max())
    return out


@pytest.mark.parametrize("p", (3, 4, 5))
def test_table1_higher_order_rows(p):
    """Table 1 rows 2p = 6, 8, 10 on the [-4, 4]^2 reading of the unstated
    domain (which reproduces the 2p = 4 row within 10%).  The higher rows
    are not matched in absolute value by any stencil reading tried (see the
    design notes); what is pinned is that our errors are no larger than the
    paper's and shrink at least as fast as the paper's row before either
    side meets its rounding floor (N = 65 -> 129).  Only the sizes where
    the paper's error is above 1e-9 are compared: below that both sides sit
    on rounding floors of their own (ours ~1e-10 on this harness)."""
    rows = [r for r in _table1()[2 * p] if r[1] > 1e-9]
    assert len(rows) >= 2
    ours = _table1_ours(p, [n for n, _ in rows])
    for (n, paper), e in zip(rows, ours):
        assert e <= 1.05 * paper, (2 * p, n, e, paper)
    assert ours[0] / ours[1] >= 0.95 * rows[0][1] / rows[1][1]
    assert ours[0] / ours[1] > 2.0 ** (2 * p) * 0.7      # order 2p on the smooth part


@pytest.mark.parametrize("p", (3, 4))
def test_reconstruction_interpolates_and_compresses(p):
    """R(u) is the identity at active points; with threshold eps the
    compressed reconstruction of a smooth field is within a few eps of it
    (Eq. 6), and the grid is closed under the order-2p predictor."""
    cfg = O.Config(n0=16, J=3, eps=1e-4, re=100.0, p=p)
    field = O.vortex_field(cfg.NJ, [-0.6, 0.6], [0.0, 0.1], [1.0, 0.8], [0.35, 0.35])
    st = O.state_from_field(cfg, field)
    A = st.active
    assert A.mean() < 0.6
    R = O.reconstruct(st.omega, A, cfg.J, p)
    assert np.array_equal(R[A], field[A])
    assert np.abs(R - field).max() <= 8 * cfg.eps
    assert np.array_equal(O.closure(A, cfg.J, p), A)


def test_higher_order_grids_are_smaller_for_smooth_fields():
    """For a smooth field, fewer details exceed eps at higher order (the
    predictor is exact to a higher degree): the grids shrink with p."""
    sizes = []
    for p in (2, 3, 4):
        cfg = O.Config(n0=16, J=3, eps=1e-5, re=100.0, p=p)
        field = O.vortex_field(cfg.NJ, [-0.6, 0.6], [0.0, 0.1], [1.0, 0.8], [0.4, 0.4])
        S = O.significant(O.details(field, np.ones_like(field, dtype=bool), cfg.J, p),
                          np.ones_like(field, dtype=bool), O.levels(cfg.n0, cfg.J), cfg.eps)
        sizes.append(int(S.sum()))
    assert sizes[0] > sizes[1] > sizes[2]


def _dense_operator(cfg, fz, n):
    return np.stack([O.apply_operator(cfg, fz, e) for e in np.eye(n)], axis=1)


@pytest.mark.parametrize("p,eps", [(3, 0.0), (3, 3e-3), (4, 3e-3)])
def test_krylov_step_matches_dense_exponential_higher_order(p, eps):
    cfg = O.Config(n0=8, J=1, eps=eps, re=50.0, dt=0.05, m=20, p=p, sgs="dynamic", cs=0.17)
    st = O.initial_state(cfg, [-0.7, 0.8], [0.2, -0.5], [1.0, -0.7], [0.6, 0.5])
    fz = O.freeze(cfg, st.active, st.omega)
    om = st.omega[st.active]
    n = om.size
    Ad = _dense_operator(cfg, fz, n)
    b = Ad @ om + fz.g[st.active]
    M = np.zeros((n + 1, n + 1))
    M[:n, :n] = cfg.dt * Ad
    M[:n, n] = cfg.dt * b
    exact = scipy.linalg.expm(M)[:n, n]
    full, _ = O.arnoldi_phi1(lambda q: O.apply_operator(cfg, fz, q), b, n, cfg.dt)
    assert np.linalg.norm(full - exact) <= 1e-10 * np.linalg.norm(exact)


@pytest.mark.parametrize("p", (3, 4))
def test_taylor_green_exact_decay_with_order_2p_symbol(p):
    """omega = 2 sin x sin y on the full grid decays as
    exp(-2 nu sigma_p(h) t), sigma_p the order-2p Laplacian symbol at
    theta = h, written here from the stencil's weights as
    -(c_0 + 2 sum_j c_j cos(j h)) / h^2 (the cosine form; the oracle uses
    the sine-squared identity)."""
    cfg = O.Config(n0=8, J=2, eps=0.0, re=20.0, dt=0.05, m=10, p=p)
    NJ, h = cfg.NJ, cfg.h
    x = -np.pi + h * np.arange(NJ)
    X, Y = np.meshgrid(x, x)
    om0 = 2 * np.sin(X) * np.sin(Y)
    st = O.state_from_field(cfg, om0)
    assert st.active.all()
    for _ in range(3):
        st, info = O.step(cfg, st)
        # the start vector is an eigenvector: the first Arnoldi residual is
        # at rounding level (with the wide stencils' large integer weights it
        # sits near the 1e-12 breakdown threshold, so the process may or may
        # not stop at k = 1; the result is the same)
        assert abs(info.H[1, 0]) <= 1e-11 * abs(info.H[0, 0])
    n, d = O.second_derivative_integers(p)
    sig = -(n[0] + 2 * sum(n[j] * np.cos(j * h) for j in range(1, p + 1))) / (d * h * h)
    exact = om0 * np.exp(-2 * cfg.nu * sig * 3 * cfg.dt)
    assert np.abs(st.omega - exact).max() <= 1e-13
