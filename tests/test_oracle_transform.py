"""Pins of the oracle's lattice, DD transform and thresholding (Sec. 2.4, Eq. 6)
against closed forms and properties the paper states."""

import numpy as np
import pytest

from oracle import wrc_oracle as O


def brute_level(i, k, J):
    for j in range(J + 1):
        s = 1 << (J - j)
        if i % s == 0 and k % s == 0:
            return j
    raise AssertionError


@pytest.mark.parametrize("n0,J", [(4, 1), (4, 3), (8, 2), (16, 3)])
def test_levels_counts_and_definition(n0, J):
    lev = O.levels(n0, J)
    NJ = n0 << J
    assert lev.shape == (NJ, NJ)
    # G^0 has N0^2 nodes; each refinement inserts 2^d - 1 = 3 children per node.
    assert (lev == 0).sum() == n0 * n0
    for j in range(1, J + 1):
        assert (lev == j).sum() == 3 * n0 * n0 * 4 ** (j - 1)
    for k in range(0, NJ, max(1, NJ // 16)):
        for i in range(NJ):
            assert lev[k, i] == brute_level(i, k, J)


def _poly_lattice(NJ, h, f):
    x = h * np.arange(NJ)          # unwrapped coordinates 0 .. (NJ-1) h
    X, Y = np.meshgrid(x, x)
    return X, Y, f(X, Y)


def _interior(NJ, J, j, margin_levels=1):
    """Mask of points whose level-j predictor stencil (+-3 s_j) does not cross the periodic seam."""
    s = 1 << (J - j)
    idx = np.arange(NJ)
    ok = (idx - 3 * s >= 0) & (idx + 3 * s < NJ)
    return ok[None, :] & ok[:, None]


def test_dd4_reproduces_bicubics():
    # Sec. 2.4: the DD basis of order 2p reproduces polynomials of degree 2p - 1 = 3;
    # the tensor-product predictor reproduces every x^a y^b with a, b <= 3, so
    # all details of such data vanish (away from the periodic seam).
    n0, J = 16, 3
    NJ = n0 << J
    h = 0.05
    rng = np.random.default_rng(0)
    C = rng.normal(size=(4, 4))
    f = lambda X, Y: sum(C[a, b] * X ** a * Y ** b for a in range(4) for b in range(4))
    X, Y, u = _poly_lattice(NJ, h, f)
    A = np.ones_like(u, dtype=bool)
    d = O.details(u, A, J)
    lev = O.levels(n0, J)
    scale = np.abs(u).max()
    for j in range(1, J + 1):
        sel = (lev == j) & _interior(NJ, J, j)
        assert sel.sum() > 0
        assert np.abs(d[sel]).max() <= 1e-12 * scale


def test_dd4_quartic_detail_closed_form():
    # Interpolation error of the cubic through -3s, -s, s, 3s at 0 for x^4 is
    # prod(0 - x_n) = 9 (s h)^4: a closed form that any wrong weight or offset breaks.
    n0, J = 16, 3
    NJ = n0 << J
    h = 0.03
    lev = O.levels(n0, J)
    for f, axis in ((lambda X, Y: X ** 4, "x"), (lambda X, Y: Y ** 4, "y")):
        X, Y, u = _poly_lattice(NJ, h, f)
        d = O.details(u, np.ones_like(u, dtype=bool), J)
        for j in range(1, J + 1):
            s = 1 << (J - j)
            sub_i = (np.arange(NJ) // s) % 2 == 1
            odd_i = sub_i[None, :] & (np.arange(NJ) % s == 0)[None, :]
            odd_k = sub_i[:, None] & (np.arange(NJ) % s == 0)[:, None]
            sel = (lev == j) & _interior(NJ, J, j)
            expect = 9.0 * (s * h) ** 4
            if axis == "x":
                typ = sel & odd_i          # points predicted along x (x-type and xy-type)
            else:
                typ = sel & odd_k
            other = sel & ~typ
            np.testing.assert_allclose(d[typ], expect, rtol=1e-9, atol=1e-12 * np.abs(u).max())
            assert np.abs(d[other]).max() <= 1e-12 * np.abs(u).max()


def test_reconstruct_interpolates_active_values():
    n0, J = 8, 3
    NJ = n0 << J
    rng = np.random.default_rng(1)
    lev = O.levels(n0, J)
    A = (rng.uniform(size=(NJ, NJ)) < 0.2) | (lev == 0)
    A = O.closure(A, J)
    vals = rng.normal(size=(NJ, NJ))
    R = O.reconstruct(vals, A, J)
    assert np.array_equal(R[A], vals[A])
    # Details of the reconstruction vanish off the grid (detail 0 there, Eq. 6),
    # and on the grid equal those of the values.
    d = O.details(R, np.ones_like(A), J)
    assert np.abs(d[~A & (lev > 0)]).max() <= 1e-12 * np.abs(vals).max()


def test_reconstruct_bicubic_from_coarse_grid():
    # Only G^0 retained: u^N of a bicubic is the bicubic itself away from the seam.
    n0, J = 16, 2
    NJ = n0 << J
    h = 0.04
    rng = np.random.default_rng(2)
    C = rng.normal(size=(4, 4))
    f = lambda X, Y: sum(C[a, b] * X ** a * Y ** b for a in range(4) for b in range(4))
    X, Y, u = _poly_lattice(NJ, h, f)
    lev = O.levels(n0, J)
    A = lev == 0
    R = O.reconstruct(u, A, J)
    # dependency radius: 3 s_1 + 3 s_2 = 6 + 3 fine cells
    idx = np.arange(NJ)
    ok = (idx >= 9) & (idx < NJ - 9)
    inner = ok[None, :] & ok[:, None]
    assert np.abs(R - u)[inner].max() <= 1e-11 * np.abs(u).max()


@pytest.mark.parametrize("eps", [1e-2, 1e-3, 1e-4])
def test_thresholded_reconstruction_error_bound(eps):
    # Eq. 6: keeping the coefficients with |d| >= eps gives |u - u^N|_inf of order eps.
    n0, J = 16, 4
    NJ = n0 << J
    u = O.vortex_field(NJ, [-0.6, 0.6], [0.0, 0.1], [1.0, 0.8], [0.3, 0.25])
    cfg = O.Config(n0=n0, J=J, eps=eps, re=1.0)
    st = O.state_from_field(cfg, u)
    R = O.reconstruct(st.omega, st.active, J)
    err = np.abs(R - u).max()
    assert err <= 4.0 * eps
    assert st.active.sum() < 0.5 * NJ * NJ


def test_zero_threshold_keeps_every_point():
    n0, J = 8, 2
    NJ = n0 << J
    u = O.vortex_field(NJ, [0.3], [-0.2], [1.0], [0.4])
    st = O.state_from_field(O.Config(n0=n0, J=J, eps=0.0, re=1.0), u)
    assert st.active.all()
    assert np.array_equal(st.omega, u)
