"""Plain FP64 CPU oracle for one Krylov-projected time step of the
Deslauriers-Dubuc (DD) wavelet-collocation solver for filtered 2-D
incompressible flow (Walsh & Alam, "Fujiwhara interaction of tropical cyclone
scale vortices using a weighted residual collocation method").

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this module.  The
library under ``paper_1604_08159_gb300/`` never imports it, and this module
shares no code with the CUDA path (the only shared module is the seeded
parameter generator ``paper_1604_08159_gb300/workloads.py``, which holds none of
the method's arithmetic).

Storage
-------
Every field is a full ``NJ x NJ`` float64 array indexed ``[k, i]`` (row ``k`` is
the y index, column ``i`` the x index) with ``x_i = -pi + i*h``,
``y_k = -pi + k*h``, ``h = 2*pi/NJ`` and ``NJ = N0 * 2**J`` on the doubly
periodic square ``[-pi, pi)^2``.  The adaptive grid is a boolean mask of the
same shape; a compact vector over the grid is ``field[mask]`` (row-major
order).  Points of level ``j`` all lie on the sublattice of stride
``s_j = 2**(J-j)``; most routines below work on such sublattice views
``F[::s, ::s]``, on which the level-``j`` points are those with an odd row or
column index.

What each function follows
--------------------------
``levels``                 Sec. 2.4: nested dyadic meshes G^0 c ... c G^J.
``dd_predictor_weights``   Sec. 2.4: the 2p-point Lagrange predictor of DD order
                           2p (Config.p; 2p = 4 is the default, 6, 8, 10 the
                           higher orders of the Sec. 2.6.2 convergence study).
``dd_scaling_derivative``  Sec. 2.5: phi'(n) at the integers from the
                           refinement relation (eigenvector for 1/2).
``first/second_derivative_integers``
                           Sec. 2.5: the collocation stencils as integers over a
                           common denominator (second derivative: a reading).
``dd_x/dd_y``              Sec. 2.4: DD subdivision along one axis.
``predict_level``          Sec. 2.4: tensor-product DD prediction in 2-D.
``reconstruct``            Eq. 6: u^N evaluated on the finest lattice from the
                           retained coefficients (details of dropped points 0).
``details``                Eq. 6: the coefficient that disappears at the coarser
                           scale, d = u - Pred(u).
``significant``            Eq. 6: epsilon-thresholding, |u - u^N|_inf < eps.
``adjacent_zone``          Sec. 2.4 (2^d - 1 children inserted in the
                           neighbourhood of a node); the rule itself is a
                           reading (the adaptive wavelet collocation zone).
``closure``                Perfect-reconstruction closure of the grid (reading).
``stencil_levels``         Sec. 2.5: the finest spacing at which a point has
                           neighbours (reading).
``ghost_set``              Points outside the grid that the Sec. 2.5 stencils
                           read, with their values from Eq. 6 (reading).
``d1/d2``                  Sec. 2.5: collocation derivatives; the first
                           derivative is the derivative of the DD interpolant at
                           the collocation points (for 2p = 4 the 5-point
                           4th-order central difference); the second-derivative
                           reading is the central stencil of order 2p on 2p + 1
                           points (phi'' is undefined at the integers for 2p = 4
                           and only of order 2p - 2 beyond; Table 1's rates
                           favour order 2p).
``streamfunction``         Poisson solve (the paper is silent): exact inverse of
                           the collocation Laplacian on the periodic finest
                           lattice.
``velocity``               U = dpsi/dy, V = -dpsi/dx.
``strain``, ``smagorinsky_nut``, ``stress_vorticity_forcing``, ``sgs_forcing``
                           Eq. 5: Smagorinsky model, vorticity form of -div(tau).
``apply_operator``         Sec. 2.1/2.5: the frozen linear right-hand side A_n q.
``arnoldi_phi1``           Abstract / Sec. 2.1: projection of the discrete system
                           onto a Krylov subspace (exponential-Euler reading).
``step``                   One full time step followed by grid adaptation.
``jacobian_operator``, ``step_rosenbrock``
                           Sec. 1 / 2.1 (the Krylov projection with the full
                           Jacobian, JFNK-style): the exponential
                           Rosenbrock-Euler step, a Poisson solve per Krylov
                           vector; the subgrid forcing held at t^n (reading).
``scalar_operator``, ``scalar_init``, ``step_with_scalar``
                           Sec. "Transport of water vapor as a passive scalar":
                           the vapour mixing ratio r_v carried by the flow,
                           Eq. (vapour) with only a diffusion term on its
                           right-hand side, advanced by the same Krylov
                           projection on the same adaptive grid, which adapts
                           to both fields (union of their significant sets; a
                           reading: the paper does not spell the joint rule).

Parity pins live in ``tests/test_oracle_*.py`` (closed forms, invariants,
brute force on tiny lattices, the paper's Table 1 convergence rate).  Every
function above is pinned; none is "parity unpinned".
"""

from __future__ import annotations

from dataclasses import dataclass
from fractions import Fraction
from math import gcd

import numpy as np
import scipy.linalg

__all__ = [
    "Config", "State", "StepInfo", "levels", "dd4_x", "dd4_y", "dd_x", "dd_y", "predict_level",
    "dd_predictor_weights", "dd_predictor_integers", "dd_scaling_derivative",
    "first_derivative_integers", "second_derivative_integers", "stencil_reach",
    "level_mask_sub", "reconstruct", "details", "significant", "adjacent_zone",
    "closure", "stencil_levels", "ghost_set", "at", "d1", "d2",
    "adaptive_derivatives", "streamfunction", "velocity", "strain",
    "smagorinsky_nut", "stress_vorticity_forcing", "sgs_forcing", "laplacian_symbol",
    "vortex_field", "Frozen", "freeze", "apply_operator", "arnoldi_phi1",
    "phi1_augmented", "adapt", "initial_state", "state_from_field", "step",
    "diagnostics", "BREAKDOWN_TOL", "scalar_operator", "adapt_two", "scalar_init",
    "step_with_scalar", "vorticity_gradient", "jacobian_operator", "step_rosenbrock", "advance",
]

# Happy-breakdown test of the Arnoldi process: stop when the new direction is
# this small relative to |A v_j| (the Krylov space is then invariant).
BREAKDOWN_TOL = 1e-12


@dataclass
class Config:
    """Run parameters.  ``sgs`` is ``"off"``, ``"apriori"`` (Eq. 5 with a
    constant strain-rate magnitude ``s_apriori``, as the paper does) or
    ``"dynamic"`` (pointwise |S| from the resolved field)."""

    n0: int
    J: int
    eps: float
    re: float
    dt: float = 1e-2
    m: int = 20
    sgs: str = "off"
    cs: float = 0.0
    s_apriori: float = 0.0
    rayleigh_r: float = 0.0
    p: int = 2           # DD order 2p (Sec. 2.4): 2p = 4, 6, 8 or 10
    scheme: str = "frozen"   # "frozen" (exponential Euler, A_n frozen) or "rosenbrock"

    @property
    def NJ(self) -> int:
        return self.n0 << self.J

    @property
    def h(self) -> float:
        return 2.0 * np.pi / self.NJ

    @property
    def nu(self) -> float:
        return 1.0 / self.re

    @property
    def nu_eff(self) -> float:
        """Viscosity inside the linear operator: nu, plus the constant eddy
        viscosity (C_s h_J)^2 |S| of Eq. 5 in the a-priori mode."""
        if self.sgs == "apriori":
            return self.nu + (self.cs * self.h) ** 2 * self.s_apriori
        return self.nu


# --------------------------------------------------------------------------
# A1: lattice and levels (Sec. 2.4)
# --------------------------------------------------------------------------

def levels(n0: int, J: int) -> np.ndarray:
    """Level of every finest-lattice point: 0 on the coarsest mesh (both
    indices multiples of 2^J), else the level j at which the point is first
    inserted, i.e. J - min(t(i), t(k)) with t(i) the number of trailing zero
    bits of i capped at J (t(0) = J)."""
    NJ = n0 << J
    idx = np.arange(NJ)
    t = np.zeros(NJ, dtype=np.int64)
    for b in range(1, J + 1):
        t[idx % (1 << b) == 0] = b
    return (J - np.minimum(t[:, None], t[None, :])).astype(np.int64)


def level_mask_sub(n: int) -> np.ndarray:
    """On a sublattice of stride 2^(J-j), the level-j points are those with an
    odd row or column index."""
    odd = np.arange(n) % 2 == 1
    return odd[None, :] | odd[:, None]


def at(F: np.ndarray, di: int = 0, dk: int = 0) -> np.ndarray:
    """Periodic neighbour access: result[k, i] = F[k + dk, i + di]."""
    return np.roll(F, shift=(-dk, -di), axis=(0, 1))


# --------------------------------------------------------------------------
# DD order 2p: predictor and collocation-derivative weights, derived here
# (Sec. 2.4: the 2p-point Lagrange predictor; Sec. 2.5: derivatives of the
# interpolant at the collocation points)
# --------------------------------------------------------------------------

def _frac_solve(A, b):
    """Exact solution of the square system A x = b over the rationals
    (Gaussian elimination on Fractions; A must be non-singular)."""
    n = len(A)
    M = [[Fraction(v) for v in row] + [Fraction(bv)] for row, bv in zip(A, b)]
    for c in range(n):
        piv = next(r for r in range(c, n) if M[r][c] != 0)
        M[c], M[piv] = M[piv], M[c]
        for r in range(n):
            if r != c and M[r][c] != 0:
                f = M[r][c] / M[c][c]
                M[r] = [a - f * bb for a, bb in zip(M[r], M[c])]
    return [M[r][n] / M[r][r] for r in range(n)]


def _common_denominator(fracs):
    d = 1
    for f in fracs:
        d = d * f.denominator // gcd(d, f.denominator)
    return d


def dd_predictor_weights(p: int):
    """Weights of the order-2p DD predictor (Sec. 2.4): the polynomial of
    degree 2p - 1 through the coarser neighbours at odd offsets
    +-1, +-3, ..., +-(2p - 1) evaluated at 0, as exact rationals; returns the
    weight of the pair at +-(2k - 1), k = 1..p (symmetric)."""
    xs = [2 * k - 1 for k in range(1, p + 1)]
    nodes = [-x for x in reversed(xs)] + xs
    w = []
    for x in xs:
        num, den = Fraction(1), Fraction(1)
        for y in nodes:
            if y != x:
                num *= -y
                den *= x - y
        w.append(num / den)
    return w


def dd_predictor_integers(p: int):
    """The predictor weights as integer numerators over a power of two:
    (c_1..c_p, q) with weight_k = c_k 2^-q (every DD weight has a power-of-two
    denominator)."""
    w = dd_predictor_weights(p)
    d = _common_denominator(w)
    q = d.bit_length() - 1
    assert d == 1 << q
    return [int(x * d) for x in w], q


def _frac_nullvector(A):
    """A vector spanning the null space of A (exact, over the rationals) when
    that null space has dimension one: reduced row echelon form, the free
    column set to 1."""
    rows, cols = len(A), len(A[0])
    M = [[Fraction(v) for v in row] for row in A]
    pivots, r = [], 0
    for c in range(cols):
        piv = next((q for q in range(r, rows) if M[q][c] != 0), None)
        if piv is None:
            continue
        M[r], M[piv] = M[piv], M[r]
        M[r] = [v / M[r][c] for v in M[r]]
        for q in range(rows):
            if q != r and M[q][c] != 0:
                f = M[q][c]
                M[q] = [a - f * b for a, b in zip(M[q], M[r])]
        pivots.append(c)
        r += 1
    free = [c for c in range(cols) if c not in pivots]
    assert len(free) == 1, "null space is not one-dimensional"
    v = [Fraction(0)] * cols
    v[free[0]] = Fraction(1)
    for q, c in enumerate(pivots):
        v[c] = -M[q][free[0]]
    return v


def dd_scaling_derivative(p: int):
    """phi'(n) at the integers for the order-2p DD scaling function: the
    refinement relation phi(x) = sum_k h_k phi(2x - k) (h_0 = 1, h_{+-(2k-1)}
    the predictor weights) differentiated gives v = 2 M v with
    M[n][m] = h_{2n-m}, i.e. the eigenvector of M for 1/2 (its null space of
    2M - I is one-dimensional), normalised by sum_n n phi'(n) = -1 (the
    derivative of sum_n n phi(x - n) = x).  Exact rationals for
    n = 1 .. 2p - 2 (phi' is odd and vanishes at the integers beyond)."""
    w = dd_predictor_weights(p)
    h = {0: Fraction(1)}
    for k, wk in enumerate(w, start=1):
        h[2 * k - 1] = wk
        h[-(2 * k - 1)] = wk
    L = 2 * p - 2
    ns = list(range(-L, L + 1))
    A = []
    for n in ns:
        row = [2 * h.get(2 * n - m, Fraction(0)) for m in ns]
        row[ns.index(n)] -= 1
        A.append(row)
    v = _frac_nullvector(A)
    scale = Fraction(-1) / sum(n * x for n, x in zip(ns, v))
    return [v[ns.index(n)] * scale for n in range(1, L + 1)]


def first_derivative_integers(p: int):
    """The first-derivative stencil of Sec. 2.5 as integers: D u_k =
    (sum_j n_j (u_{k+j} - u_{k-j})) / (d h), j = 1 .. 2p - 2, with
    n_j / d = -phi'(j) (the interpolant's derivative at the collocation point).
    For 2p = 4 this is (8, -1) / 12, the 4th-order central difference."""
    c = [-x for x in dd_scaling_derivative(p)]
    d = _common_denominator(c)
    return [int(x * d) for x in c], d


def second_derivative_integers(p: int):
    """The second-derivative stencil (reading: the central stencil of order
    2p on the 2p + 1 points j = -p..p, exact for polynomials of degree
    2p + 1) as integers: D2 u_k = (n_0 u_k + sum_j n_j (u_{k+j} + u_{k-j})) /
    (d h^2).  For 2p = 4 this is (-30; 16, -1) / 12."""
    pts = list(range(-p, p + 1))
    A = [[Fraction(x) ** r for x in pts] for r in range(len(pts))]
    b = [Fraction(0)] * len(pts)
    b[2] = Fraction(2)
    c = _frac_solve(A, b)
    cs = [c[pts.index(j)] for j in range(0, p + 1)]
    d = _common_denominator(cs)
    return [int(x * d) for x in cs], d


def stencil_reach(p: int) -> int:
    """Largest offset (in units of the stencil spacing) read by the
    derivative stencils of order 2p: 2p - 2 for the first derivative, p for
    the second."""
    return max(2 * p - 2, p)


# --------------------------------------------------------------------------
# A2: DD prediction, reconstruction and details (Sec. 2.4, Eq. 6)
# --------------------------------------------------------------------------

def dd_x(F: np.ndarray, p: int = 2) -> np.ndarray:
    """DD order-2p prediction along x on a sublattice: the polynomial through
    the neighbours at odd offsets +-1 .. +-(2p - 1) evaluated at 0, evaluated
    with integer numerators as s = c_1 (a_1 + b_1), s = s + c_k (a_k + b_k)
    for k = 2..p, then s 2^-q (a_k, b_k the neighbours at -+(2k - 1)).  For
    2p = 4: (9 (a + b) - (c + d)) / 16."""
    c, q = dd_predictor_integers(p)
    acc = float(c[0]) * (at(F, -1) + at(F, 1))
    for k in range(2, p + 1):
        o = 2 * k - 1
        acc = acc + float(c[k - 1]) * (at(F, -o) + at(F, o))
    return acc * (2.0 ** -q)


def dd_y(F: np.ndarray, p: int = 2) -> np.ndarray:
    """As ``dd_x`` along y."""
    c, q = dd_predictor_integers(p)
    acc = float(c[0]) * (at(F, 0, -1) + at(F, 0, 1))
    for k in range(2, p + 1):
        o = 2 * k - 1
        acc = acc + float(c[k - 1]) * (at(F, 0, -o) + at(F, 0, o))
    return acc * (2.0 ** -q)


def dd4_x(F: np.ndarray) -> np.ndarray:
    """DD order-4 prediction along x: weights (-1, 9, 9, -1)/16."""
    return dd_x(F, 2)


def dd4_y(F: np.ndarray) -> np.ndarray:
    """As ``dd4_x`` along y."""
    return dd_y(F, 2)


def predict_level(F: np.ndarray, J: int, j: int, p: int = 2) -> np.ndarray:
    """DD prediction of every level-j point from coarser points.  Returns an
    array on the stride-2^(J-j) sublattice: points odd in x only are predicted
    along x, points odd in y only along y, points odd in both by the tensor
    product (x prediction of the four rows, then y prediction).  Entries at
    even-even sublattice points are not meaningful."""
    s = 1 << (J - j)
    sub = F[::s, ::s]
    n = sub.shape[0]
    odd = np.arange(n) % 2 == 1
    oi, ok = odd[None, :], odd[:, None]
    px = dd_x(sub, p)
    py = dd_y(sub, p)
    pxy = dd_y(px, p)
    return np.where(oi & ~ok, px, np.where(~oi & ok, py, pxy))


def reconstruct(values: np.ndarray, active: np.ndarray, J: int, p: int = 2) -> np.ndarray:
    """R(u) of Eq. 6 on the full finest lattice: the values on the active set,
    and coarse-to-fine DD prediction (detail 0) at every other point."""
    R = np.where(active, values, 0.0)
    for j in range(1, J + 1):
        s = 1 << (J - j)
        P = predict_level(R, J, j, p)
        sub = R[::s, ::s]
        fill = level_mask_sub(sub.shape[0]) & ~active[::s, ::s]
        sub[fill] = P[fill]
    return R


def details(R: np.ndarray, active: np.ndarray, J: int, p: int = 2) -> np.ndarray:
    """Wavelet coefficients d = u - Pred(u) at active points of level >= 1
    (Eq. 6); 0 elsewhere.  ``R`` must hold the values on the active set and on
    the predictor points of every active point (true for a closed grid)."""
    d = np.zeros_like(R)
    for j in range(1, J + 1):
        s = 1 << (J - j)
        P = predict_level(R, J, j, p)
        sub = R[::s, ::s]
        sel = level_mask_sub(sub.shape[0]) & active[::s, ::s]
        dv = d[::s, ::s]
        dv[sel] = (sub - P)[sel]
    return d


# --------------------------------------------------------------------------
# A3: significance, adjacent zone, closure, stencil levels, ghosts
# --------------------------------------------------------------------------

def significant(d: np.ndarray, active: np.ndarray, lev: np.ndarray, eps: float) -> np.ndarray:
    """S = level 0 plus every active point of level >= 1 with |d| >= eps."""
    return (lev == 0) | (active & (lev >= 1) & (np.abs(d) >= eps))


def adjacent_zone(S: np.ndarray, lev: np.ndarray, J: int) -> np.ndarray:
    """S plus its adjacent zone: every significant point of level j >= 1 adds
    the lattice points of level j and j+1 (j+1 <= J) lying within 2^(J-j)
    finest cells of it in both x and y (periodic).  Level 0 adds nothing."""
    A = S.copy()
    for j in range(1, J + 1):
        Sj = S & (lev == j)
        if not Sj.any():
            continue
        s = 1 << (J - j)
        step = s // 2 if j < J else s
        target = (lev == j) | (lev == j + 1)
        offs = range(-s, s + 1, step)
        for dk in offs:
            for di in offs:
                A |= np.roll(Sj, (dk, di), axis=(0, 1)) & target
    return A


def _predictor_marks(src: np.ndarray, p: int = 2) -> np.ndarray:
    """Given a mask of level-j points on their sublattice, mark the DD
    predictor points of each one (odd offsets +-1 .. +-(2p - 1) along x,
    along y, or their 2p x 2p tensor product, according to the point's
    type)."""
    n = src.shape[0]
    odd = np.arange(n) % 2 == 1
    oi, ok = odd[None, :], odd[:, None]
    X = src & oi & ~ok
    Y = src & ~oi & ok
    XY = src & oi & ok
    M = np.zeros_like(src)
    offs = [o for k in range(1, p + 1) for o in (-(2 * k - 1), 2 * k - 1)]
    for a in offs:
        M |= np.roll(X, a, axis=1)
        M |= np.roll(Y, a, axis=0)
        for b in offs:
            M |= np.roll(XY, (b, a), axis=(0, 1))
    return M


def closure(A: np.ndarray, J: int, p: int = 2) -> np.ndarray:
    """Close the grid under DD prediction, finest level first: every point of
    level j in the grid adds its predictor points (all of coarser level), so
    that the grid's values are a valid multiresolution representation."""
    A = A.copy()
    for j in range(J, 0, -1):
        s = 1 << (J - j)
        sub = A[::s, ::s]
        src = sub & level_mask_sub(sub.shape[0])
        sub |= _predictor_marks(src, p)
    return A


def stencil_levels(A: np.ndarray, lev: np.ndarray, J: int):
    """Stencil level j* per axis for each active point P: the largest
    j in [lev(P), J] such that P + h_j e or P - h_j e is active; lev(P) if
    there is none.  Returns (jx, jy), -1 outside the grid."""
    jx = np.where(A, lev, -1)
    jy = jx.copy()
    for j in range(0, J + 1):
        s = 1 << (J - j)
        sA = A[::s, ::s]
        nbx = np.roll(sA, 1, axis=1) | np.roll(sA, -1, axis=1)
        nby = np.roll(sA, 1, axis=0) | np.roll(sA, -1, axis=0)
        vx = jx[::s, ::s]
        vy = jy[::s, ::s]
        vx[sA & nbx] = j
        vy[sA & nby] = j
    return jx, jy


def ghost_set(A: np.ndarray, jx: np.ndarray, jy: np.ndarray, J: int, p: int = 2) -> np.ndarray:
    """Ghost points: the points P +- r h_{j*} e (r = 1 .. stencil_reach(p))
    read by the derivative stencils of an active point P that are not
    active, plus, finest level first, the non-active predictor points of
    every ghost."""
    R = stencil_reach(p)
    G = np.zeros_like(A)
    for j in range(0, J + 1):
        s = 1 << (J - j)
        sx = (A & (jx == j))[::s, ::s]
        sy = (A & (jy == j))[::s, ::s]
        M = np.zeros_like(sx)
        for r in range(1, R + 1):
            for a in (-r, r):
                M |= np.roll(sx, a, axis=1)
                M |= np.roll(sy, a, axis=0)
        gv = G[::s, ::s]
        gv |= M
    G &= ~A
    for j in range(J, 0, -1):
        s = 1 << (J - j)
        gv = G[::s, ::s]
        src = gv & level_mask_sub(gv.shape[0])
        gv |= _predictor_marks(src, p) & ~A[::s, ::s]
    return G


# --------------------------------------------------------------------------
# Collocation derivatives (Sec. 2.5)
# --------------------------------------------------------------------------

def _shift(F, axis, r):
    return at(F, r) if axis == 1 else at(F, 0, r)


def d1(F: np.ndarray, axis: int, h: float, p: int = 2) -> np.ndarray:
    """First derivative with unit (sub)lattice offsets and spacing h, the
    stencil of ``first_derivative_integers``: acc = n_1 (u_{+1} - u_{-1}),
    acc = acc + n_j (u_{+j} - u_{-j}) for j = 2 .., then acc / (d h).  For
    2p = 4: (8 (u_{+1} - u_{-1}) - (u_{+2} - u_{-2})) / (12 h)."""
    n, d = first_derivative_integers(p)
    acc = float(n[0]) * (_shift(F, axis, 1) - _shift(F, axis, -1))
    for j in range(2, len(n) + 1):
        acc = acc + float(n[j - 1]) * (_shift(F, axis, j) - _shift(F, axis, -j))
    return acc / (float(d) * h)


def d2(F: np.ndarray, axis: int, h: float, p: int = 2) -> np.ndarray:
    """Second derivative, the stencil of ``second_derivative_integers``:
    acc = n_p (u_{+p} + u_{-p}), acc = acc + n_j (u_{+j} + u_{-j}) for
    j = p - 1 .. 1, acc = acc + n_0 u, then acc / (d h^2).  For 2p = 4:
    (-(u_{+2} + u_{-2}) + 16 (u_{+1} + u_{-1}) - 30 u) / (12 h^2)."""
    n, d = second_derivative_integers(p)
    acc = float(n[p]) * (_shift(F, axis, p) + _shift(F, axis, -p))
    for j in range(p - 1, 0, -1):
        acc = acc + float(n[j]) * (_shift(F, axis, j) + _shift(F, axis, -j))
    acc = acc + float(n[0]) * F
    return acc / (float(d) * h * h)


def adaptive_derivatives(R: np.ndarray, A: np.ndarray, jx: np.ndarray, jy: np.ndarray,
                         J: int, hJ: float, p: int = 2):
    """Dx, Dy, Dxx, Dyy of the reconstructed field R at active points, each
    along its axis with spacing h_{j*} = h_J 2^(J-j*) (lattice arrays, 0 off
    the grid)."""
    Dx = np.zeros_like(R)
    Dy = np.zeros_like(R)
    Dxx = np.zeros_like(R)
    Dyy = np.zeros_like(R)
    for j in range(0, J + 1):
        s = 1 << (J - j)
        h = hJ * s
        sub = R[::s, ::s]
        sx = (A & (jx == j))[::s, ::s]
        sy = (A & (jy == j))[::s, ::s]
        if sx.any():
            Dx[::s, ::s][sx] = d1(sub, 1, h, p)[sx]
            Dxx[::s, ::s][sx] = d2(sub, 1, h, p)[sx]
        if sy.any():
            Dy[::s, ::s][sy] = d1(sub, 0, h, p)[sy]
            Dyy[::s, ::s][sy] = d2(sub, 0, h, p)[sy]
    return Dx, Dy, Dxx, Dyy


# --------------------------------------------------------------------------
# A4/A5: streamfunction, velocity, Smagorinsky (Eq. 5)
# --------------------------------------------------------------------------

def laplacian_symbol(NJ: int, h: float, p: int = 2) -> np.ndarray:
    """sigma(theta): minus the Fourier symbol of the second-derivative stencil
    at theta = 2 pi n / NJ.  With the stencil's integers (n_0; n_1..n_p) / d
    and n_0 = -2 sum n_j, -(n_0 + 2 sum n_j cos j theta) = 4 sum n_j
    sin^2(j theta / 2), so sigma = 4 sum_j n_j sin^2(j theta / 2) / (d h^2),
    free of the cancellation of the cosine form at small theta.  For 2p = 4
    it is evaluated through the identity 30 - 32 cos t + 2 cos 2t =
    16 s^2 (3 + s^2), s = sin(t/2)."""
    if p == 2:
        s2 = np.sin(np.pi * np.arange(NJ) / NJ) ** 2
        return 16.0 * s2 * (3.0 + s2) / (12.0 * h * h)
    n, d = second_derivative_integers(p)
    t = 2.0 * np.pi * np.arange(NJ) / NJ
    acc = np.zeros(NJ)
    for j in range(1, p + 1):
        acc = acc + float(n[j]) * np.sin(0.5 * j * t) ** 2
    return 4.0 * acc / (float(d) * h * h)


def streamfunction(R: np.ndarray, h: float, p: int = 2) -> np.ndarray:
    """psi with L_h psi = -(R - mean R), L_h the collocation Laplacian of
    order 2p on the periodic lattice, mean(psi) = 0."""
    NJ = R.shape[0]
    sig = laplacian_symbol(NJ, h, p)
    den = sig[:, None] + sig[None, :]
    den[0, 0] = 1.0
    F = np.fft.fft2(R) / den
    F[0, 0] = 0.0
    return np.real(np.fft.ifft2(F))


def velocity(psi: np.ndarray, h: float, p: int = 2):
    """U = dpsi/dy, V = -dpsi/dx (finest-lattice stencils)."""
    return d1(psi, 0, h, p), -d1(psi, 1, h, p)


def strain(psi: np.ndarray, U: np.ndarray, h: float, p: int = 2):
    """Resolved strain of the velocity (U, V) = (psi_y, -psi_x):
    S11 = dU/dx = d2psi/dxdy (= -S22), S12 = (dU/dy + dV/dx)/2 = (psi_yy - psi_xx)/2."""
    return d1(U, 1, h, p), 0.5 * (d2(psi, 0, h, p) - d2(psi, 1, h, p))


def smagorinsky_nut(S11: np.ndarray, S12: np.ndarray, cs: float, h: float) -> np.ndarray:
    """Eq. 5: nu_t = (C_s Delta)^2 |S|, |S| = sqrt(2 S_ij S_ij) = 2 sqrt(S11^2 + S12^2)
    in 2-D incompressible flow, Delta = h_J (the smallest DD scale)."""
    return (cs * h) ** 2 * (2.0 * np.sqrt(S11 * S11 + S12 * S12))


def stress_vorticity_forcing(S11: np.ndarray, S12: np.ndarray, nut: np.ndarray, h: float,
                             p: int = 2) -> np.ndarray:
    """Vorticity of the momentum forcing -d tau_ij/dx_j with tau_ij = -2 nu_t S_ij:
    g = (Dxx - Dyy)(2 nu_t S12) - 4 Dx Dy (nu_t S11)."""
    a = 2.0 * nut * S12
    c = nut * S11
    return d2(a, 1, h, p) - d2(a, 0, h, p) - 4.0 * d1(d1(c, 0, h, p), 1, h, p)


def sgs_forcing(psi: np.ndarray, U: np.ndarray, cs: float, h: float, p: int = 2):
    """Smagorinsky forcing of the vorticity equation with pointwise |S| (Eq. 5).
    Returns (g, nu_t) on the lattice."""
    S11, S12 = strain(psi, U, h, p)
    nut = smagorinsky_nut(S11, S12, cs, h)
    return stress_vorticity_forcing(S11, S12, nut, h, p), nut


def vortex_field(NJ: int, xc, yc, gamma, s) -> np.ndarray:
    """Sum of Gaussian vortices omega = Gamma/(pi s^2) exp(-r^2/s^2) (Sec. 3.1,
    the Lamb-Oseen core), r the minimum-image distance on [-pi, pi)^2."""
    h = 2.0 * np.pi / NJ
    x = -np.pi + h * np.arange(NJ)
    X = x[None, :]
    Y = x[:, None]
    om = np.zeros((NJ, NJ))
    for xc_, yc_, g_, s_ in zip(np.atleast_1d(xc), np.atleast_1d(yc),
                                np.atleast_1d(gamma), np.atleast_1d(s)):
        dx = np.mod(X - xc_ + np.pi, 2.0 * np.pi) - np.pi
        dy = np.mod(Y - yc_ + np.pi, 2.0 * np.pi) - np.pi
        om = om + g_ / (np.pi * s_ * s_) * np.exp(-(dx * dx + dy * dy) / (s_ * s_))
    return om


# --------------------------------------------------------------------------
# A6-A9: frozen operator, Arnoldi, phi_1, update
# --------------------------------------------------------------------------

@dataclass
class Frozen:
    """The linearisation frozen at t^n: grid, stencil levels, velocity and SGS
    forcing at the lattice, effective viscosity and Rayleigh coefficient."""
    A: np.ndarray
    jx: np.ndarray
    jy: np.ndarray
    U: np.ndarray
    V: np.ndarray
    g: np.ndarray
    R: np.ndarray
    psi: np.ndarray
    nu_eff: float
    r: float


def freeze(cfg: Config, A: np.ndarray, omega: np.ndarray) -> Frozen:
    """A4-A5: reconstruct omega, solve for psi, velocities and SGS forcing."""
    lev = levels(cfg.n0, cfg.J)
    jx, jy = stencil_levels(A, lev, cfg.J)
    R = reconstruct(omega, A, cfg.J, cfg.p)
    psi = streamfunction(R, cfg.h, cfg.p)
    U, V = velocity(psi, cfg.h, cfg.p)
    if cfg.sgs == "dynamic":
        g, _ = sgs_forcing(psi, U, cfg.cs, cfg.h, cfg.p)
    else:
        g = np.zeros_like(R)
    return Frozen(A, jx, jy, U, V, g, R, psi, cfg.nu_eff, cfg.rayleigh_r)


def apply_operator(cfg: Config, fz: Frozen, q: np.ndarray) -> np.ndarray:
    """A_n q = -U Dx q - V Dy q + nu_eff (Dxx + Dyy) q - r q at the active
    points (compact vector in, compact vector out); derivatives at each point's
    stencil level with ghost values from the DD reconstruction of q."""
    Q = np.zeros_like(fz.R)
    Q[fz.A] = q
    RQ = reconstruct(Q, fz.A, cfg.J, cfg.p)
    Dx, Dy, Dxx, Dyy = adaptive_derivatives(RQ, fz.A, fz.jx, fz.jy, cfg.J, cfg.h, cfg.p)
    a = fz.A
    return -fz.U[a] * Dx[a] - fz.V[a] * Dy[a] + fz.nu_eff * (Dxx[a] + Dyy[a]) - fz.r * q


def phi1_augmented(H: np.ndarray, dt: float) -> np.ndarray:
    """y = phi_1(dt H) e_1 from the exponential of the augmented matrix
    [[dt H, e_1], [0, 0]] (its last column above the corner)."""
    k = H.shape[0]
    M = np.zeros((k + 1, k + 1))
    M[:k, :k] = dt * H
    M[0, k] = 1.0
    E = scipy.linalg.expm(M)
    return E[:k, k]


@dataclass
class StepInfo:
    beta: float
    k: int               # Krylov dimension used (< m after a happy breakdown)
    h_last: float        # h_{k+1,k}
    H: np.ndarray
    y: np.ndarray


def arnoldi_phi1(matvec, b: np.ndarray, m: int, dt: float):
    """Krylov projection of dt * phi_1(dt A) b: Arnoldi with classical
    Gram-Schmidt applied twice, unweighted l2 inner product over the active
    points, happy breakdown when h_{j+1,j} <= BREAKDOWN_TOL |A v_j|.
    Returns (dt * beta * V_k phi_1(dt H_k) e_1, StepInfo)."""
    n = b.size
    beta = float(np.linalg.norm(b))
    if beta == 0.0:
        return np.zeros(n), StepInfo(0.0, 0, 0.0, np.zeros((0, 0)), np.zeros(0))
    Vb = np.zeros((n, m + 1))
    H = np.zeros((m + 1, m))
    Vb[:, 0] = b / beta
    k = m
    for j in range(m):
        w = matvec(Vb[:, j])
        wn = float(np.linalg.norm(w))
        for _ in range(2):
            c = Vb[:, : j + 1].T @ w
            w = w - Vb[:, : j + 1] @ c
            H[: j + 1, j] += c
        H[j + 1, j] = np.linalg.norm(w)
        if H[j + 1, j] <= BREAKDOWN_TOL * wn:
            k = j + 1
            break
        Vb[:, j + 1] = w / H[j + 1, j]
    y = phi1_augmented(H[:k, :k], dt)
    return dt * beta * (Vb[:, :k] @ y), StepInfo(beta, k, float(H[k, k - 1]), H[: k + 1, :k].copy(), y)


# --------------------------------------------------------------------------
# A10: adaptation, initial state, full step, diagnostics
# --------------------------------------------------------------------------

@dataclass
class State:
    active: np.ndarray
    omega: np.ndarray    # lattice array, meaningful on ``active``
    t: float = 0.0
    nstep: int = 0


def adapt(cfg: Config, active: np.ndarray, omega: np.ndarray):
    """Grid adaptation: details of omega on the current grid, threshold,
    adjacent zone, closure; values at newly added points from the
    reconstruction R(omega) on the current grid.  Returns (A', omega', d)."""
    lev = levels(cfg.n0, cfg.J)
    R = reconstruct(omega, active, cfg.J, cfg.p)
    d = details(R, active, cfg.J, cfg.p)
    S = significant(d, active, lev, cfg.eps)
    A2 = closure(adjacent_zone(S, lev, cfg.J), cfg.J, cfg.p)
    return A2, np.where(A2, R, 0.0), d


def state_from_field(cfg: Config, omega_lattice: np.ndarray) -> State:
    """Initial grid from a field sampled on the full lattice: the full-lattice
    transform, then one thresholding/adaptation pass."""
    full = np.ones(omega_lattice.shape, dtype=bool)
    A, om, _ = adapt(cfg, full, np.asarray(omega_lattice, dtype=np.float64))
    return State(A, om)


def initial_state(cfg: Config, xc, yc, gamma, s) -> State:
    return state_from_field(cfg, vortex_field(cfg.NJ, xc, yc, gamma, s))


def step(cfg: Config, st: State):
    """One Krylov-projected exponential-Euler step,
    omega^{n+1} = omega^n + dt phi_1(dt A_n)(A_n omega^n + g_n),
    followed by grid adaptation.  Returns (new state, StepInfo)."""
    fz = freeze(cfg, st.active, st.omega)
    om = st.omega[st.active]
    b = apply_operator(cfg, fz, om) + fz.g[st.active]
    inc, info = arnoldi_phi1(lambda q: apply_operator(cfg, fz, q), b, cfg.m, cfg.dt)
    new = np.zeros_like(st.omega)
    new[st.active] = om + inc
    A2, om2, _ = adapt(cfg, st.active, new)
    return State(A2, om2, st.t + cfg.dt, st.nstep + 1), info


def vorticity_gradient(cfg: Config, fz: Frozen, omega: np.ndarray):
    """D_x omega, D_y omega at the active points: the collocation derivatives
    of Sec. 2.5 at each point's stencil level, ghost values from R(omega)
    (the gradient the advection term of A_n omega uses)."""
    R = reconstruct(omega, fz.A, cfg.J, cfg.p)
    Dx, Dy, _, _ = adaptive_derivatives(R, fz.A, fz.jx, fz.jy, cfg.J, cfg.h, cfg.p)
    return Dx[fz.A], Dy[fz.A]


def jacobian_operator(cfg: Config, fz: Frozen, dwx: np.ndarray, dwy: np.ndarray, q: np.ndarray) -> np.ndarray:
    """J_n q = A_n q - U[q] D_x omega_n - V[q] D_y omega_n at the active points:
    the derivative of the right-hand side F(omega) = -U(omega) . grad omega
    + nu_eff lap omega - r omega + g at omega_n in the direction q, with
    U[q] = D_y psi[q], V[q] = -D_x psi[q] the velocity of q itself (its
    reconstruction R(q) on the finest lattice, the streamfunction solve, the
    finest-lattice stencils; a Poisson solve per application).  The subgrid
    forcing g is held at t^n (a reading: its derivative is left out)."""
    aq = apply_operator(cfg, fz, q)
    Q = np.zeros_like(fz.R)
    Q[fz.A] = q
    RQ = reconstruct(Q, fz.A, cfg.J, cfg.p)
    psi_q = streamfunction(RQ, cfg.h, cfg.p)
    Uq, Vq = velocity(psi_q, cfg.h, cfg.p)
    a = fz.A
    return aq - Uq[a] * dwx - Vq[a] * dwy


def step_rosenbrock(cfg: Config, st: State):
    """One exponential Rosenbrock-Euler step (the full-Jacobian form of the
    Krylov projection, Sec. 1 and 2.1):
    omega^{n+1} = omega^n + dt phi_1(dt J_n) F(omega^n),
    F(omega^n) = A_n omega^n + g_n (the same b as the frozen step), J_n the
    Jacobian of ``jacobian_operator``; second order in time where g is
    absent.  Followed by grid adaptation.  Returns (new state, StepInfo)."""
    fz = freeze(cfg, st.active, st.omega)
    om = st.omega[st.active]
    b = apply_operator(cfg, fz, om) + fz.g[st.active]
    dwx, dwy = vorticity_gradient(cfg, fz, st.omega)
    inc, info = arnoldi_phi1(lambda q: jacobian_operator(cfg, fz, dwx, dwy, q), b, cfg.m, cfg.dt)
    new = np.zeros_like(st.omega)
    new[st.active] = om + inc
    A2, om2, _ = adapt(cfg, st.active, new)
    return State(A2, om2, st.t + cfg.dt, st.nstep + 1), info


def advance(cfg: Config, st: State):
    """One step of the scheme cfg.scheme: ``step`` (frozen linearisation) or
    ``step_rosenbrock`` (full Jacobian)."""
    return step_rosenbrock(cfg, st) if cfg.scheme == "rosenbrock" else step(cfg, st)


def diagnostics(cfg: Config, st: State) -> dict:
    """Energy E = 1/2 int |U|^2, enstrophy Z = 1/2 int omega^2, palinstrophy
    P = 1/2 int |grad omega|^2 and circulation int omega, by the rectangle rule
    on the reconstructed lattice fields."""
    h = cfg.h
    R = reconstruct(st.omega, st.active, cfg.J, cfg.p)
    psi = streamfunction(R, h, cfg.p)
    U, V = velocity(psi, h, cfg.p)
    gx, gy = d1(R, 1, h, cfg.p), d1(R, 0, h, cfg.p)
    w = h * h
    return {
        "E": 0.5 * w * float(np.sum(U * U + V * V)),
        "Z": 0.5 * w * float(np.sum(R * R)),
        "P": 0.5 * w * float(np.sum(gx * gx + gy * gy)),
        "circulation": w * float(np.sum(R)),
        "n_active": int(st.active.sum()),
    }


# --------------------------------------------------------------------------
# Passive scalar: the vapour mixing ratio with diffusion only (the section on
# the transport of water vapor; Eq. (vapour) with its right-hand side
# replaced by a diffusion term)
# --------------------------------------------------------------------------

def scalar_operator(cfg: Config, fz: Frozen, kappa: float, q: np.ndarray) -> np.ndarray:
    """A_r q = -U Dx q - V Dy q + kappa (Dxx + Dyy) q at the active points: the
    material derivative with the frozen velocity and a diffusion term of
    diffusivity kappa (no Rayleigh friction, no subgrid forcing), derivatives
    as in ``apply_operator``."""
    Q = np.zeros_like(fz.R)
    Q[fz.A] = q
    RQ = reconstruct(Q, fz.A, cfg.J, cfg.p)
    Dx, Dy, Dxx, Dyy = adaptive_derivatives(RQ, fz.A, fz.jx, fz.jy, cfg.J, cfg.h, cfg.p)
    a = fz.A
    return -fz.U[a] * Dx[a] - fz.V[a] * Dy[a] + kappa * (Dxx[a] + Dyy[a])


def adapt_two(cfg: Config, active: np.ndarray, omega: np.ndarray, rv: np.ndarray, rv_whole: bool = False):
    """Grid adaptation driven by both fields: the significant sets of omega
    and of r_v (each from its own details on the grid, or on every lattice
    point for a freshly sampled r_v when ``rv_whole``) are joined, then the
    adjacent zone and the closure; values at the new grid from the
    reconstructions.  Returns (A', omega', r_v')."""
    lev = levels(cfg.n0, cfg.J)
    Rw = reconstruct(omega, active, cfg.J, cfg.p)
    Sw = significant(details(Rw, active, cfg.J, cfg.p), active, lev, cfg.eps)
    if rv_whole:
        full = np.ones_like(active)
        Rr = np.asarray(rv, dtype=np.float64)
        Sr = significant(details(Rr, full, cfg.J, cfg.p), full, lev, cfg.eps)
    else:
        Rr = reconstruct(rv, active, cfg.J, cfg.p)
        Sr = significant(details(Rr, active, cfg.J, cfg.p), active, lev, cfg.eps)
    A2 = closure(adjacent_zone(Sw | Sr, lev, cfg.J), cfg.J, cfg.p)
    return A2, np.where(A2, Rw, 0.0), np.where(A2, Rr, 0.0)


def scalar_init(cfg: Config, st: State, rv_lattice: np.ndarray):
    """Start the passive scalar from a field sampled on the full lattice: one
    joint adaptation of the current omega grid and the sampled field.
    Returns (state on the joint grid, r_v lattice array on it)."""
    A2, om2, rv2 = adapt_two(cfg, st.active, st.omega, rv_lattice, rv_whole=True)
    return State(A2, om2, st.t, st.nstep), rv2


def step_with_scalar(cfg: Config, st: State, rv: np.ndarray, kappa: float):
    """One step of omega (as ``step``) and of r_v with the same frozen
    velocity: r_v^{n+1} = r_v^n + dt phi_1(dt A_r) A_r r_v^n, then the joint
    adaptation.  Returns (new state, new r_v, StepInfo of omega, StepInfo of
    r_v)."""
    fz = freeze(cfg, st.active, st.omega)
    om = st.omega[st.active]
    b = apply_operator(cfg, fz, om) + fz.g[st.active]
    inc, info = arnoldi_phi1(lambda q: apply_operator(cfg, fz, q), b, cfg.m, cfg.dt)
    new = np.zeros_like(st.omega)
    new[st.active] = om + inc
    r = rv[st.active]
    br = scalar_operator(cfg, fz, kappa, r)
    inc_r, info_r = arnoldi_phi1(lambda q: scalar_operator(cfg, fz, kappa, q), br, cfg.m, cfg.dt)
    newr = np.zeros_like(rv)
    newr[st.active] = r + inc_r
    A2, om2, rv2 = adapt_two(cfg, st.active, new, newr)
    return State(A2, om2, st.t + cfg.dt, st.nstep + 1), rv2, info, info_r
