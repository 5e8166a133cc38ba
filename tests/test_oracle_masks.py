"""Brute-force pins of the adaptive index sets: each rule is enumerated point by
point with explicit periodic coordinates on tiny lattices and compared with the
oracle's array formulation, plus the structural invariants the sets must have."""

import itertools

import numpy as np
import pytest

from oracle import wrc_oracle as O


def lev_of(i, k, J):
    for j in range(J + 1):
        s = 1 << (J - j)
        if i % s == 0 and k % s == 0:
            return j


def pdist(a, b, n):
    d = abs(a - b) % n
    return min(d, n - d)


def predictor_points(i, k, J, NJ, p=2):
    """Coordinates of the DD predictor points (order 2p) of a level >= 1
    point: odd multiples of its level's spacing, up to (2p - 1)."""
    j = lev_of(i, k, J)
    s = 1 << (J - j)
    oi, ok = (i // s) % 2 == 1, (k // s) % 2 == 1
    offs = [o * s for o in range(-(2 * p - 1), 2 * p, 2)]
    if oi and not ok:
        return [((i + o) % NJ, k) for o in offs]
    if ok and not oi:
        return [(i, (k + o) % NJ) for o in offs]
    return [((i + a) % NJ, (k + b) % NJ) for a in offs for b in offs]


def brute_adjacent(S, J, NJ):
    out = S.copy()
    pts = [(i, k) for k in range(NJ) for i in range(NJ)]
    for (i, k) in pts:
        if not S[k, i]:
            continue
        j = lev_of(i, k, J)
        if j == 0:
            continue
        r = 1 << (J - j)
        for (qi, qk) in pts:
            if pdist(qi, i, NJ) <= r and pdist(qk, k, NJ) <= r and lev_of(qi, qk, J) in (j, j + 1):
                out[qk, qi] = True
    return out


def brute_closure(A, J, NJ, p=2):
    A = A.copy()
    for j in range(J, 0, -1):
        for k in range(NJ):
            for i in range(NJ):
                if A[k, i] and lev_of(i, k, J) == j:
                    for (pi, pk) in predictor_points(i, k, J, NJ, p):
                        A[pk, pi] = True
    return A


def brute_stencil_levels(A, J, NJ):
    jx = np.full(A.shape, -1)
    jy = np.full(A.shape, -1)
    for k in range(NJ):
        for i in range(NJ):
            if not A[k, i]:
                continue
            l = lev_of(i, k, J)
            jx[k, i] = jy[k, i] = l
            for j in range(J, l - 1, -1):
                s = 1 << (J - j)
                if A[k, (i + s) % NJ] or A[k, (i - s) % NJ]:
                    jx[k, i] = j
                    break
            for j in range(J, l - 1, -1):
                s = 1 << (J - j)
                if A[(k + s) % NJ, i] or A[(k - s) % NJ, i]:
                    jy[k, i] = j
                    break
    return jx, jy


def brute_ghosts(A, jx, jy, J, NJ, p=2):
    # the first-derivative stencil of order 2p reads 2p - 2 points each side,
    # the second-derivative one p
    reach = max(2 * p - 2, p)
    G = np.zeros_like(A)
    for k in range(NJ):
        for i in range(NJ):
            if not A[k, i]:
                continue
            sx, sy = 1 << (J - jx[k, i]), 1 << (J - jy[k, i])
            for o in [q for q in range(-reach, reach + 1) if q]:
                for (qi, qk) in (((i + o * sx) % NJ, k), (i, (k + o * sy) % NJ)):
                    if not A[qk, qi]:
                        G[qk, qi] = True
    for j in range(J, 0, -1):
        for k in range(NJ):
            for i in range(NJ):
                if G[k, i] and lev_of(i, k, J) == j:
                    for (pi, pk) in predictor_points(i, k, J, NJ, p):
                        if not A[pk, pi]:
                            G[pk, pi] = True
    return G


def random_significance(n0, J, frac, seed):
    NJ = n0 << J
    rng = np.random.default_rng(seed)
    lev = O.levels(n0, J)
    S = (rng.uniform(size=(NJ, NJ)) < frac) | (lev == 0)
    return S, lev


@pytest.mark.parametrize("n0,J,frac,seed,p", [(4, 2, 0.05, 0, 2), (4, 2, 0.2, 1, 2), (4, 3, 0.02, 2, 2),
                                               (8, 2, 0.03, 3, 2), (8, 2, 0.02, 7, 3), (16, 2, 0.01, 8, 4)])
def test_adjacent_and_closure_match_brute_force(n0, J, frac, seed, p):
    NJ = n0 << J
    S, lev = random_significance(n0, J, frac, seed)
    adj = O.adjacent_zone(S, lev, J)
    assert np.array_equal(adj, brute_adjacent(S, J, NJ))
    A = O.closure(adj, J, p)
    assert np.array_equal(A, brute_closure(adj, J, NJ, p))


@pytest.mark.parametrize("n0,J,frac,seed,p", [(4, 2, 0.05, 4, 2), (4, 3, 0.03, 5, 2), (8, 2, 0.1, 6, 2),
                                               (8, 2, 0.02, 9, 3), (16, 2, 0.01, 10, 4)])
def test_stencil_levels_and_ghosts_match_brute_force(n0, J, frac, seed, p):
    NJ = n0 << J
    S, lev = random_significance(n0, J, frac, seed)
    A = O.closure(O.adjacent_zone(S, lev, J), J, p)
    jx, jy = O.stencil_levels(A, lev, J)
    bx, by = brute_stencil_levels(A, J, NJ)
    assert np.array_equal(jx, bx) and np.array_equal(jy, by)
    G = O.ghost_set(A, jx, jy, J, p)
    assert np.array_equal(G, brute_ghosts(A, jx, jy, J, NJ, p))


def test_grid_invariants_on_vortex_pair():
    cfg = O.Config(n0=16, J=3, eps=1e-3, re=5000.0)
    st = O.initial_state(cfg, [-0.6, 0.6], [0.0, 0.0], [1.0, 1.0], [0.3, 0.3])
    A = st.active
    NJ = cfg.NJ
    lev = O.levels(cfg.n0, cfg.J)
    assert A[lev == 0].all()
    # closed under prediction
    for (k, i) in zip(*np.nonzero(A & (lev > 0))):
        for (pi, pk) in predictor_points(i, k, cfg.J, NJ):
            assert A[pk, pi]
    jx, jy = O.stencil_levels(A, lev, cfg.J)
    G = O.ghost_set(A, jx, jy, cfg.J)
    assert not (G & A).any()
    AG = A | G
    for (k, i) in zip(*np.nonzero(A)):
        sx, sy = 1 << (cfg.J - jx[k, i]), 1 << (cfg.J - jy[k, i])
        for o in (-2, -1, 1, 2):
            assert AG[k, (i + o * sx) % NJ] and AG[(k + o * sy) % NJ, i]
    for (k, i) in zip(*np.nonzero(G)):
        for (pi, pk) in predictor_points(i, k, cfg.J, NJ):
            assert AG[pk, pi]
