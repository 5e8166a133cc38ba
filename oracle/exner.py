"""Plain FP64 CPU oracle for the compressible velocity-Exner form of the
model (Eqs. 1-2 with the f-plane Coriolis term and the Rayleigh-friction
reading of Eq. 4), advanced by the same Krylov projection on the same
adaptive Deslauriers-Dubuc collocation grid as the vorticity form.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this module.  It
shares no code with the CUDA path; it reuses the DD machinery of
``oracle/wrc_oracle.py`` (levels, reconstruction, details, thresholding,
closure, stencil levels, collocation derivatives, Arnoldi and phi_1).

The system (readings in capitals are the choices where the paper is silent)
---------------------------------------------------------------------------
State: the velocity (u, v) and the Exner function pi on the doubly periodic
square [-pi, pi)^2, nondimensional.

  d pi / dt = -(u pi_x + v pi_y) - pi (u_x + v_y)                       (Eq. 1)
  d u  / dt = -(u u_x + v u_y) - C pi_x + f (v - G_y) - r u + nu lap u  (Eq. 2)
  d v  / dt = -(u v_x + v v_y) - C pi_y - f (u - G_x) - r v + nu lap v  (Eq. 2)

* Eq. 1 is taken as printed: the Exner function multiplies the divergence
  with coefficient one (the factor R_d / c_v of the textbook form is absorbed
  in the nondimensional scaling).  Linearised about rest (u = 0, pi = pi_0)
  it is an acoustic system with sound speed c = sqrt(C pi_0).
* C is c_p theta_0 of Eq. 2 (``Config.cpt``), f the Coriolis parameter of
  the f-plane (``coriolis``), (G_x, G_y) the mean geostrophic wind
  (``gx``, ``gy``): -eps_ijk f_j (u_k - G_k) with f along z gives
  +f (v - G_y) in the x equation and -f (u - G_x) in the y equation.
* EQ. 4 READING: the balance of surface friction, geostrophic pressure
  gradient, Coriolis force and vertical mixing is represented by Rayleigh
  friction -r u_i (``rayleigh_r``; the paper's 1e-5 s^-1 in its units).
* SUBGRID READING: the a-priori Smagorinsky stress of Eq. 5 with a constant
  |S| (the paper's choice) acts as the constant eddy viscosity
  (C_s h_J)^2 |S| on each velocity component, added to 1/Re
  (``Config.nu_eff``); the part of div(tau) proportional to grad(div u) is
  left out (it needs the mixed derivative d^2/dxdy, which the collocation
  stencils of Sec. 2.5 do not provide on the adaptive grid).  The pointwise
  (dynamic) |S| is not part of this form.

Time step: the same Krylov projection as the vorticity form, on the stacked
vector [u; v; pi] over the active points with the unweighted l2 inner product
(a reading).  ``scheme = "rosenbrock"``: exponential Rosenbrock-Euler with the
exact Jacobian J_n of the discrete right-hand side F (second order);
``scheme = "frozen"``: exponential Euler with the operator A_n whose
coefficients (u, v, pi) are frozen at t^n, F(U^n) = A_n U^n + g with the
constant geostrophic forcing g = (-f G_y, f G_x, 0) (first order).  No
Poisson solve is needed in either.

Grid adaptation: the grid adapts to all three fields: the union of the
significant sets of u, v and pi (each thresholded with the same eps on its
own details), then the adjacent zone and the closure (a reading, as for the
passive scalar).
"""

from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import wrc_oracle as W

__all__ = ["ExnerConfig", "ExnerState", "Base", "freeze_exner", "exner_rhs", "exner_linear",
           "exner_adapt", "exner_initial_state", "exner_vortex_state", "exner_step", "stack", "unstack"]


@dataclass
class ExnerConfig(W.Config):
    """Run parameters of the velocity-Exner form (``sgs`` "off" or "apriori")."""

    cpt: float = 1.0         # C = c_p theta_0 of Eq. 2
    coriolis: float = 0.0    # f of the f-plane
    gx: float = 0.0          # mean geostrophic wind G
    gy: float = 0.0


@dataclass
class ExnerState:
    active: np.ndarray
    u: np.ndarray            # lattice arrays, meaningful on ``active``
    v: np.ndarray
    pi: np.ndarray
    t: float = 0.0
    nstep: int = 0


@dataclass
class Base:
    """The state at t^n on its grid: compact values and their collocation
    first derivatives at the active points (each at its stencil level)."""

    A: np.ndarray
    jx: np.ndarray
    jy: np.ndarray
    u: np.ndarray
    v: np.ndarray
    pi: np.ndarray
    ux: np.ndarray
    uy: np.ndarray
    vx: np.ndarray
    vy: np.ndarray
    px: np.ndarray
    py: np.ndarray
    lu: np.ndarray           # lap u, lap v at the active points
    lv: np.ndarray


def stack(u: np.ndarray, v: np.ndarray, pi: np.ndarray) -> np.ndarray:
    """The Krylov vector [u; v; pi] of compact arrays."""
    return np.concatenate([u, v, pi])


def unstack(x: np.ndarray):
    n = x.size // 3
    return x[:n], x[n:2 * n], x[2 * n:]


def _derivs(cfg: ExnerConfig, A, jx, jy, q: np.ndarray):
    """Dx, Dy, Dxx + Dyy of a compact field at the active points (ghost values
    from its DD reconstruction, derivatives at the stencil levels, Sec. 2.5)."""
    Q = np.zeros(A.shape)
    Q[A] = q
    RQ = W.reconstruct(Q, A, cfg.J, cfg.p)
    Dx, Dy, Dxx, Dyy = W.adaptive_derivatives(RQ, A, jx, jy, cfg.J, cfg.h, cfg.p)
    return Dx[A], Dy[A], Dxx[A] + Dyy[A]


def freeze_exner(cfg: ExnerConfig, st: ExnerState) -> Base:
    """Stencil levels of the grid and the derivatives of the state at t^n."""
    A = st.active
    lev = W.levels(cfg.n0, cfg.J)
    jx, jy = W.stencil_levels(A, lev, cfg.J)
    u, v, p = st.u[A], st.v[A], st.pi[A]
    ux, uy, lu = _derivs(cfg, A, jx, jy, u)
    vx, vy, lv = _derivs(cfg, A, jx, jy, v)
    px, py, _ = _derivs(cfg, A, jx, jy, p)
    return Base(A, jx, jy, u, v, p, ux, uy, vx, vy, px, py, lu, lv)


def exner_rhs(cfg: ExnerConfig, b: Base) -> np.ndarray:
    """F(U^n) at the active points, stacked [F_u; F_v; F_pi] (Eqs. 1-2)."""
    C, f, r, nu = cfg.cpt, cfg.coriolis, cfg.rayleigh_r, cfg.nu_eff
    Fu = -(b.u * b.ux + b.v * b.uy) - C * b.px + f * (b.v - cfg.gy) - r * b.u + nu * b.lu
    Fv = -(b.u * b.vx + b.v * b.vy) - C * b.py - f * (b.u - cfg.gx) - r * b.v + nu * b.lv
    Fp = -(b.u * b.px + b.v * b.py) - b.pi * (b.ux + b.vy)
    return stack(Fu, Fv, Fp)


def exner_linear(cfg: ExnerConfig, b: Base, q: np.ndarray, full: bool) -> np.ndarray:
    """The linear operator on a stacked perturbation q = [du; dv; dpi]:
    the frozen-coefficient operator A_n q (advection by the frozen velocity,
    pressure gradient C grad(dpi), the frozen pi times div(du), Coriolis,
    friction, viscosity) and, with ``full``, the remaining terms of the exact
    Jacobian of F: -(du u_x + dv u_y), -(du v_x + dv v_y),
    -(du pi_x + dv pi_y) - dpi (u_x + v_y)."""
    C, f, r, nu = cfg.cpt, cfg.coriolis, cfg.rayleigh_r, cfg.nu_eff
    du, dv, dp = unstack(q)
    dux, duy, dlu = _derivs(cfg, b.A, b.jx, b.jy, du)
    dvx, dvy, dlv = _derivs(cfg, b.A, b.jx, b.jy, dv)
    dpx, dpy, _ = _derivs(cfg, b.A, b.jx, b.jy, dp)
    Ju = -(b.u * dux + b.v * duy) - C * dpx + f * dv - r * du + nu * dlu
    Jv = -(b.u * dvx + b.v * dvy) - C * dpy - f * du - r * dv + nu * dlv
    Jp = -(b.u * dpx + b.v * dpy) - b.pi * (dux + dvy)
    if full:
        Ju = Ju - (du * b.ux + dv * b.uy)
        Jv = Jv - (du * b.vx + dv * b.vy)
        Jp = Jp - (du * b.px + dv * b.py) - dp * (b.ux + b.vy)
    return stack(Ju, Jv, Jp)


def exner_adapt(cfg: ExnerConfig, active: np.ndarray, fields, whole: bool = False):
    """Grid adaptation driven by the three fields: each field's details on the
    grid (on every lattice point for freshly sampled fields, ``whole``),
    their significant sets joined, adjacent zone, closure; values at the new
    grid from the reconstructions.  Returns (A', [u', v', pi'])."""
    lev = W.levels(cfg.n0, cfg.J)
    base = np.ones_like(active) if whole else active
    S = np.zeros_like(active)
    Rs = []
    for F in fields:
        R = np.asarray(F, dtype=np.float64) if whole else W.reconstruct(F, active, cfg.J, cfg.p)
        S |= W.significant(W.details(R, base, cfg.J, cfg.p), base, lev, cfg.eps)
        Rs.append(R)
    A2 = W.closure(W.adjacent_zone(S, lev, cfg.J), cfg.J, cfg.p)
    return A2, [np.where(A2, R, 0.0) for R in Rs]


def exner_initial_state(cfg: ExnerConfig, u, v, pi) -> ExnerState:
    """Initial grid from fields sampled on the full lattice (one joint
    thresholding of the full-lattice transforms)."""
    A, (u2, v2, p2) = exner_adapt(cfg, np.ones(np.shape(u), dtype=bool), [u, v, pi], whole=True)
    return ExnerState(A, u2, v2, p2)


def exner_vortex_state(cfg: ExnerConfig, xc, yc, gamma, s, pi0: float) -> ExnerState:
    """Initial state of Gaussian vortices in the velocity form: the vortex
    field of Sec. 3.1 sampled on the lattice, its streamfunction (exact
    inverse of the collocation Laplacian), u = D_y psi, v = -D_x psi on the
    finest lattice, pi = pi0 everywhere; then the joint thresholding."""
    om = W.vortex_field(cfg.NJ, xc, yc, gamma, s)
    psi = W.streamfunction(om, cfg.h, cfg.p)
    u, v = W.velocity(psi, cfg.h, cfg.p)
    return exner_initial_state(cfg, u, v, np.full_like(u, float(pi0)))


def exner_step(cfg: ExnerConfig, st: ExnerState):
    """One Krylov-projected step of the velocity-Exner system,
    U^{n+1} = U^n + dt phi_1(dt M) F(U^n), M = J_n (``rosenbrock``) or A_n
    (``frozen``), then the joint grid adaptation.  Returns (state, StepInfo)."""
    b = freeze_exner(cfg, st)
    rhs = exner_rhs(cfg, b)
    full = cfg.scheme == "rosenbrock"
    inc, info = W.arnoldi_phi1(lambda q: exner_linear(cfg, b, q, full), rhs, cfg.m, cfg.dt)
    du, dv, dp = unstack(inc)
    A = st.active
    new = []
    for F, d in zip((st.u, st.v, st.pi), (du, dv, dp)):
        G = np.zeros_like(F)
        G[A] = F[A] + d
        new.append(G)
    A2, (u2, v2, p2) = exner_adapt(cfg, A, new)
    return ExnerState(A2, u2, v2, p2, st.t + cfg.dt, st.nstep + 1), info
