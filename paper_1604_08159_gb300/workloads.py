"""Seeded synthetic workloads: run parameters and vortex parameter draws.

This module only draws numbers.  It holds none of the method's arithmetic
(no field sampling, no transform, no stencil), so both the CUDA path and the
CPU oracle may take their inputs from it.

The draws stand in for the paper's cyclone experiments (Sec. 3.2: an equal
Gaussian pair at Re = 5000; Sec. 3.3: unequal pairs at Re = 37440), whose
observational and DNS data are not available: every input here is synthetic.
"""

from __future__ import annotations

from dataclasses import dataclass, field, asdict

import numpy as np

SGS_OFF, SGS_APRIORI, SGS_DYNAMIC = 0, 1, 2
SCHEME_FROZEN, SCHEME_ROSENBROCK = 0, 1
MODEL_VORTICITY, MODEL_EXNER = 0, 1
PREC_FP64, PREC_MIXED = 0, 1


@dataclass
class RunParams:
    """Parameters of one run (mirrors ``wrc_config`` in include/wrc.h)."""
    n0: int
    J: int
    eps: float
    re: float
    dt: float = 1e-2
    m: int = 20
    sgs: int = SGS_OFF
    cs: float = 0.0
    s_apriori: float = 0.0
    rayleigh_r: float = 0.0
    prec: int = PREC_FP64
    p: int = 2              # half the DD order 2p (2p = 4, 6, 8)
    scheme: int = 0         # 0: frozen linearisation, 1: exponential Rosenbrock (full Jacobian)
    model: int = MODEL_VORTICITY   # 1: the compressible velocity-Exner form (Eqs. 1-2)
    cpt: float = 0.0        # velocity-Exner form: C = c_p theta_0, Coriolis f, geostrophic wind G
    coriolis: float = 0.0
    gx: float = 0.0
    gy: float = 0.0

    @property
    def NJ(self) -> int:
        return self.n0 << self.J

    def sgs_name(self) -> str:
        return {SGS_OFF: "off", SGS_APRIORI: "apriori", SGS_DYNAMIC: "dynamic"}[self.sgs]

    def as_dict(self) -> dict:
        return asdict(self)


@dataclass
class Vortices:
    xc: np.ndarray
    yc: np.ndarray
    gamma: np.ndarray
    s: np.ndarray

    @property
    def n(self) -> int:
        return int(self.xc.size)


@dataclass
class Workload:
    name: str
    params: RunParams
    vortices: Vortices
    nsteps: int
    extra: dict = field(default_factory=dict)


def _pair(d: float, g1: float, g2: float, s: float, jitter=None) -> Vortices:
    xc = np.array([-0.5 * d, 0.5 * d])
    yc = np.zeros(2)
    if jitter is not None:
        xc = xc + jitter[0]
        yc = yc + jitter[1]
    return Vortices(xc, yc, np.array([g1, g2]), np.array([s, s]))


def fujiwhara_small() -> Workload:
    """Equal Gaussian pair, Gamma = 1, s = 0.3, centres (+-0.6, 0), Re = 5000,
    no SGS, coarsest 16^2, finest 128^2 (J = 3), eps = 1e-3, m = 20, dt = 1e-2,
    50 steps."""
    p = RunParams(n0=16, J=3, eps=1e-3, re=5000.0, dt=1e-2, m=20)
    return Workload("fujiwhara_pair_128_fp64", p, _pair(1.2, 1.0, 1.0, 0.3), 50)


def fujiwhara_1024(seed: int = 2) -> Workload:
    """The same pair with dynamic Smagorinsky (C_s = 0.17), coarsest 32^2,
    finest 1024^2 (J = 5), eps = 1e-4, m = 30, dt = 1e-2, 2000 steps; centres
    jittered by U[-0.01, 0.01] per coordinate."""
    rng = np.random.default_rng(seed)
    jit = rng.uniform(-0.01, 0.01, size=(2, 2))
    p = RunParams(n0=32, J=5, eps=1e-4, re=5000.0, dt=1e-2, m=30,
                  sgs=SGS_DYNAMIC, cs=0.17)
    return Workload("fujiwhara_pair_1024_sgs_fp64", p, _pair(1.2, 1.0, 1.0, 0.3, jit), 2000)


def fujiwhara_exner_1024(seed: int = 2) -> Workload:
    """The 1024^2 pair of ``fujiwhara_1024`` in the compressible velocity-Exner
    form (Eqs. 1-2): the vortices' velocity, pi = 1, C = c_p theta_0 = 25 (sound
    speed 5, about 15 times the vortices' peak speed, so dt = 1e-2 is some 8
    acoustic CFL numbers), f = 0.5, no subgrid model, the exact-Jacobian
    (Rosenbrock) step, m = 30, eps = 1e-4."""
    rng = np.random.default_rng(seed)
    jit = rng.uniform(-0.01, 0.01, size=(2, 2))
    p = RunParams(n0=32, J=5, eps=1e-4, re=5000.0, dt=1e-2, m=30, scheme=SCHEME_ROSENBROCK,
                  model=MODEL_EXNER, cpt=25.0, coriolis=0.5)
    return Workload("fujiwhara_pair_1024_exner_fp64", p, _pair(1.2, 1.0, 1.0, 0.3, jit), 200, {"pi0": 1.0})


def three_vortex_4096(seed: int = 3) -> Workload:
    """Three Gaussians s = 0.25, Gamma ~ U[0.8, 1.2], positions by rejection in
    the disc r <= 1.2 until every pair distance lies in [1.0, 1.6]; Re = 37440,
    C_s = 0.17 dynamic, coarsest 32^2, finest 4096^2 (J = 7), eps = 1e-4,
    m = 30, mixed precision, 5000 steps."""
    rng = np.random.default_rng(seed)
    pts = _three_positions(rng)
    gam = rng.uniform(0.8, 1.2, size=3)
    p = RunParams(n0=32, J=7, eps=1e-4, re=37440.0, dt=1e-2, m=30,
                  sgs=SGS_DYNAMIC, cs=0.17, prec=PREC_MIXED)
    v = Vortices(pts[:, 0].copy(), pts[:, 1].copy(), gam, np.full(3, 0.25))
    return Workload("three_vortex_4096_mixed", p, v, 5000)


def _three_positions(rng) -> np.ndarray:
    while True:
        r = 1.2 * np.sqrt(rng.uniform(0.0, 1.0, size=3))
        th = rng.uniform(0.0, 2.0 * np.pi, size=3)
        pts = np.stack([r * np.cos(th), r * np.sin(th)], axis=1)
        dd = [np.hypot(*(pts[a] - pts[b])) for a, b in ((0, 1), (0, 2), (1, 2))]
        if all(1.0 <= x <= 1.6 for x in dd):
            return pts


def ensemble_members(n: int = 256, seed: int = 4, prec: int = PREC_MIXED):
    """Uneven ensemble: two Gaussians s = 0.3 at (+-d/2, 0), d ~ U[0.8, 2.0],
    Gamma_1 = 1, Gamma_2 ~ U[0.5, 1.0], Re ~ U[5000, 37440], C_s = 0.17
    dynamic, coarsest 32^2, finest uniform over {256, 512, 1024, 2048}^2,
    eps = 1e-4, m = 30."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        d = rng.uniform(0.8, 2.0)
        g2 = rng.uniform(0.5, 1.0)
        re = rng.uniform(5000.0, 37440.0)
        J = int(rng.integers(3, 7))          # 32 * 2^J in {256, ..., 2048}
        p = RunParams(n0=32, J=J, eps=1e-4, re=re, dt=1e-2, m=30,
                      sgs=SGS_DYNAMIC, cs=0.17, prec=prec)
        out.append((p, _pair(d, 1.0, g2, 0.3)))
    return out


def serving_trace(n: int = 400, seed: int = 5, rate_hz: float = 50.0,
                  k_range=(7, 12), steps_range=(200, 2000)):
    """Request trace: exponential inter-arrival times (mean 1/rate), 2 or 3
    vortices with probability 1/2 each, finest 2^k with k ~ U{k_range},
    steps ~ U{steps_range}, Re ~ U[5000, 37440].  Returns a list of
    (arrival_s, RunParams, Vortices, nsteps)."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for _ in range(n):
        t += rng.exponential(1.0 / rate_hz)
        k = int(rng.integers(k_range[0], k_range[1] + 1))
        J = k - 5                            # coarsest 32^2
        re = rng.uniform(5000.0, 37440.0)
        nsteps = int(rng.integers(steps_range[0], steps_range[1] + 1))
        if rng.uniform() < 0.5:
            d = rng.uniform(0.8, 2.0)
            v = _pair(d, 1.0, rng.uniform(0.5, 1.0), 0.3)
        else:
            pts = _three_positions(rng)
            v = Vortices(pts[:, 0].copy(), pts[:, 1].copy(),
                         rng.uniform(0.8, 1.2, size=3), np.full(3, 0.25))
        p = RunParams(n0=32, J=J, eps=1e-4, re=re, dt=1e-2, m=30,
                      sgs=SGS_DYNAMIC, cs=0.17, prec=PREC_MIXED)
        out.append((t, p, v, nsteps))
    return out


def random_field_params(seed: int, n: int = 4):
    """Random Gaussian-vortex parameters for parity tests: n vortices with
    centres U[-2, 2]^2, Gamma ~ U[-1.2, 1.2], s ~ U[0.2, 0.5]."""
    rng = np.random.default_rng(seed)
    return Vortices(rng.uniform(-2, 2, n), rng.uniform(-2, 2, n),
                    rng.uniform(-1.2, 1.2, n), rng.uniform(0.2, 0.5, n))
