"""Shared test helpers: oracle configs from run parameters, comparisons."""

import numpy as np

from oracle import exner as E
from oracle import wrc_oracle as O
from paper_1604_08159_gb300 import workloads as W


def oracle_config(p) -> O.Config:
    kw = dict(n0=p.n0, J=p.J, eps=p.eps, re=p.re, dt=p.dt, m=p.m, sgs=p.sgs_name(), cs=p.cs,
              s_apriori=p.s_apriori, rayleigh_r=p.rayleigh_r, p=p.p,
              scheme="rosenbrock" if p.scheme == W.SCHEME_ROSENBROCK else "frozen")
    if p.model == W.MODEL_EXNER:
        return E.ExnerConfig(**kw, cpt=p.cpt, coriolis=p.coriolis, gx=p.gx, gy=p.gy)
    return O.Config(**kw)


def rel_l2(a, b) -> float:
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    den = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (den if den > 0 else 1.0))


def small_params(**kw) -> W.RunParams:
    base = dict(n0=16, J=3, eps=1e-3, re=5000.0, dt=1e-2, m=20)
    base.update(kw)
    return W.RunParams(**base)
