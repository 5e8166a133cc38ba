"""Writes tests/golden/three_vortex_4096_20steps.npz: the FP64 oracle's first
20 steps of the 4096^2 three-vortex workload (finest 4096^2, J = 7,
Re = 37440, dynamic Smagorinsky C_s = 0.17, eps = 1e-4, m = 30, dt = 1e-2;
seeded draws from paper_1604_08159_gb300/workloads.py), for the step-by-step
comparison of the mixed-precision GPU path (tests/test_gpu_mixed.py).

Calls only the oracle (and the seeded parameter draws).  Per step s = 0..20
(s = 0 is the initial grid) it stores, compactly:
  grid_s      the active lattice indices, as int32 gaps from the previous one;
  samp_s      every 4th active point (lattice indices, same gap coding);
  omega_s     omega at those sampled points (float64);
  diag        E, Z, P, circulation and the active count per step.
Run time: about 30 min on 8 host cores.  Usage: python tests/golden/make_three_vortex_4096.py
"""

import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from oracle import wrc_oracle as O  # noqa: E402
from paper_1604_08159_gb300 import workloads as W  # noqa: E402

STEPS = 20
SAMPLE = 4
OUT = os.path.join(HERE, "three_vortex_4096_20steps.npz")


def gaps(idx):
    idx = np.asarray(idx, dtype=np.int64)
    return np.diff(np.concatenate([[0], idx])).astype(np.int32)


def main():
    wl = W.three_vortex_4096()
    p = wl.params
    cfg = O.Config(n0=p.n0, J=p.J, eps=p.eps, re=p.re, dt=p.dt, m=p.m, sgs=p.sgs_name(), cs=p.cs,
                   s_apriori=p.s_apriori, rayleigh_r=p.rayleigh_r)
    v = wl.vortices
    st = O.initial_state(cfg, v.xc, v.yc, v.gamma, v.s)
    out = {}
    diag = []
    t0 = time.time()
    for s in range(STEPS + 1):
        if s > 0:
            st, _ = O.step(cfg, st)
        idx = np.flatnonzero(st.active.ravel())
        om = st.omega.ravel()[idx]
        out[f"grid_{s}"] = gaps(idx)
        out[f"samp_{s}"] = gaps(idx[::SAMPLE])
        out[f"omega_{s}"] = om[::SAMPLE].astype(np.float64)
        d = O.diagnostics(cfg, st)
        diag.append([d["E"], d["Z"], d["P"], d["circulation"], float(idx.size)])
        print(f"step {s}: n_active={idx.size} ({time.time() - t0:.0f} s)", flush=True)
    out["diag"] = np.array(diag)
    out["meta"] = np.array([STEPS, SAMPLE, cfg.NJ], dtype=np.int64)
    np.savez_compressed(OUT, **out)
    print("wrote", OUT, os.path.getsize(OUT), "bytes")


if __name__ == "__main__":
    main()
