"""Batched ensemble: uneven members in one cooperative Krylov launch per step.
Each member's result must equal its solo run (the reductions are only split
into different blocks: FP64 within 1e-12, mixed within the mixed bound), the
grids must be identical, and a member must match the FP64 oracle."""

import numpy as np
import pytest

from oracle import wrc_oracle as O
from paper_1604_08159_gb300 import binding as B
from paper_1604_08159_gb300 import workloads as W

from helpers import oracle_config, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1604_08159_gb300 import build
    build.build()
    B.load()


def uneven_members(prec, n=6, seed=40):
    rng = np.random.default_rng(seed)
    out = []
    for q in range(n):
        J = [1, 2, 3][q % 3]
        p = W.RunParams(n0=32, J=J, eps=float(rng.choice([1e-3, 3e-4])), re=float(rng.uniform(500, 5000)),
                        dt=1e-2, m=int(rng.choice([12, 20, 30])),
                        sgs=[W.SGS_OFF, W.SGS_DYNAMIC, W.SGS_APRIORI][q % 3], cs=0.17, s_apriori=3.0,
                        prec=prec)
        out.append((p, W.random_field_params(seed=seed + q, n=2 + q % 2)))
    return out


def run_solo(p, v, nsteps):
    with B.Run(p) as run:
        run.init_vortices(v)
        run.step(nsteps)
        run.sync()
        return run.active()


@pytest.mark.parametrize("prec,tol", [(W.PREC_FP64, 1e-12), (W.PREC_MIXED, 1e-6)])
def test_members_equal_solo_runs(prec, tol):
    members = uneven_members(prec)
    nsteps = 4
    with B.Ensemble([p for p, _ in members]) as ens:
        for m, (_, v) in zip(ens.members, members):
            m.init_vortices(v)
        ens.step(nsteps)
        st = ens.stats()
        assert st["members"] == len(members) and st["steps"] == nsteps and st["blocks"] >= len(members)
        got = [m.active() for m in ens.members]
    for (p, v), (idx, om) in zip(members, got):
        ridx, rom = run_solo(p, v, nsteps)
        assert np.array_equal(idx, ridx)
        assert rel_l2(om, rom) <= tol


def test_member_matches_oracle():
    members = uneven_members(W.PREC_FP64, n=3, seed=7)
    p, v = members[2]
    cfg = oracle_config(p)
    st = O.initial_state(cfg, v.xc, v.yc, v.gamma, v.s)
    with B.Ensemble([q for q, _ in members]) as ens:
        for m, (_, vv) in zip(ens.members, members):
            m.init_vortices(vv)
        ens.members[2].set_grid(st.active, st.omega)
        for _ in range(2):
            ens.step(1)
            st, _ = O.step(cfg, st)
            idx, om = ens.members[2].active()
            assert np.array_equal(idx, np.flatnonzero(st.active.ravel()))
            assert rel_l2(om, st.omega[st.active]) <= 1e-10


def test_autotuner_picks_a_valid_shape_and_caches_it():
    members = uneven_members(W.PREC_MIXED, n=4, seed=11)
    with B.Ensemble([p for p, _ in members]) as ens:
        for m, (_, v) in zip(ens.members, members):
            m.init_vortices(v)
        shape = ens.tune(1)
        assert shape[0] in (64, 128, 256) and shape[1] in (1, 2, 4)
        steps_after_tune = ens.stats()["steps"]
        assert steps_after_tune == 9                 # one real step per candidate
        assert ens.tune(1) == shape                  # cached: no further steps
        assert ens.stats()["steps"] == steps_after_tune
        ens.step(2)
        st = ens.stats()
        assert (st["threads_per_block"], st["points_per_thread"]) == shape


def test_ensemble_rejects_mixed_precisions():
    p64 = W.RunParams(n0=16, J=1, eps=1e-3, re=1000.0)
    p32 = W.RunParams(n0=16, J=1, eps=1e-3, re=1000.0, prec=W.PREC_MIXED)
    with pytest.raises(B.WrcError):
        B.Ensemble([p64, p32])
