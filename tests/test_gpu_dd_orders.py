"""Parity of the CUDA path with the FP64 oracle at the higher DD orders
2p = 6 and 8 (wrc_config.p = 3, 4; Sec. 2.4 predictor of 2p points, Sec. 2.5
stencils, Sec. 2.6.2): the index sets and the DD transform bit-exact given
the same field, the frozen fields and the operator within 1e-12, several
steps within the FP64 field bound 1e-10 with the grid identical after every
step, the mixed mode within its bound, and an ensemble member equal to its
solo run."""

import numpy as np
import pytest

from oracle import wrc_oracle as O
from paper_1604_08159_gb300 import binding as B
from paper_1604_08159_gb300 import workloads as W

from helpers import oracle_config, rel_l2, small_params

pytestmark = pytest.mark.gpu

FIELD_TOL = 1e-10
OP_TOL = 1e-12
ORDERS = (3, 4)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1604_08159_gb300 import build
    build.build()
    B.load()


def _masks_equal(run, st, cfg):
    act, gho, _ = run.masks()
    assert np.array_equal(act, st.active)
    lev = O.levels(cfg.n0, cfg.J)
    jx, jy = O.stencil_levels(st.active, lev, cfg.J)
    assert np.array_equal(gho, O.ghost_set(st.active, jx, jy, cfg.J, cfg.p))
    gjx, gjy = run.stencil_levels()
    assert np.array_equal(gjx, jx[st.active]) and np.array_equal(gjy, jy[st.active])


@pytest.mark.parametrize("p", ORDERS)
@pytest.mark.parametrize("case", [dict(n0=16, J=3, eps=1e-3), dict(n0=8, J=2, eps=2e-3, sgs=W.SGS_DYNAMIC, cs=0.17)])
def test_initial_grid_and_transform_bit_exact(p, case):
    prm = small_params(p=p, **case)
    cfg = oracle_config(prm)
    v = W.random_field_params(seed=31, n=3)
    field = O.vortex_field(cfg.NJ, v.xc, v.yc, v.gamma, v.s)
    st = O.state_from_field(cfg, field)
    assert st.active.sum() < cfg.NJ ** 2
    with B.Run(prm) as run:
        run.init_field(field)
        _masks_equal(run, st, cfg)
        idx, om = run.active()
        assert np.array_equal(om, st.omega[st.active])
        R = run.field(B.FIELD_OMEGA)
        assert np.array_equal(R, O.reconstruct(st.omega, st.active, cfg.J, p))
        na = run.counts()[0]
        run.threshold(3e-3)
        d = O.details(O.reconstruct(st.omega, st.active, cfg.J, p), st.active, cfg.J, p)
        assert np.array_equal(run.details(na), d[st.active])


@pytest.mark.parametrize("p", ORDERS)
def test_frozen_fields_and_operator(p):
    prm = small_params(n0=16, J=2, eps=5e-4, sgs=W.SGS_DYNAMIC, cs=0.17, p=p)
    cfg = oracle_config(prm)
    v = W.random_field_params(seed=5, n=4)
    st = O.initial_state(cfg, v.xc, v.yc, v.gamma, v.s)
    fz = O.freeze(cfg, st.active, st.omega)
    with B.Run(prm) as run:
        run.set_grid(st.active, st.omega)
        run.freeze()
        psi = run.field(B.FIELD_PSI)
        assert np.abs(psi - fz.psi).max() <= OP_TOL * np.abs(fz.psi).max()
        assert rel_l2(run.field(B.FIELD_U), fz.U) <= OP_TOL
        assert rel_l2(run.field(B.FIELD_V), fz.V) <= OP_TOL
        S11, S12 = O.strain(fz.psi, fz.U, cfg.h, p)
        assert rel_l2(run.field(B.FIELD_NUT), O.smagorinsky_nut(S11, S12, cfg.cs, cfg.h)) <= 1e-11
        run.freeze()
        rng = np.random.default_rng(3)
        for q in (st.omega[st.active], rng.normal(size=int(st.active.sum()))):
            w, g = run.apply_operator(q)
            assert rel_l2(w, O.apply_operator(cfg, fz, q)) <= OP_TOL
        assert rel_l2(g, fz.g[st.active]) <= 1e-11


@pytest.mark.parametrize("p", ORDERS)
@pytest.mark.parametrize("sgs", [W.SGS_OFF, W.SGS_DYNAMIC])
def test_steps_match_oracle(p, sgs):
    prm = small_params(n0=16, J=3, eps=1e-3, m=16, p=p, sgs=sgs, cs=0.17, re=2000.0)
    cfg = oracle_config(prm)
    v = W.fujiwhara_small().vortices
    st = O.initial_state(cfg, v.xc, v.yc, v.gamma, v.s)
    with B.Run(prm) as run:
        run.set_grid(st.active, st.omega)
        for n in range(3):
            st, info = O.step(cfg, st)
            run.step(1)
            run.sync()
            kr = run.krylov()
            assert kr["k"] == info.k
            assert abs(kr["beta"] - info.beta) <= 1e-12 * info.beta
            act, _, _ = run.masks()
            assert np.array_equal(act, st.active), f"grid differs after step {n + 1}"
            idx, om = run.active()
            assert rel_l2(om, st.omega[st.active]) <= FIELD_TOL
        d = run.diagnostics()
        od = O.diagnostics(cfg, st)
        for key in ("E", "Z", "P", "circulation"):
            assert abs(d[key] - od[key]) <= 1e-10 * abs(od[key]), key


@pytest.mark.parametrize("p", ORDERS)
def test_mixed_precision_within_bound(p):
    prm = small_params(n0=16, J=3, eps=1e-3, m=16, p=p, sgs=W.SGS_DYNAMIC, cs=0.17, re=2000.0,
                       prec=W.PREC_MIXED)
    cfg = oracle_config(prm)
    v = W.fujiwhara_small().vortices
    st = O.initial_state(cfg, v.xc, v.yc, v.gamma, v.s)
    with B.Run(prm) as run:
        run.set_grid(st.active, st.omega)
        st, _ = O.step(cfg, st)
        run.step(1)
        run.sync()
        idx, om = run.active()
        ref_idx = np.flatnonzero(st.active.ravel())
        common, ia, ib = np.intersect1d(idx, ref_idx, return_indices=True)
        assert idx.size + ref_idx.size - 2 * common.size <= 0.002 * ref_idx.size
        assert rel_l2(om[ia], st.omega.ravel()[ref_idx][ib]) <= 1e-6


@pytest.mark.parametrize("p", ORDERS)
def test_ensemble_member_equals_solo(p):
    import torch
    members = [(small_params(n0=16, J=3, eps=1e-3, m=16, p=p, re=re), W.random_field_params(seed=s, n=2))
               for re, s in ((1500.0, 41), (3000.0, 42), (800.0, 43))]
    stream = torch.cuda.Stream()
    with B.Ensemble([m[0] for m in members], stream=stream.cuda_stream) as ens:
        for run, (_, v) in zip(ens.members, members):
            run.init_vortices(v)
        ens.step(2)
        ens.sync()
        got = [run.active() for run in ens.members]
    for (prm, v), (gi, go) in zip(members, got):
        with B.Run(prm) as solo:
            solo.init_vortices(v)
            solo.step(2)
            solo.sync()
            si, so = solo.active()
        assert np.array_equal(gi, si)
        assert rel_l2(go, so) <= 1e-12


def test_invalid_order_rejected():
    with pytest.raises(B.WrcError) as e:
        B.Run(small_params(p=5))
    assert e.value.status == -1
