"""Parity of the compressible velocity-Exner form on the GPU (model
WRC_MODEL_EXNER; Eqs. 1-2 with the f-plane Coriolis term and Rayleigh
friction) with the FP64 oracle ``oracle/exner.py``: the initial grid and
fields from lattice fields and from vortex parameters, then steps of the
Rosenbrock (exact Jacobian) and frozen schemes with grids identical after
every step, u, v, pi within 1e-10, Krylov dimension and beta equal; a
discrete geostrophic jet stays steady on the GPU; the calls of the vorticity
form and the batched forms refuse the model."""

import numpy as np
import pytest

from oracle import exner as E
from oracle import wrc_oracle as O
from paper_1604_08159_gb300 import binding as B
from paper_1604_08159_gb300 import workloads as W

from helpers import oracle_config, rel_l2, small_params

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1604_08159_gb300 import build
    build.build()
    B.load()


def exner_params(**kw):
    base = dict(model=W.MODEL_EXNER, cpt=4.0, coriolis=0.5, re=1000.0, dt=0.02, scheme=W.SCHEME_ROSENBROCK)
    base.update(kw)
    return small_params(**base)


def _check(run, st, tol=1e-10):
    act, _, _ = run.masks()
    assert np.array_equal(act, st.active)
    idx, u, v, p = run.exner()
    a = st.active
    got = np.concatenate([u, v, p])
    want = np.concatenate([st.u[a], st.v[a], st.pi[a]])
    assert rel_l2(got, want) <= tol, rel_l2(got, want)


VORT = dict(xc=[-0.7, 0.6], yc=[0.1, -0.2], gamma=[2.0, 1.2], s=[0.45, 0.5])

CASES = [
    dict(),
    dict(scheme=W.SCHEME_FROZEN, gx=0.2, gy=-0.1, rayleigh_r=0.05),
    dict(sgs=W.SGS_APRIORI, cs=0.17, s_apriori=2.0, cpt=25.0, dt=0.05, m=24),
    dict(p=3, J=2, coriolis=-0.8),
    dict(p=4, J=2, scheme=W.SCHEME_FROZEN, m=16),
]


@pytest.mark.parametrize("case", CASES)
def test_exner_steps_match_oracle(case):
    prm = exner_params(**case)
    cfg = oracle_config(prm)
    assert isinstance(cfg, E.ExnerConfig)
    st = E.exner_vortex_state(cfg, VORT["xc"], VORT["yc"], VORT["gamma"], VORT["s"], 1.0)
    om = O.vortex_field(cfg.NJ, VORT["xc"], VORT["yc"], VORT["gamma"], VORT["s"])
    psi = O.streamfunction(om, cfg.h, cfg.p)
    u0, v0 = O.velocity(psi, cfg.h, cfg.p)
    with B.Run(prm) as run:
        run.exner_init(u0, v0, np.ones_like(u0))
        _check(run, st, 1e-13)
        for n in range(3):
            st, info = E.exner_step(cfg, st)
            run.step(1)
            run.sync()
            kr = run.krylov()
            assert kr["k"] == info.k
            assert abs(kr["beta"] - info.beta) <= 1e-12 * info.beta
            _check(run, st)


def test_exner_init_vortices_matches_oracle():
    prm = exner_params()
    cfg = oracle_config(prm)
    st = E.exner_vortex_state(cfg, VORT["xc"], VORT["yc"], VORT["gamma"], VORT["s"], 1.3)
    with B.Run(prm) as run:
        run.exner_init_vortices(W.Vortices(*(np.array(VORT[k]) for k in ("xc", "yc", "gamma", "s"))), 1.3)
        _check(run, st, 1e-12)


def test_discrete_geostrophic_jet_stays_steady_on_the_gpu():
    prm = exner_params(n0=16, J=1, eps=0.0, re=1e300, cpt=2.0, coriolis=0.8, gx=0.25, m=10, dt=0.1)
    NJ = prm.NJ
    h = 2.0 * np.pi / NJ
    x = -np.pi + h * np.arange(NJ)
    Y = np.repeat(x[:, None], NJ, axis=1)
    s1 = (8.0 * np.sin(h) - np.sin(2.0 * h)) / (6.0 * h)
    a = 0.6
    u = prm.gx + a * np.cos(Y)
    v = np.zeros_like(u)
    p = 1.3 - prm.coriolis * a / (prm.cpt * s1) * np.sin(Y)
    with B.Run(prm) as run:
        run.exner_init(u, v, p)
        run.step(3)
        run.sync()
        idx, u1, v1, p1 = run.exner()
        assert idx.size == NJ * NJ
        assert np.max(np.abs(u1 - u.ravel())) <= 1e-12
        assert np.max(np.abs(v1)) <= 1e-12
        assert np.max(np.abs(p1 - p.ravel())) <= 1e-12


def test_vorticity_calls_and_batched_forms_refuse_the_exner_model():
    prm = exner_params()
    with B.Run(prm) as run:
        with pytest.raises(B.WrcError) as e:
            run.init_vortices(W.fujiwhara_small().vortices)
        assert e.value.status == -7
        run.exner_init_vortices(W.fujiwhara_small().vortices, 1.0)
        for call in (lambda: run.active(), lambda: run.field(0), lambda: run.threshold(1e-3)):
            with pytest.raises(B.WrcError) as e:
                call()
            assert e.value.status == -7
    with pytest.raises(B.WrcError) as e:
        B.Ensemble([prm, prm])
    assert e.value.status == -1
    with B.Run(small_params()) as run:
        with pytest.raises(B.WrcError) as e:
            run.exner_init_vortices(W.fujiwhara_small().vortices, 1.0)
        assert e.value.status == -7


def test_exner_barrier_wait_limit_runs_out():
    """A wait limit of 100 ns: a grid barrier of the velocity-Exner Krylov
    kernel runs out, every block returns, the step reports WRC_ERR_TIMEOUT,
    and the run steps correctly after a new initial condition."""
    prm = exner_params()
    cfg = oracle_config(prm)
    st = E.exner_vortex_state(cfg, VORT["xc"], VORT["yc"], VORT["gamma"], VORT["s"], 1.0)
    st1, _ = E.exner_step(cfg, st)
    vort = W.Vortices(*(np.array(VORT[k]) for k in ("xc", "yc", "gamma", "s")))
    with B.Run(prm) as run:
        run.exner_init_vortices(vort, 1.0)
        run.set_wait_limit(1e-7)
        with pytest.raises(B.WrcError) as e:
            run.step(1)
        assert e.value.status == -5, e.value
        run.sync()
        run.set_wait_limit(2.0)
        run.exner_init_vortices(vort, 1.0)
        run.step(1)
        run.sync()
        _check(run, st1)


def test_exner_uniform_geostrophic_wind_has_no_krylov_space():
    """u = G, pi uniform: F(U) = 0 exactly, so beta = 0, the Krylov dimension
    is 0 and the state does not change (the breakdown path at k = 0)."""
    prm = exner_params(n0=16, J=2, eps=1e-3, gx=0.3, gy=-0.2, re=float("inf"))
    NJ = prm.NJ
    one = np.ones((NJ, NJ))
    with B.Run(prm) as run:
        run.exner_init(prm.gx * one, prm.gy * one, 1.2 * one)
        idx0, u0, v0, p0 = run.exner()
        run.step(2)
        run.sync()
        kr = run.krylov()
        assert kr["k"] == 0 and kr["beta"] == 0.0
        idx, u, v, p = run.exner()
        assert np.array_equal(idx, idx0)
        assert np.array_equal(u, u0) and np.array_equal(v, v0) and np.array_equal(p, p0)
