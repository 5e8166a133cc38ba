"""The passive scalar (vapour mixing ratio with diffusion only) on the GPU
against the oracle: the joint grid bit-exact, r_v and omega within the field
bounds after several steps, the exact decay of a Fourier mode without flow,
and a scalar started from omega staying equal to it."""

import numpy as np
import pytest

from oracle import wrc_oracle as O
from paper_1604_08159_gb300 import binding as B
from paper_1604_08159_gb300 import workloads as W

from helpers import oracle_config, rel_l2, small_params

pytestmark = pytest.mark.gpu

FIELD_TOL = {W.PREC_FP64: 1e-10, W.PREC_MIXED: 1e-5}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1604_08159_gb300 import build
    build.build()
    B.load()


def _lattice(cfg):
    x = -np.pi + cfg.h * np.arange(cfg.NJ)
    return np.meshgrid(x, x)


def test_scalar_front_matches_oracle(prec=W.PREC_FP64):
    p = small_params(n0=16, J=3, eps=1e-3, sgs=W.SGS_DYNAMIC, cs=0.17, re=2000.0, m=16, prec=prec)
    cfg = oracle_config(p)
    vort = W.fujiwhara_small().vortices
    kappa = 2e-3
    st = O.initial_state(cfg, vort.xc, vort.yc, vort.gamma, vort.s)
    X, Y = _lattice(cfg)
    front = 0.5 * (1.0 + np.tanh((Y - 0.3 * np.sin(X)) / 0.2))
    with B.Run(p) as run:
        run.set_grid(st.active, st.omega)
        run.scalar_init(kappa, front)
        st, rv = O.scalar_init(cfg, st, front)
        act, _, _ = run.masks()
        assert np.array_equal(act, st.active)
        idx, r = run.scalar()
        assert np.array_equal(idx, np.flatnonzero(st.active.ravel()))
        assert rel_l2(r, rv[st.active]) <= (0.0 if prec == W.PREC_FP64 else 1e-7)
        for n in range(3):
            st, rv, _, info_r = O.step_with_scalar(cfg, st, rv, kappa)
            run.step(1)
            run.sync()
            act, _, _ = run.masks()
            assert np.array_equal(act, st.active), f"grid differs after step {n + 1}"
            idx, om = run.active()
            assert rel_l2(om, st.omega[st.active]) <= FIELD_TOL[prec]
            idx, r = run.scalar()
            assert rel_l2(r, rv[st.active]) <= FIELD_TOL[prec]
        assert info_r.k > 1


def test_scalar_fourier_mode_decays_exactly():
    p = small_params(n0=8, J=2, eps=10.0, re=100.0, dt=0.05, m=10)
    cfg = oracle_config(p)
    kappa = 0.05
    X, Y = _lattice(cfg)
    r0 = np.sin(X) * np.sin(Y)
    with B.Run(p) as run:
        run.init_field(np.zeros((cfg.NJ, cfg.NJ)))
        run.scalar_init(kappa, r0)
        run.step(4)
        run.sync()
        idx, r = run.scalar()
    lev = O.levels(cfg.n0, cfg.J)
    assert np.array_equal(idx, np.flatnonzero((lev == 0).ravel()))
    h0 = 2.0 * np.pi / cfg.n0
    sigma = (32.0 * np.cos(h0) - 2.0 * np.cos(2.0 * h0) - 30.0) / (12.0 * h0 * h0)
    exact = (r0 * np.exp(2.0 * kappa * sigma * 4 * cfg.dt)).ravel()[idx]
    assert np.abs(r - exact).max() <= 1e-13


def test_scalar_started_from_omega_stays_equal_to_it():
    p = small_params(n0=16, J=3, eps=1e-3, re=1500.0, m=16)
    cfg = oracle_config(p)
    vort = W.fujiwhara_small().vortices
    field = O.vortex_field(cfg.NJ, vort.xc, vort.yc, vort.gamma, vort.s)
    with B.Run(p) as run:
        run.init_field(field)
        na0 = run.counts()[0]
        run.scalar_init(1.0 / p.re, field)
        assert run.counts()[0] == na0
        run.step(3)
        run.sync()
        _, om = run.active()
        _, r = run.scalar()
    assert np.array_equal(r, om)      # same operator, same inputs, same launches


def test_scalar_errors_and_reinitialisation():
    p = small_params(n0=8, J=2, eps=1e-3)
    with B.Run(p) as run:
        run.init_field(np.zeros((32, 32)))
        with pytest.raises(B.WrcError) as e:
            run.scalar()
        assert e.value.status == -7
        with pytest.raises(B.WrcError):
            run.scalar_init(-1.0, np.zeros((32, 32)))
        run.scalar_init(0.1, np.ones((32, 32)))
        run.step(1)
        _, r = run.scalar()
        assert np.abs(r - 1.0).max() <= 1e-14
        run.init_field(np.zeros((32, 32)))     # a new initial condition drops it
        with pytest.raises(B.WrcError):
            run.scalar()


def test_mixed_scalar_close_to_fp64():
    """FP32 bulk: r_v against the FP64 run of the same case, on the points the
    two grids share (the grids may differ where a detail sits near eps)."""
    res = {}
    for prec in (W.PREC_FP64, W.PREC_MIXED):
        p = small_params(n0=16, J=3, eps=1e-3, re=2000.0, m=16, prec=prec)
        cfg = oracle_config(p)
        vort = W.fujiwhara_small().vortices
        X, Y = _lattice(cfg)
        front = 0.5 * (1.0 + np.tanh(Y / 0.25))
        with B.Run(p) as run:
            run.init_field(O.vortex_field(cfg.NJ, vort.xc, vort.yc, vort.gamma, vort.s))
            run.scalar_init(1e-3, front)
            run.step(3)
            run.sync()
            res[prec] = run.scalar()
    (i64, r64), (i32, r32) = res[W.PREC_FP64], res[W.PREC_MIXED]
    common, a, b = np.intersect1d(i64, i32, return_indices=True)
    assert common.size >= 0.99 * max(i64.size, i32.size)
    assert rel_l2(r32[b], r64[a]) <= 1e-5
