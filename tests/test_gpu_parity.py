"""Parity of the CUDA path (through the C-ABI) with the FP64 oracle.

Index sets (active, ghost, significant masks, stencil levels) must be
bit-exact given the same coefficients; the DD reconstruction and details are
evaluated in the same operation order on both sides and must be bit-exact too.
Fields must agree within the FP64 bound 1e-10 (relative L2); single
operator applications and spectral fields within 1e-12.
"""

import numpy as np
import pytest

from oracle import wrc_oracle as O
from paper_1604_08159_gb300 import binding as B
from paper_1604_08159_gb300 import workloads as W

from helpers import oracle_config, rel_l2, small_params

pytestmark = pytest.mark.gpu

FIELD_TOL = 1e-10      # FP64 vorticity bound (relative L2)
OP_TOL = 1e-12         # one operator application / spectral solve


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1604_08159_gb300 import build
    build.build()
    B.load()


def _masks_equal(run, st, cfg):
    act, gho, sig = run.masks()
    assert np.array_equal(act, st.active)
    lev = O.levels(cfg.n0, cfg.J)
    jx, jy = O.stencil_levels(st.active, lev, cfg.J)
    G = O.ghost_set(st.active, jx, jy, cfg.J)
    assert np.array_equal(gho, G)
    gjx, gjy = run.stencil_levels()
    assert np.array_equal(gjx, jx[st.active]) and np.array_equal(gjy, jy[st.active])


def _state_equal(run, st, tol=FIELD_TOL):
    idx, om = run.active()
    NJ = st.active.shape[0]
    assert np.array_equal(idx, np.flatnonzero(st.active.ravel()))
    assert rel_l2(om, st.omega[st.active]) <= tol


CASES = [
    dict(n0=16, J=3, eps=1e-3),                       # the 128^2 pair workload grid
    dict(n0=8, J=2, eps=3e-3, sgs=W.SGS_DYNAMIC, cs=0.17, re=800.0),
    dict(n0=4, J=1, eps=1e-2),                        # smallest lattice
    dict(n0=32, J=2, eps=1e-4, sgs=W.SGS_APRIORI, cs=0.17, s_apriori=5.0, rayleigh_r=0.05),
]


@pytest.mark.parametrize("case", CASES)
def test_initial_grid_bit_exact_given_same_field(case):
    p = small_params(**case)
    cfg = oracle_config(p)
    v = W.random_field_params(seed=11, n=3)
    field = O.vortex_field(cfg.NJ, v.xc, v.yc, v.gamma, v.s)
    st = O.state_from_field(cfg, field)
    with B.Run(p) as run:
        run.init_field(field)
        _masks_equal(run, st, cfg)
        idx, om = run.active()
        assert np.array_equal(om, st.omega[st.active])      # values copied, no arithmetic
        R = run.field(B.FIELD_OMEGA)
        assert np.array_equal(R, O.reconstruct(st.omega, st.active, cfg.J))


def test_threshold_details_bit_exact():
    p = small_params(n0=16, J=3, eps=1e-3)
    cfg = oracle_config(p)
    field = O.vortex_field(cfg.NJ, [-0.6, 0.6], [0.0, 0.05], [1.0, 0.8], [0.3, 0.35])
    st = O.state_from_field(cfg, field)
    with B.Run(p) as run:
        run.init_field(field)
        na = run.counts()[0]
        run.threshold(3e-3)
        R = O.reconstruct(st.omega, st.active, cfg.J)
        d = O.details(R, st.active, cfg.J)
        assert np.array_equal(run.details(na), d[st.active])
        cfg.eps = 3e-3
        A2, om2, _ = O.adapt(cfg, st.active, st.omega)
        _, _, sig = run.masks()
        lev = O.levels(cfg.n0, cfg.J)
        assert np.array_equal(sig, O.significant(d, st.active, lev, 3e-3))
        _masks_equal(run, O.State(A2, om2), cfg)
        _state_equal(run, O.State(A2, om2), tol=0.0)


def test_init_vortices_matches_oracle_ic():
    p = small_params(n0=16, J=3, eps=1e-3)
    cfg = oracle_config(p)
    v = W.fujiwhara_small().vortices
    st = O.initial_state(cfg, v.xc, v.yc, v.gamma, v.s)
    with B.Run(p) as run:
        run.init_vortices(v)
        idx, om = run.active()
        # both sides sample exp(), which may differ in the last bit; the
        # inputs are chosen so that no detail lies within rounding of eps
        # (otherwise a point could flip), and the test says so if they stop
        # being so rather than passing without an assertion
        d = np.abs(O.details(O.vortex_field(cfg.NJ, v.xc, v.yc, v.gamma, v.s), np.ones_like(st.active), cfg.J))
        near = np.abs(d - cfg.eps) < 1e-12 * cfg.eps
        assert not near.any(), "a detail of the initial field lies within rounding of eps"
        assert np.array_equal(idx, np.flatnonzero(st.active.ravel()))
        assert rel_l2(om, st.omega[st.active]) <= 1e-14


def test_set_grid_validates_closure():
    p = small_params(n0=8, J=2, eps=1e-3)
    cfg = oracle_config(p)
    lev = O.levels(cfg.n0, cfg.J)
    with B.Run(p) as run:
        bad = (lev == 0).copy()
        bad[1, 1] = True                      # a level-2 point without its predictor points
        with pytest.raises(B.WrcError) as e:
            run.set_grid(bad, np.zeros(lev.shape))
        assert e.value.status == -1
        with pytest.raises(B.WrcError):
            run.set_grid(np.zeros(lev.shape, dtype=bool), np.zeros(lev.shape))


@pytest.mark.parametrize("case", CASES[:2] + [dict(n0=16, J=2, eps=5e-4, sgs=W.SGS_DYNAMIC, cs=0.17)])
def test_frozen_fields_and_operator(case):
    p = small_params(**case)
    cfg = oracle_config(p)
    v = W.random_field_params(seed=5, n=4)
    st = O.initial_state(cfg, v.xc, v.yc, v.gamma, v.s)
    fz = O.freeze(cfg, st.active, st.omega)
    NJ = cfg.NJ
    with B.Run(p) as run:
        run.set_grid(st.active, st.omega)
        run.freeze()
        psi = run.field(B.FIELD_PSI)
        assert np.abs(psi - fz.psi).max() <= OP_TOL * np.abs(fz.psi).max()
        U = run.field(B.FIELD_U)
        V = run.field(B.FIELD_V)
        assert rel_l2(U, fz.U) <= OP_TOL and rel_l2(V, fz.V) <= OP_TOL
        if cfg.cs > 0:
            S11, S12 = O.strain(fz.psi, fz.U, cfg.h)
            nut = O.smagorinsky_nut(S11, S12, cfg.cs, cfg.h)
            assert rel_l2(run.field(B.FIELD_NUT), nut) <= 1e-11
        run.freeze()
        rng = np.random.default_rng(3)
        for q in (st.omega[st.active], rng.normal(size=int(st.active.sum()))):
            w, g = run.apply_operator(q)
            assert rel_l2(w, O.apply_operator(cfg, fz, q)) <= OP_TOL
        if p.sgs == W.SGS_DYNAMIC:
            assert rel_l2(g, fz.g[st.active]) <= 1e-11
        else:
            assert not g.any()


def _run_steps_compare(p, vort, nsteps):
    """Step the GPU and the oracle side by side.  The Arnoldi basis and the
    trailing Hessenberg columns are ill-conditioned functions of the data (a
    1e-16 change of b moves late columns of H by ~1e-11 on the 128^2 pair,
    while the step increment moves by ~1e-16), so H is held tightly only in
    its leading columns; the step result omega, a stable function, is held to
    the FP64 field bound."""
    cfg = oracle_config(p)
    st = O.initial_state(cfg, vort.xc, vort.yc, vort.gamma, vort.s)
    with B.Run(p) as run:
        run.set_grid(st.active, st.omega)
        for n in range(nsteps):
            st, info = O.step(cfg, st)
            run.step(1)
            run.sync()
            kr = run.krylov()
            assert kr["k"] == info.k
            assert abs(kr["beta"] - info.beta) <= 1e-12 * info.beta
            lead = min(2, info.k)
            assert rel_l2(kr["H"][: lead + 1, :lead], info.H[: lead + 1, :lead]) <= 1e-12
            assert rel_l2(kr["H"][: info.k + 1, : info.k], info.H) <= 1e-6
            act, _, _ = run.masks()
            assert np.array_equal(act, st.active), f"grid differs after step {n + 1}"
            _state_equal(run, st)
        d = run.diagnostics()
        od = O.diagnostics(cfg, st)
        for key in ("E", "Z", "P", "circulation"):
            assert abs(d[key] - od[key]) <= 1e-10 * abs(od[key]), key
        assert d["nstep"] == nsteps
        # the Krylov error estimate of the last step from the oracle's H and y
        # (an estimate far below the increment's rounding level, dt beta 1e-12,
        # is compared only against that level)
        est = cfg.dt * info.beta * info.h_last * abs(info.y[info.k - 1]) if info.k > 0 else 0.0
        assert abs(d["krylov_err"] - est) <= 1e-4 * est + 1e-12 * cfg.dt * info.beta


def test_steps_pair_128_matches_oracle():
    wl = W.fujiwhara_small()
    _run_steps_compare(wl.params, wl.vortices, nsteps=5)


def test_steps_dynamic_sgs_matches_oracle():
    p = small_params(n0=16, J=3, eps=1e-3, sgs=W.SGS_DYNAMIC, cs=0.17, re=2000.0, m=12, dt=2e-2)
    _run_steps_compare(p, W.random_field_params(seed=21, n=3), nsteps=3)


def test_steps_apriori_and_rayleigh_match_oracle():
    p = small_params(n0=8, J=3, eps=2e-3, sgs=W.SGS_APRIORI, cs=0.17, s_apriori=8.0, rayleigh_r=0.1, m=8)
    _run_steps_compare(p, W.random_field_params(seed=22, n=2), nsteps=3)


def test_taylor_green_breakdown_and_zero_field():
    p = small_params(n0=8, J=2, eps=0.0, re=20.0, dt=0.05, m=10)
    cfg = oracle_config(p)
    NJ, h = cfg.NJ, cfg.h
    x = -np.pi + h * np.arange(NJ)
    X, Y = np.meshgrid(x, x)
    om0 = 2 * np.sin(X) * np.sin(Y)
    with B.Run(p) as run:
        run.init_field(om0)
        run.step(4)
        run.sync()
        assert run.krylov()["k"] == 1
        sig = (30 - 32 * np.cos(h) + 2 * np.cos(2 * h)) / (12 * h * h)
        exact = om0 * np.exp(-2 * cfg.nu * sig * 4 * cfg.dt)
        idx, om = run.active()
        assert np.abs(om - exact.ravel()[idx]).max() <= 1e-13
    with B.Run(p) as run:
        run.init_field(np.zeros((NJ, NJ)))
        run.step(2)
        run.sync()
        assert run.krylov()["k"] == 0 and run.krylov()["beta"] == 0.0
        idx, om = run.active()
        assert not om.any()


def test_fujiwhara_1024_first_steps_match_oracle():
    """The 1024^2 workload with dynamic Smagorinsky, as timed by the bench:
    two steps against the oracle."""
    wl = W.fujiwhara_1024()
    _run_steps_compare(wl.params, wl.vortices, nsteps=2)


def test_4096_lattice_grid_and_streamfunction():
    """Full 4096^2 lattice (J = 7): initial grid bit-exact and the
    streamfunction within the spectral bound, checked at every point."""
    wl = W.three_vortex_4096()
    p = W.RunParams(**{**wl.params.as_dict(), "prec": W.PREC_FP64})
    cfg = oracle_config(p)
    v = wl.vortices
    field = O.vortex_field(cfg.NJ, v.xc, v.yc, v.gamma, v.s)
    st = O.state_from_field(cfg, field)
    with B.Run(p) as run:
        run.init_field(field)
        act, _, _ = run.masks()
        assert np.array_equal(act, st.active)
        run.freeze()
        psi = run.field(B.FIELD_PSI)
        R = O.reconstruct(st.omega, st.active, cfg.J)
        ref = O.streamfunction(R, cfg.h)
        assert np.abs(psi - ref).max() <= OP_TOL * np.abs(ref).max()


@pytest.mark.parametrize("prec", [W.PREC_FP64, W.PREC_MIXED])
def test_graph_replayed_steps_bit_identical_to_direct_launches(prec):
    """On a non-default stream the step phases run as captured CUDA graphs
    (re-captured when buffers grow); the results must be bit-identical to
    the directly launched run, since the kernels and their order are the same
    and every reduction is deterministic."""
    import torch
    p = W.RunParams(**{**W.fujiwhara_small().params.as_dict(), "prec": prec,
                       "sgs": W.SGS_DYNAMIC, "cs": 0.17})
    v = W.fujiwhara_small().vortices
    outs = []
    for use_stream in (False, True):
        stream = torch.cuda.Stream() if use_stream else None
        with B.Run(p, stream=stream.cuda_stream if stream else None) as run:
            run.init_vortices(v)
            run.step(6)
            run.sync()
            outs.append(run.active())
    assert np.array_equal(outs[0][0], outs[1][0])
    assert np.array_equal(outs[0][1], outs[1][1])


@pytest.mark.parametrize("prec", [W.PREC_FP64, W.PREC_MIXED])
def test_runs_of_different_sizes_coexist(prec):
    """Per-kernel launch limits are process-wide: creating a small run after a
    large one must not break the large one's steps (graph-captured too)."""
    import torch
    big = W.RunParams(n0=32, J=3, eps=1e-3, re=2000.0, sgs=W.SGS_DYNAMIC, cs=0.17, prec=prec)
    small = W.RunParams(n0=16, J=1, eps=1e-3, re=2000.0, prec=prec)
    v = W.random_field_params(seed=3, n=2)
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    with B.Run(big, stream=s1.cuda_stream) as a, B.Run(small, stream=s2.cuda_stream) as b:
        a.init_vortices(v)
        b.init_vortices(v)
        a.step(2)
        b.step(2)
        a.sync()
        b.sync()
        assert a.counts()[0] > 0 and b.counts()[0] > 0


@pytest.mark.parametrize("cluster", ["1", "2"])
def test_unclustered_krylov_kernel_matches_oracle(cluster, monkeypatch):
    """The Krylov launch without thread-block clusters (WRC_KRYLOV_CLUSTER=1,
    the form profilers run) and with clusters of two: the same steps against
    the oracle.  The cluster size only changes the order of the cross-block
    additions."""
    monkeypatch.setenv("WRC_KRYLOV_CLUSTER", cluster)
    wl = W.fujiwhara_small()
    _run_steps_compare(wl.params, wl.vortices, nsteps=3)


def test_fujiwhara_128_whole_run_of_50_steps():
    """The whole 128^2 pair workload (50 steps of dt = 1e-2) against the
    oracle: the grid identical after every step, omega within the FP64 bound
    after every tenth, the Krylov dimension equal throughout."""
    wl = W.fujiwhara_small()
    cfg = oracle_config(wl.params)
    v = wl.vortices
    st = O.initial_state(cfg, v.xc, v.yc, v.gamma, v.s)
    with B.Run(wl.params) as run:
        run.init_vortices(v)
        for n in range(wl.nsteps):
            st, info = O.step(cfg, st)
            run.step(1)
            run.sync()
            assert run.krylov()["k"] == info.k
            act, _, _ = run.masks()
            assert np.array_equal(act, st.active), f"grid differs after step {n + 1}"
            if (n + 1) % 10 == 0:
                _state_equal(run, st)
