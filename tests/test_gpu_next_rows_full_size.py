"""The next rows at the bench's full size (the 1024^2 pair, in the launch
configuration the bench times: a run on its own stream, graph-replayed
phases): the first step of the full-Jacobian Rosenbrock scheme, of the DD
order 2p = 6, and of the velocity-Exner form against the FP64 oracle, grids
identical, fields within 1e-10, Krylov dimension and beta equal.  One oracle
step of each takes 5-15 s on the host."""

import dataclasses

import numpy as np
import pytest

from oracle import exner as E
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


def _krylov_equal(run, info):
    kr = run.krylov()
    assert kr["k"] == info.k
    assert abs(kr["beta"] - info.beta) <= 1e-12 * info.beta


@pytest.mark.parametrize("change", [{"scheme": W.SCHEME_ROSENBROCK}, {"p": 3}], ids=["rosenbrock", "dd6"])
def test_1024_pair_first_step(change):
    import torch
    wl = W.fujiwhara_1024()
    prm = dataclasses.replace(wl.params, **change)
    cfg = oracle_config(prm)
    v = wl.vortices
    st = O.initial_state(cfg, v.xc, v.yc, v.gamma, v.s)
    stream = torch.cuda.Stream()
    with B.Run(prm, stream=stream.cuda_stream) as run:
        run.init_vortices(v)
        act, _, _ = run.masks()
        assert np.array_equal(act, st.active)
        st, info = O.advance(cfg, st)
        run.step(1)
        run.sync()
        _krylov_equal(run, info)
        idx, om = run.active()
        assert np.array_equal(idx, np.flatnonzero(st.active.ravel()))
        assert rel_l2(om, st.omega[st.active]) <= 1e-10


def test_exner_1024_pair_first_step():
    import torch
    wl = W.fujiwhara_exner_1024()
    cfg = oracle_config(wl.params)
    v = wl.vortices
    st = E.exner_vortex_state(cfg, v.xc, v.yc, v.gamma, v.s, wl.extra["pi0"])
    stream = torch.cuda.Stream()
    with B.Run(wl.params, stream=stream.cuda_stream) as run:
        run.exner_init_vortices(v, wl.extra["pi0"])
        for n in range(2):
            act, _, _ = run.masks()
            assert np.array_equal(act, st.active), f"grid differs before step {n + 1}"
            idx, u, vv, p = run.exner()
            a = st.active
            assert rel_l2(np.concatenate([u, vv, p]), np.concatenate([st.u[a], st.v[a], st.pi[a]])) <= 1e-10
            if n == 1:
                break
            st, info = E.exner_step(cfg, st)
            run.step(1)
            run.sync()
            _krylov_equal(run, info)
