"""Parity of the exponential Rosenbrock-Euler step (WRC_SCHEME_ROSENBROCK:
the Krylov projection with the full Jacobian of the advection, a Poisson
solve per Krylov vector; Sec. 1 and 2.1) with the FP64 oracle's
``step_rosenbrock``: grids identical after every step, omega within the FP64
field bound 1e-10 (1e-6 in the mixed mode), the Krylov dimension and beta
equal; the step differs from the frozen-linearisation step; the batched
forms refuse it."""

import numpy as np
import pytest

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


CASES = [
    dict(n0=16, J=3, eps=1e-3, m=20),
    dict(n0=16, J=3, eps=1e-3, m=16, sgs=W.SGS_DYNAMIC, cs=0.17, re=2000.0),
    dict(n0=16, J=2, eps=1e-3, m=16, p=3, rayleigh_r=0.05),
]


@pytest.mark.parametrize("case", CASES)
def test_rosenbrock_steps_match_oracle(case):
    prm = small_params(scheme=W.SCHEME_ROSENBROCK, **case)
    cfg = oracle_config(prm)
    assert cfg.scheme == "rosenbrock"
    v = W.fujiwhara_small().vortices
    st = O.initial_state(cfg, v.xc, v.yc, v.gamma, v.s)
    with B.Run(prm) as run:
        run.set_grid(st.active, st.omega)
        for n in range(3):
            st, info = O.step_rosenbrock(cfg, st)
            run.step(1)
            run.sync()
            kr = run.krylov()
            assert kr["k"] == info.k
            assert abs(kr["beta"] - info.beta) <= 1e-12 * info.beta
            act, _, _ = run.masks()
            assert np.array_equal(act, st.active), f"grid differs after step {n + 1}"
            idx, om = run.active()
            assert rel_l2(om, st.omega[st.active]) <= 1e-10


def test_rosenbrock_mixed_within_bound():
    prm = small_params(n0=16, J=3, eps=1e-3, m=16, scheme=W.SCHEME_ROSENBROCK, prec=W.PREC_MIXED)
    cfg = oracle_config(prm)
    v = W.fujiwhara_small().vortices
    st = O.initial_state(cfg, v.xc, v.yc, v.gamma, v.s)
    with B.Run(prm) as run:
        run.set_grid(st.active, st.omega)
        for _ in range(2):
            st, _ = O.step_rosenbrock(cfg, st)
            run.step(1)
        run.sync()
        idx, om = run.active()
        ref_idx = np.flatnonzero(st.active.ravel())
        common, ia, ib = np.intersect1d(idx, ref_idx, return_indices=True)
        assert idx.size + ref_idx.size - 2 * common.size <= 0.002 * ref_idx.size
        assert rel_l2(om[ia], st.omega.ravel()[ref_idx][ib]) <= 1e-6


def test_rosenbrock_differs_from_frozen_step():
    v = W.fujiwhara_small().vortices
    out = []
    for scheme in (W.SCHEME_FROZEN, W.SCHEME_ROSENBROCK):
        with B.Run(small_params(n0=16, J=3, eps=0.0, m=20, dt=0.05, scheme=scheme)) as run:
            run.init_vortices(v)
            run.step(2)
            run.sync()
            out.append(run.active()[1])
    assert rel_l2(out[1], out[0]) > 1e-7


def test_batched_forms_refuse_rosenbrock():
    import torch
    prm = small_params(scheme=W.SCHEME_ROSENBROCK)
    stream = torch.cuda.Stream()
    with B.Ensemble([prm, small_params()], stream=stream.cuda_stream) as ens:
        for run in ens.members:
            run.init_vortices(W.fujiwhara_small().vortices)
        with pytest.raises(B.WrcError) as e:
            ens.step(1)
        assert e.value.status == -1
