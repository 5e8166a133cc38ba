"""In a step the inverse row passes of the Poisson solve run only on the row
pairs within two stencil reaches of a grid point (FP64: psi; FP32 bulk: U, V
and the strain), and the FP32 subgrid lattice passes only on those rows.
With the test switch WRC_TEST_POISON_ROWS=1 every other row of those
lattices is set to NaN after the solve, so a step that read one would carry
a NaN into omega: steps of sparse grids (where a quarter or more of the rows
are not listed) at DD orders 2p = 4 and 8, with and without the dynamic
subgrid model, in FP64 and in the mixed mode, still match the oracle."""

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


CASES = [
    dict(n0=4, J=8, eps=1e-2, p=4, sgs=W.SGS_DYNAMIC, cs=0.17, re=2000.0, m=16),   # 1024^2, ~25% rows unlisted
    dict(n0=4, J=8, eps=1e-3, p=2, sgs=W.SGS_DYNAMIC, cs=0.17, re=2000.0, m=16),
    dict(n0=4, J=8, eps=1e-3, p=2, m=16),
    dict(n0=4, J=8, eps=1e-2, p=2, sgs=W.SGS_DYNAMIC, cs=0.17, re=2000.0, m=16, prec=W.PREC_MIXED),
]


@pytest.mark.parametrize("case", CASES, ids=["p4_sgs", "p2_sgs", "p2", "p2_sgs_mixed"])
def test_steps_with_unlisted_rows_poisoned(case, monkeypatch):
    monkeypatch.setenv("WRC_TEST_POISON_ROWS", "1")   # read when the step's phases are captured
    prm = small_params(**case)
    cfg = oracle_config(prm)
    v = W.fujiwhara_small().vortices
    st = O.initial_state(cfg, v.xc, v.yc, v.gamma, v.s)
    rows = np.flatnonzero(st.active.any(axis=1))
    listed = np.zeros(cfg.NJ, dtype=bool)
    reach = 2 * max(2 * cfg.p - 2, cfg.p)
    for d in range(-reach, reach + 1):
        listed[(rows + d) % cfg.NJ] = True
    assert listed.mean() < 0.95, listed.mean()     # the pruning has rows to leave out
    prec = case.get("prec", W.PREC_FP64)
    with B.Run(prm) as run:
        run.set_grid(st.active, st.omega)
        for n in range(2):
            st, _ = O.step(cfg, st)
            run.step(1)
            run.sync()
            act, _, _ = run.masks()
            if prec == W.PREC_FP64:
                assert np.array_equal(act, st.active), f"grid differs after step {n + 1}"
            idx, om = run.active()
            assert np.all(np.isfinite(om)), f"a poisoned row was read in step {n + 1}"
            common = np.intersect1d(idx, np.flatnonzero(st.active.ravel()))
            ref = st.omega.ravel()[common]
            got = om[np.searchsorted(idx, common)]
            assert rel_l2(got, ref) <= FIELD_TOL[prec]
