"""Nine-level hierarchies (n0 = 4, J = 8: a 1024^2 lattice over a 4^2
coarsest grid) against the FP64 oracle.  Their ghosts lie on up to six
levels, so the interpolation rows, built in one launch in which a ghost
waits for the rows of its coarser ghost predictors, chain through several
levels; the tiled reconstruction's coarse regions are many tiles wide.
Three steps: the ghost set as the oracle's, the grid identical after every
step, omega within the FP64 field bound, k and beta equal."""

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


@pytest.mark.parametrize("p", [2, 3])
def test_nine_level_steps_match_oracle(p):
    prm = small_params(n0=4, J=8, eps=1e-3, m=20, p=p)
    cfg = oracle_config(prm)
    v = W.fujiwhara_small().vortices
    st = O.initial_state(cfg, v.xc, v.yc, v.gamma, v.s)
    lev = O.levels(cfg.n0, cfg.J)
    with B.Run(prm) as run:
        run.set_grid(st.active, st.omega)
        jx, jy = O.stencil_levels(st.active, lev, cfg.J)
        ghosts = O.ghost_set(st.active, jx, jy, cfg.J, cfg.p)
        _, gho, _ = run.masks()
        assert np.array_equal(gho, ghosts)
        ghost_levels = {int(j) for j in np.unique(lev[ghosts])}
        assert len(ghost_levels) >= 4, ghost_levels     # chains through several levels
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
            assert np.array_equal(idx, np.flatnonzero(st.active.ravel()))
            assert rel_l2(om, st.omega[st.active]) <= 1e-10
