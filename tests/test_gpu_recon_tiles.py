"""The one-launch tiled DD reconstruction R(omega) (Eq. 6) against the FP64
oracle, bit-exact, for every tile size the library can pick (64, 32, 16 and
the level-by-level kernels, WRC_RECON_TILE = 0) and the DD orders 2p = 4, 6,
8: lattices of one tile and of many, tiles smaller than the coarsest spacing
(their coarse regions overlap the periodic seam and wrap), and the level-0
region wider than the lattice."""

import numpy as np
import pytest

from oracle import wrc_oracle as O
from paper_1604_08159_gb300 import binding as B
from paper_1604_08159_gb300 import workloads as W

from helpers import oracle_config, small_params

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
    dict(n0=16, J=3, eps=1e-3, p=2),    # 128^2: two 64-tiles per row
    dict(n0=4, J=7, eps=1e-3, p=2),     # 512^2, coarsest spacing 128 > tile
    dict(n0=8, J=4, eps=1e-3, p=3),     # 128^2, 2p = 6
    dict(n0=4, J=5, eps=1e-3, p=4),     # 128^2, 2p = 8, coarse regions wider than the lattice
    dict(n0=4, J=1, eps=1e-2, p=2),     # 8^2: a single tile smaller than 64
    dict(n0=4, J=8, eps=1e-3, p=2),     # 1024^2, nine levels: coarse regions far wider than a tile
    dict(n0=4, J=8, eps=1e-3, p=4),     # the same with 2p = 8 (the largest shared-memory layout here)
]


@pytest.mark.parametrize("tile", ["0", "16", "32", "64"])
@pytest.mark.parametrize("case", CASES, ids=lambda c: f"n0{c['n0']}_J{c['J']}_p{c['p']}")
def test_reconstruction_bit_exact_for_every_tile(tile, case, monkeypatch):
    monkeypatch.setenv("WRC_RECON_TILE", tile)   # read at every reconstruction launch
    prm = small_params(**case)
    cfg = oracle_config(prm)
    v = W.random_field_params(seed=41, n=4)
    field = O.vortex_field(cfg.NJ, v.xc, v.yc, v.gamma, v.s)
    st = O.state_from_field(cfg, field)
    assert 0 < st.active.sum() < cfg.NJ ** 2
    with B.Run(prm) as run:
        run.init_field(field)
        act, _, _ = run.masks()
        assert np.array_equal(act, st.active)
        R = run.field(B.FIELD_OMEGA)
        assert np.array_equal(R, O.reconstruct(st.omega, st.active, cfg.J, case["p"]))


@pytest.mark.parametrize("case", [dict(n0=16, J=3, eps=1e-3, p=2, sgs=W.SGS_DYNAMIC, cs=0.17),
                                  dict(n0=8, J=4, eps=1e-3, p=3)],
                         ids=["p2_sgs", "p3"])
def test_steps_identical_for_every_tile(case, monkeypatch):
    """Every step reconstructs R(omega) before the Poisson solve with the
    tiled kernel.  Five steps give bit-identical grids and values for every
    tile size and for the level-by-level kernels, and match the oracle."""
    prm = small_params(**case)
    cfg = oracle_config(prm)
    v = W.fujiwhara_small().vortices
    st = O.initial_state(cfg, v.xc, v.yc, v.gamma, v.s)
    for _ in range(5):
        st, _ = O.step(cfg, st)
    out = {}
    for tile in ["0", "16", "32", "64"]:
        monkeypatch.setenv("WRC_RECON_TILE", tile)
        with B.Run(prm) as run:
            run.init_vortices(v)
            run.step(5)
            run.sync()
            out[tile] = run.active()
    idx0, om0 = out["0"]
    assert np.array_equal(idx0, np.flatnonzero(st.active.ravel()))
    assert np.linalg.norm(om0 - st.omega[st.active]) <= 1e-10 * np.linalg.norm(st.omega[st.active])
    for tile, (idx, om) in out.items():
        assert np.array_equal(idx, idx0), tile
        assert np.array_equal(om, om0), tile
