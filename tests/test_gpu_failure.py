"""Failure detection on the GPU without a fault: bounded device-side waits
(grid barriers of the Krylov kernel, the ghost-row ready flags) that run
out and report WRC_ERR_TIMEOUT, the time limit of wrc_sync, and
the fallback of the Krylov launch to its unclustered form when a launch
path does not form thread-block clusters (made to happen by a test switch
that has the first clustered launch behave exactly as it does when its
clusters are missing)."""

import json
import os
import subprocess
import sys

import numpy as np
import pytest

from oracle import wrc_oracle as O
from paper_1604_08159_gb300 import binding as B
from paper_1604_08159_gb300 import workloads as W

from helpers import oracle_config, rel_l2

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1604_08159_gb300 import build
    build.build()
    B.load()


def _oracle_steps(p, v, n):
    cfg = oracle_config(p)
    st = O.initial_state(cfg, v.xc, v.yc, v.gamma, v.s)
    for _ in range(n):
        st, _ = O.step(cfg, st)
    return st


def _check_against(run, st):
    idx, om = run.active()
    assert np.array_equal(idx, np.flatnonzero(st.active.ravel()))
    assert rel_l2(om, st.omega[st.active]) <= 1e-10


@pytest.mark.parametrize("cluster_cap", [None, "1"])
def test_grid_barrier_wait_limit_runs_out(cluster_cap, monkeypatch):
    """A wait limit of 100 ns: a grid barrier of the Krylov kernel runs out,
    every block returns (clustered blocks after passing the same cluster
    barriers as their peers), the step reports WRC_ERR_TIMEOUT, and the run
    can be re-initialised and stepped correctly; a fresh run afterwards
    steps correctly too."""
    import torch
    if cluster_cap:
        monkeypatch.setenv("WRC_KRYLOV_CLUSTER", cluster_cap)
    wl = W.fujiwhara_small()
    p = W.RunParams(**{**wl.params.as_dict(), "sgs": W.SGS_DYNAMIC, "cs": 0.17})
    v = wl.vortices
    st2 = _oracle_steps(p, v, 2)
    stream = torch.cuda.Stream()
    with B.Run(p, stream=stream.cuda_stream) as run:
        run.init_vortices(v)
        if cluster_cap:
            assert run.krylov_form() == 1
        run.set_wait_limit(1e-7)
        with pytest.raises(B.WrcError) as e:
            run.step(1)
        assert e.value.status == -5, e.value
        run.sync()                                  # the context is still usable
        run.set_wait_limit(2.0)
        run.init_vortices(v)                        # state is undefined until re-initialised
        run.step(2)
        run.sync()
        _check_against(run, st2)
    with B.Run(p, stream=stream.cuda_stream) as fresh:
        fresh.init_vortices(v)
        fresh.step(2)
        fresh.sync()
        _check_against(fresh, st2)


def test_scalar_pair_wait_limit_runs_out():
    """The passive scalar's step runs omega and r_v as two problems of one
    cooperative launch, each with its own grid barrier.  With a wait limit
    of 100 ns a barrier runs out and the step reports WRC_ERR_TIMEOUT; after
    re-initialising, both problems' barriers start clean and the next steps
    match the oracle's omega and r_v."""
    import torch
    from helpers import small_params
    p = small_params(n0=16, J=3, eps=1e-3, re=2000.0, m=16)
    cfg = oracle_config(p)
    v = W.fujiwhara_small().vortices
    kappa = 2e-3
    x = -np.pi + cfg.h * np.arange(cfg.NJ)
    X, Y = np.meshgrid(x, x)
    front = 0.5 * (1.0 + np.tanh((Y - 0.3 * np.sin(X)) / 0.2))
    st = O.initial_state(cfg, v.xc, v.yc, v.gamma, v.s)
    st, rv = O.scalar_init(cfg, st, front)
    stream = torch.cuda.Stream()
    with B.Run(p, stream=stream.cuda_stream) as run:
        st0 = O.initial_state(cfg, v.xc, v.yc, v.gamma, v.s)
        run.set_grid(st0.active, st0.omega)
        run.scalar_init(kappa, front)
        run.set_wait_limit(1e-7)
        with pytest.raises(B.WrcError) as e:
            run.step(1)
        assert e.value.status == -5, e.value
        run.sync()
        run.set_wait_limit(2.0)
        run.set_grid(st0.active, st0.omega)
        run.scalar_init(kappa, front)
        for _ in range(2):
            st, rv, _, _ = O.step_with_scalar(cfg, st, rv, kappa)
        run.step(2)
        run.sync()
        _check_against(run, st)
        idx, r = run.scalar()
        assert np.array_equal(idx, np.flatnonzero(st.active.ravel()))
        assert rel_l2(r, rv[st.active]) <= 1e-10


def test_ghost_row_wait_limit_runs_out(monkeypatch):
    """The interpolation rows of all ghosts are built in one launch in which
    a ghost waits (bounded by the wait limit) for the rows of its coarser
    ghost predictors.  With the test switch WRC_TEST_GHOST_STALL=1 the first
    ghost's warp waits for a flag nothing sets: the wait runs out after the
    limit, the next step reports WRC_ERR_TIMEOUT, and after re-initialising
    without the switch the run steps like the oracle."""
    import torch
    wl = W.fujiwhara_small()
    p = W.RunParams(**{**wl.params.as_dict(), "sgs": W.SGS_DYNAMIC, "cs": 0.17})
    v = wl.vortices
    st2 = _oracle_steps(p, v, 2)
    stream = torch.cuda.Stream()
    with B.Run(p, stream=stream.cuda_stream) as run:
        run.set_wait_limit(0.01)
        monkeypatch.setenv("WRC_TEST_GHOST_STALL", "1")
        run.init_vortices(v)                        # the rebuild's ghost rows: one wait runs out
        monkeypatch.delenv("WRC_TEST_GHOST_STALL")
        assert run.counts()[1] > 0
        with pytest.raises(B.WrcError) as e:
            run.step(1)
        assert e.value.status == -5, e.value
        run.sync()
        run.set_wait_limit(2.0)
        run.init_vortices(v)
        run.step(2)
        run.sync()
        _check_against(run, st2)


def test_wait_limit_rejects_out_of_range():
    wl = W.fujiwhara_small()
    with B.Run(wl.params) as run:
        for bad in (0.0, -1.0, 61.0, float("nan")):
            with pytest.raises(B.WrcError) as e:
                run.set_wait_limit(bad)
            assert e.value.status == -1


def test_sync_time_limit():
    """wrc_sync(run, t) returns WRC_ERR_TIMEOUT while the run's stream is still
    busy (a spin kernel queued on it) and leaves the work queued; an
    unbounded wrc_sync then waits for it."""
    import torch
    wl = W.fujiwhara_small()
    stream = torch.cuda.Stream()
    with B.Run(wl.params, stream=stream.cuda_stream) as run:
        run.init_vortices(wl.vortices)
        run.sync()
        with torch.cuda.stream(stream):
            torch.cuda._sleep(400_000_000)          # ~0.2 s of clock cycles
        with pytest.raises(B.WrcError) as e:
            run.sync(0)
        assert e.value.status == -5
        run.sync(-1)
        run.sync(0)                                 # idle now: returns at once


_CHILD = r"""
import json, sys
sys.path.insert(0, {root!r})
sys.path.insert(0, {tests!r})
import torch
from paper_1604_08159_gb300 import binding as B
from paper_1604_08159_gb300 import workloads as W
B.load()
wl = W.fujiwhara_small()
p = W.RunParams(**{{**wl.params.as_dict(), "sgs": W.SGS_DYNAMIC, "cs": 0.17}})
stream = torch.cuda.Stream()
with B.Run(p, stream=stream.cuda_stream) as run:
    run.init_vortices(wl.vortices)
    before = run.krylov_form()
    run.step(2)
    run.sync()
    after = run.krylov_form()
    idx, om = run.active()
print(json.dumps({{"before": before, "after": after, "idx": idx.tolist(), "om": om.tolist()}}))
"""


def test_unformed_clusters_fall_back_to_unclustered_launch():
    """In a fresh process with the test switch WRC_KRYLOV_TEST_REFUSE=1 the
    first clustered Krylov launch behaves as when its clusters are missing:
    it runs as the unclustered kernel in the same launch and says so; the
    library keeps the device unclustered from then on, and the steps match
    the oracle and the clustered run."""
    import torch
    env = dict(os.environ, WRC_KRYLOV_TEST_REFUSE="1")
    env.pop("WRC_KRYLOV_CLUSTER", None)
    code = _CHILD.format(root=ROOT, tests=os.path.join(ROOT, "tests"))
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    out = json.loads(r.stdout.strip().splitlines()[-1])
    assert out["before"] > 1, "the workload should use a clustered launch"
    assert out["after"] == 1
    wl = W.fujiwhara_small()
    p = W.RunParams(**{**wl.params.as_dict(), "sgs": W.SGS_DYNAMIC, "cs": 0.17})
    st2 = _oracle_steps(p, wl.vortices, 2)
    idx = np.array(out["idx"])
    om = np.array(out["om"])
    assert np.array_equal(idx, np.flatnonzero(st2.active.ravel()))
    assert rel_l2(om, st2.omega[st2.active]) <= 1e-10
    stream = torch.cuda.Stream()
    with B.Run(p, stream=stream.cuda_stream) as run:
        run.init_vortices(wl.vortices)
        run.step(2)
        run.sync()
        cidx, com = run.active()
    assert np.array_equal(cidx, idx)
    assert rel_l2(com, om) <= 1e-12
