"""Request server: continuous batching of runs that arrive over time.

Each result must be the same alone and in the mix -- a run that joins a batch
already stepping other runs (of other sizes and precisions), and that others
join while it runs, ends with the grid of its solo run and its values within
the stated tolerance (FP64 1e-12, mixed 1e-6: only the block split of its
reductions differs).  Admission must respect the slot count and the HBM
budget in arrival order; a run that fails leaves the others unharmed."""

import numpy as np
import pytest

from oracle import wrc_oracle as O
from paper_1604_08159_gb300 import binding as B
from paper_1604_08159_gb300 import workloads as W

from helpers import oracle_config, rel_l2

pytestmark = pytest.mark.gpu

TOL = {W.PREC_FP64: 1e-12, W.PREC_MIXED: 1e-6}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1604_08159_gb300 import build
    build.build()
    B.load()


def params(n0, J, prec, seed, **kw):
    rng = np.random.default_rng(seed)
    base = dict(n0=n0, J=J, eps=1e-4, re=float(rng.uniform(5000, 37440)), dt=1e-2, m=20,
                sgs=W.SGS_DYNAMIC, cs=0.17, prec=prec)
    base.update(kw)
    return W.RunParams(**base)


def pair(seed):
    rng = np.random.default_rng(seed)
    d = rng.uniform(0.8, 2.0)
    return W.Vortices(np.array([-0.5 * d, 0.5 * d]), np.zeros(2), np.array([1.0, rng.uniform(0.5, 1.0)]),
                      np.array([0.3, 0.3]))


def run_solo(p, v, nsteps):
    with B.Run(p) as run:
        run.init_vortices(v)
        run.step(nsteps)
        run.sync()
        idx, om = run.active()
        return idx, om, run.diagnostics()


def overlaps(a, b):
    return a.t_admit < b.t_done and b.t_admit < a.t_done


def test_each_result_same_alone_and_in_the_mix():
    # long runs start the batch; the targets arrive while it steps, and one
    # more arrives while the targets run
    long_ = [(params(32, 3, W.PREC_FP64, 1), pair(1), 600, 0.0),
             (params(32, 4, W.PREC_MIXED, 2), pair(2), 500, 0.0),
             (params(16, 3, W.PREC_FP64, 3, eps=1e-3, sgs=W.SGS_OFF), pair(3), 600, 0.0)]
    targets = [(params(32, 2, W.PREC_FP64, 4), pair(4), 12, 0.15),
               (params(32, 3, W.PREC_MIXED, 5), pair(5), 10, 0.15),
               (params(16, 3, W.PREC_FP64, 6, m=30), W.random_field_params(seed=6, n=3), 8, 0.3)]
    late = [(params(32, 2, W.PREC_MIXED, 7), pair(7), 20, 0.35)]
    reqs = long_ + targets + late
    with B.Server(max_slots=16) as srv:
        ids = [srv.submit(p, v, n, t) for p, v, n, t in reqs]
        srv.wait(timeout_s=600)
        infos = [srv.query(i) for i in ids]
        for i, info in zip(ids, infos):
            assert info.state == B.REQ_DONE, srv.error(i)
        results = [srv.result(i) for i in ids]
        st = srv.stats()
    assert st["done"] == len(reqs) and st["failed"] == 0 and st["peak_resident"] >= 4
    nl, nt = len(long_), len(targets)
    for k in range(nl, nl + nt):
        tgt = infos[k]
        # the mix was real: admitted while long runs were stepping, and
        # overlapped by a run admitted after it
        assert any(infos[j].t_admit < tgt.t_admit and overlaps(infos[j], tgt) for j in range(nl)), \
            "target did not join a running batch"
        assert tgt.steps == reqs[k][2]
    for (p, v, n, _), info, (idx, om) in zip(reqs, infos, results):
        ridx, rom, rdiag = run_solo(p, v, n)
        assert np.array_equal(idx, ridx), "grid differs from the solo run"
        assert rel_l2(om, rom) <= TOL[p.prec]
        assert info.n_active == ridx.size and info.steps == n
        for k, key in enumerate(("E", "Z", "P")):
            assert abs(info.diag[k] - rdiag[key]) <= 1e3 * TOL[p.prec] * abs(rdiag[key]), key
        assert info.t_arrival <= info.t_admit <= info.t_done


def test_request_in_the_mix_matches_oracle():
    wl = W.fujiwhara_small()
    p, v = wl.params, wl.vortices
    cfg = oracle_config(p)
    st = O.initial_state(cfg, v.xc, v.yc, v.gamma, v.s)
    d = np.abs(O.details(O.vortex_field(cfg.NJ, v.xc, v.yc, v.gamma, v.s), np.ones_like(st.active), cfg.J))
    if (np.abs(d - cfg.eps) < 1e-12 * cfg.eps).any():
        pytest.skip("a detail lies within rounding of eps")
    nsteps = 3
    for _ in range(nsteps):
        st, _ = O.step(cfg, st)
    with B.Server(max_slots=8) as srv:
        others = [srv.submit(params(32, 3, W.PREC_MIXED, 11), pair(11), 200, 0.0),
                  srv.submit(params(32, 2, W.PREC_FP64, 12), pair(12), 200, 0.0)]
        rid = srv.submit(p, v, nsteps, 0.05)
        srv.wait(timeout_s=600)
        assert all(srv.query(i).state == B.REQ_DONE for i in others + [rid])
        idx, om = srv.result(rid)
        info = srv.query(rid)
    assert np.array_equal(idx, np.flatnonzero(st.active.ravel()))
    assert rel_l2(om, st.omega[st.active]) <= 1e-10
    od = O.diagnostics(cfg, st)
    for k, key in enumerate(("E", "Z", "P", "circulation")):
        assert abs(info.diag[k] - od[key]) <= 1e-10 * max(abs(od[key]), 1e-300), key


def test_admission_by_hbm_budget_and_slots_in_arrival_order():
    p = params(32, 3, W.PREC_FP64, 20)
    est = B.wrc_server_estimate(B.make_config(p))
    budget = 2.5 * est
    with B.Server(max_slots=16, hbm_budget_bytes=budget) as srv:
        ids = [srv.submit(p, pair(20 + k), 30, 0.0) for k in range(6)]
        # a run that can never fit is refused at once
        big = params(32, 5, W.PREC_FP64, 21)
        with pytest.raises(B.WrcError) as e:
            srv.submit(big, pair(21), 1, 0.0)
        assert e.value.status == -6
        srv.wait(timeout_s=600)
        infos = [srv.query(i) for i in ids]
        st = srv.stats()
    assert all(i.state == B.REQ_DONE for i in infos)
    print("estimate", est, "charged", [i.charged_bytes for i in infos], "peak", st["peak_charged_bytes"])
    assert st["peak_resident"] == 2              # two fit the budget, the third does not
    # charged = max(estimate, bytes held): within the budget unless a run grew past its estimate
    assert st["peak_charged_bytes"] <= max(budget, 2 * max(i.charged_bytes for i in infos))
    assert st["charged_bytes"] == 0 and st["resident"] == 0
    admits = [i.t_admit for i in infos]
    assert admits == sorted(admits)              # arrival order
    assert all(i.charged_bytes >= est for i in infos)
    with B.Server(max_slots=3) as srv:
        ids = [srv.submit(params(32, 2, W.PREC_MIXED, 30 + k), pair(30 + k), 25, 0.0) for k in range(8)]
        srv.wait(timeout_s=600)
        st = srv.stats()
    assert st["done"] == 8 and st["peak_resident"] == 3


def test_fifo_policy_is_the_solo_path():
    reqs = [(params(32, 2, W.PREC_FP64, 40), pair(40), 15), (params(32, 3, W.PREC_MIXED, 41), pair(41), 10)]
    with B.Server(policy=B.SERVE_FIFO) as srv:
        ids = [srv.submit(p, v, n, 0.0) for p, v, n in reqs]
        srv.wait(timeout_s=600)
        got = [srv.result(i) for i in ids]
        infos = [srv.query(i) for i in ids]
        st = srv.stats()
    assert st["peak_resident"] == 1
    assert infos[1].t_admit >= infos[0].t_done
    for (p, v, n), (idx, om) in zip(reqs, got):
        ridx, rom, _ = run_solo(p, v, n)
        assert np.array_equal(idx, ridx)
        assert np.array_equal(om, rom)           # the same launches: bit-identical


def test_failed_run_leaves_the_others_unharmed():
    good = [(params(32, 2, W.PREC_FP64, 50), pair(50), 12), (params(32, 3, W.PREC_FP64, 51), pair(51), 12)]
    # vorticity of order 1e200: the operator overflows, the Arnoldi process
    # meets non-finite values and the run fails with WRC_ERR_BREAKDOWN_NAN
    bad_v = W.Vortices(np.array([0.0]), np.array([0.0]), np.array([1e200]), np.array([0.3]))
    with B.Server(max_slots=8) as srv:
        ids = [srv.submit(p, v, n, 0.0) for p, v, n in good]
        bad = srv.submit(params(32, 2, W.PREC_FP64, 52), bad_v, 12, 0.0)
        srv.wait(timeout_s=600)
        info = srv.query(bad)
        assert info.state == B.REQ_FAILED and info.status == -4, srv.error(bad)
        assert "non-finite" in srv.error(bad)
        got = [srv.result(i) for i in ids]
        st = srv.stats()
    assert st["failed"] == 1 and st["done"] == 2 and st["fatal"] == 0
    for (p, v, n), (idx, om) in zip(good, got):
        ridx, rom, _ = run_solo(p, v, n)
        assert np.array_equal(idx, ridx)
        assert rel_l2(om, rom) <= TOL[p.prec]


def test_wait_timeout_release_and_destroy_with_work_left():
    srv = B.Server(max_slots=2)
    rid = srv.submit(params(32, 3, W.PREC_FP64, 60), pair(60), 100000, 0.0)
    later = srv.submit(params(32, 2, W.PREC_FP64, 61), pair(61), 5, 1e6)   # arrives far in the future
    with pytest.raises(B.WrcError) as e:
        srv.wait(rid, timeout_s=0.2)
    assert e.value.status == -5
    assert srv.query(rid).state == B.REQ_RUNNING and srv.query(later).state == B.REQ_QUEUED
    with pytest.raises(B.WrcError):
        srv.release(rid)                          # not finished
    quick = srv.submit(params(32, 2, W.PREC_MIXED, 62), pair(62), 3, 0.0)
    srv.wait(quick, timeout_s=600)
    assert srv.query(quick).state == B.REQ_DONE
    srv.release(quick)
    with pytest.raises(B.WrcError):
        srv.query(quick)
    srv.close()                                   # fails the resident and the queued request
