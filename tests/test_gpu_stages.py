"""Stage timing (wrc_profile mode 3): the step's results do not change, every
stage of every step is timed, and the stages add up to no more than the
steps' own event-timed duration."""

import numpy as np
import pytest

from paper_1604_08159_gb300 import binding as B
from paper_1604_08159_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1604_08159_gb300 import build
    build.build()
    B.load()


@pytest.mark.parametrize("prec", [W.PREC_FP64, W.PREC_MIXED])
def test_stage_timing_leaves_results_unchanged_and_covers_the_step(prec):
    import torch
    p = W.RunParams(**{**W.fujiwhara_small().params.as_dict(), "prec": prec,
                       "sgs": W.SGS_DYNAMIC, "cs": 0.17})
    v = W.fujiwhara_small().vortices
    nsteps = 4
    outs = []
    for mode in (0, 3):
        stream = torch.cuda.Stream()           # graphs on, except while stages are timed
        with B.Run(p, stream=stream.cuda_stream) as run:
            run.init_vortices(v)
            run.step(2)
            run.sync()
            run.profile(mode)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            run.step(nsteps)
            e1.record(stream)
            run.sync()
            outs.append(run.active())
            if mode == 3:
                steps, ms = run.stages()
                total = e0.elapsed_time(e1)
                assert steps == nsteps
                assert set(ms) == set(B.STAGES)
                assert all(t >= 0.0 for t in ms.values())
                for name in ("reconstruct", "poisson", "velocity", "sgs", "krylov", "adapt"):
                    assert ms[name] > 0.0, name
                assert sum(ms.values()) <= 1.001 * total + 1e-3
                assert sum(ms.values()) >= 0.5 * total
                run.profile(0)
                with pytest.raises(B.WrcError) as e:
                    run.stages()
                assert e.value.status == -7
    assert np.array_equal(outs[0][0], outs[1][0])
    assert np.array_equal(outs[0][1], outs[1][1])


def test_stage_record_restarts_and_rejects_bad_modes():
    p = W.fujiwhara_small().params
    with B.Run(p) as run:
        run.init_vortices(W.fujiwhara_small().vortices)
        run.profile(3)
        run.step(2)
        assert run.stages()[0] == 2
        run.profile(3)                          # enabling again clears the record
        assert run.stages() == (0, {s: 0.0 for s in B.STAGES})
        run.step(1)
        assert run.stages()[0] == 1
        with pytest.raises(B.WrcError):
            run.profile(4)
