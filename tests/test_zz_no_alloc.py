"""The allocation-free diagnostics entry point, for callers that cannot
allocate device memory (inside stream capture, under a framework that owns
the device memory, in real-time loops).  Checked through the C ABI against
wrc_diagnostics on the same state, on two calls in a row (the shared scratch
keeps the previous call's contents, so the second call checks that the entry
point clears what must start at zero).  This file is collected last."""

import numpy as np
import pytest

from paper_1604_08159_gb300 import binding as B
from paper_1604_08159_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def test_noalloc_diagnostics_match_wrc_diagnostics_twice():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1604_08159_gb300 import build
    build.build()
    B.load()
    wl = W.fujiwhara_small()
    p = W.RunParams(**{**wl.params.as_dict(), "sgs": W.SGS_DYNAMIC, "cs": 0.17})
    with B.Run(p) as run:
        run.init_vortices(wl.vortices)
        run.step(3)
        run.sync()
        ref = run.diagnostics()
        NJ = run.NJ
        omega = torch.empty(NJ * NJ, dtype=torch.float64, device="cuda")
        psi = torch.empty(NJ * NJ, dtype=torch.float64, device="cuda")
        B.wrc_query_field(run.h, B.FIELD_OMEGA, omega)
        B.wrc_query_field(run.h, B.FIELD_PSI, psi)
        expect = np.array([ref["E"], ref["Z"], ref["P"], ref["circulation"]])
        for _ in range(2):
            out = torch.full((4,), float("nan"), dtype=torch.float64, device="cuda")
            B.wrc_lattice_diagnostics_noalloc(omega, psi, NJ, out)
            torch.cuda.synchronize()
            got = out.cpu().numpy()
            np.testing.assert_allclose(got, expect, rtol=1e-12, atol=0)
    with pytest.raises(B.WrcError):
        B.wrc_lattice_diagnostics_noalloc(omega, psi, 100, out)     # not a power of two
