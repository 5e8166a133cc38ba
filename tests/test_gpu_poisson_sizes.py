"""Streamfunction and the spectral velocity and strain on every lattice size
the library accepts (NJ = 8 .. 4096): each FFT shape (a radix-2, -4 or -8
pass before the radix-16 passes, or a single 8-point transform) against the
oracle's solve of the same reconstructed field.

FP64: psi within OP_TOL of max|psi| at every point.  Mixed: psi, U, V and the
eddy viscosity nu_t (from the strain) within FP32 rounding of the FFT
(relative L2 5e-6; the FFT error grows like log2 NJ times the FP32 unit)."""

import numpy as np
import pytest

from oracle import wrc_oracle as O
from paper_1604_08159_gb300 import binding as B
from paper_1604_08159_gb300 import workloads as W

from helpers import oracle_config

pytestmark = pytest.mark.gpu

OP_TOL = 1e-12
FP32_TOL = 5e-6

SIZES = [(4, 1), (8, 1), (16, 1), (16, 2), (16, 3), (32, 3), (32, 4), (32, 5), (32, 6), (32, 7)]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1604_08159_gb300 import build
    build.build()
    B.load()


def field_for(NJ, seed):
    """Three Gaussian vortices (the workloads' large scales) plus a tenth of
    random Fourier modes up to NJ/4: every FFT bin is exercised, while psi
    keeps the vortices' low-wavenumber content, as in the runs (a field with
    only high modes would have a psi so small that FP32 rounding of the
    forward FFT, amplified by 1/sigma(k) at low k, dominates it)."""
    rng = np.random.default_rng(seed)
    v = W.random_field_params(seed=seed, n=3)
    f = O.vortex_field(NJ, v.xc, v.yc, v.gamma, v.s)
    x = -np.pi + 2 * np.pi * np.arange(NJ) / NJ
    X, Y = np.meshgrid(x, x, indexing="xy")
    for _ in range(12):
        kx, ky = rng.integers(0, max(1, NJ // 4) + 1, size=2)
        a, ph = rng.normal(), rng.uniform(0, 2 * np.pi)
        f += 0.1 * a * np.cos(kx * X + ky * Y + ph)
    return f


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("n0,J", SIZES)
def test_streamfunction_fp64_every_size(n0, J):
    p = W.RunParams(n0=n0, J=J, eps=0.0, re=5000.0)
    cfg = oracle_config(p)
    f = field_for(cfg.NJ, seed=cfg.NJ)
    with B.Run(p) as run:
        run.init_field(f)            # eps = 0: every point active, R(omega) = f
        run.freeze()
        psi = run.field(B.FIELD_PSI)
    ref = O.streamfunction(f, cfg.h)
    assert np.abs(psi - ref).max() <= OP_TOL * np.abs(ref).max()


@pytest.mark.parametrize("n0,J", SIZES)
def test_spectral_fields_mixed_every_size(n0, J):
    p = W.RunParams(n0=n0, J=J, eps=0.0, re=5000.0, sgs=W.SGS_DYNAMIC, cs=0.17, prec=W.PREC_MIXED)
    cfg = oracle_config(p)
    f = field_for(cfg.NJ, seed=cfg.NJ + 1)
    with B.Run(p) as run:
        run.init_field(f)
        run.freeze()
        got = {k: run.field(k) for k in (B.FIELD_PSI, B.FIELD_U, B.FIELD_V, B.FIELD_NUT)}
    Rf = f.astype(np.float32).astype(np.float64)   # the run holds omega in FP32
    psi = O.streamfunction(Rf, cfg.h)
    U, V = O.velocity(psi, cfg.h)
    S11, S12 = O.strain(psi, U, cfg.h)
    nut = O.smagorinsky_nut(S11, S12, cfg.cs, cfg.h)
    for k, ref in ((B.FIELD_PSI, psi), (B.FIELD_U, U), (B.FIELD_V, V), (B.FIELD_NUT, nut)):
        err = rel_l2(got[k], ref)
        assert err <= FP32_TOL, (k, err)
