"""ctypes binding of ``libwrc.so`` (include/wrc.h): argument marshalling only.

Every function below has the name of the C entry point it calls and does no
arithmetic of the method.  Host arrays are numpy arrays; device arrays are
CUDA tensors (``torch``), passed with ``device_ptr = 1``.  If the library is
missing, loading fails with an error: there is no fallback.
"""

from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, byref, c_double, c_int32, c_int64, c_uint8, c_void_p

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libwrc.so")

WRC_OK = 0
STATUS = {0: "WRC_OK", -1: "WRC_ERR_ARG", -2: "WRC_ERR_OOM", -3: "WRC_ERR_CUDA",
          -4: "WRC_ERR_BREAKDOWN_NAN", -5: "WRC_ERR_TIMEOUT", -6: "WRC_ERR_BUSY", -7: "WRC_ERR_STATE"}
FIELD_OMEGA, FIELD_PSI, FIELD_U, FIELD_V, FIELD_NUT = range(5)
MAX_M = 31
# stages of a step timed by wrc_profile(run, 3), in the order of the WRC_STAGE_* values
STAGES = ("reconstruct", "poisson", "velocity", "sgs", "krylov", "adapt", "host")


class WrcConfig(ctypes.Structure):
    _fields_ = [("n0", c_int32), ("J", c_int32), ("krylov_m", c_int32), ("sgs", c_int32),
                ("prec", c_int32), ("p", c_int32), ("eps", c_double), ("re", c_double),
                ("cs", c_double), ("s_apriori", c_double), ("rayleigh_r", c_double), ("dt", c_double),
                ("scheme", c_int32), ("model", c_int32), ("cpt", c_double), ("coriolis", c_double),
                ("gx", c_double), ("gy", c_double)]


class WrcServerConfig(ctypes.Structure):
    _fields_ = [("policy", c_int32), ("max_slots", c_int32), ("threads_per_block", c_int32),
                ("points_per_thread", c_int32), ("hbm_budget_bytes", c_double)]


class WrcRequestInfo(ctypes.Structure):
    _fields_ = [("state", c_int32), ("status", c_int32), ("steps", c_int64), ("n_active", c_int64),
                ("n_ghost", c_int64), ("t_arrival", c_double), ("t_admit", c_double), ("t_done", c_double),
                ("diag", c_double * 4), ("time", c_double), ("updates", c_double), ("charged_bytes", c_double)]


SERVE_BATCHED, SERVE_FIFO = 0, 1
SCHEME_FROZEN, SCHEME_ROSENBROCK = 0, 1
MODEL_VORTICITY, MODEL_EXNER = 0, 1
REQ_QUEUED, REQ_RUNNING, REQ_DONE, REQ_FAILED = 0, 1, 2, 3

# name -> (restype, argtypes); the list of entry points of include/wrc.h
SIGNATURES = {
    "wrc_create": (c_int32, [POINTER(WrcConfig), c_void_p, POINTER(c_void_p)]),
    "wrc_init_vortices": (c_int32, [c_void_p, c_int32, c_void_p, c_void_p, c_void_p, c_void_p]),
    "wrc_init_field": (c_int32, [c_void_p, c_void_p, c_int32]),
    "wrc_set_grid": (c_int32, [c_void_p, c_void_p, c_void_p, c_int32]),
    "wrc_threshold": (c_int32, [c_void_p, c_double]),
    "wrc_step": (c_int32, [c_void_p, c_int32]),
    "wrc_sync": (c_int32, [c_void_p, c_int32]),
    "wrc_set_wait_limit": (c_int32, [c_void_p, c_double]),
    "wrc_query_krylov_form": (c_int32, [c_void_p, POINTER(c_int32)]),
    "wrc_query_counts": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p]),
    "wrc_query_active": (c_int32, [c_void_p, c_void_p, c_void_p, c_int64, c_int32]),
    "wrc_scalar_init": (c_int32, [c_void_p, c_double, c_void_p, c_int32]),
    "wrc_query_scalar": (c_int32, [c_void_p, c_void_p, c_void_p, c_int64, c_int32]),
    "wrc_exner_init": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p, c_int32]),
    "wrc_exner_init_vortices": (c_int32, [c_void_p, c_int32, c_void_p, c_void_p, c_void_p, c_void_p, c_double]),
    "wrc_query_exner": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_int64, c_int32]),
    "wrc_query_masks": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p, c_int32]),
    "wrc_query_details": (c_int32, [c_void_p, c_void_p, c_int64, c_int32]),
    "wrc_query_stencil_levels": (c_int32, [c_void_p, c_void_p, c_void_p, c_int64, c_int32]),
    "wrc_query_field": (c_int32, [c_void_p, c_int32, c_void_p, c_int32]),
    "wrc_freeze": (c_int32, [c_void_p]),
    "wrc_apply_operator": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p, c_int32]),
    "wrc_query_krylov": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "wrc_diagnostics": (c_int32, [c_void_p, c_void_p]),
    "wrc_query_stats": (c_int32, [c_void_p, c_void_p]),
    "wrc_profile": (c_int32, [c_void_p, c_int32]),
    "wrc_query_profile": (c_int32, [c_void_p, c_void_p]),
    "wrc_query_stages": (c_int32, [c_void_p, c_void_p, c_int32]),
    "wrc_query_phase_trace": (c_int32, [c_void_p, c_void_p, c_int32, POINTER(c_int32)]),
    "wrc_last_error": (ctypes.c_char_p, [c_void_p]),
    "wrc_destroy": (None, [c_void_p]),
    "wrc_lattice_diagnostics_noalloc": (c_int32, [c_void_p, c_void_p, c_int32, c_void_p, c_void_p]),
    "wrc_ensemble_create": (c_int32, [c_int32, c_void_p, c_void_p, POINTER(c_void_p)]),
    "wrc_ensemble_member": (c_int32, [c_void_p, c_int32, POINTER(c_void_p)]),
    "wrc_ensemble_step": (c_int32, [c_void_p, c_int32]),
    "wrc_ensemble_set_shape": (c_int32, [c_void_p, c_int32, c_int32]),
    "wrc_ensemble_tune": (c_int32, [c_void_p, c_int32, c_void_p]),
    "wrc_ensemble_stats": (c_int32, [c_void_p, c_void_p]),
    "wrc_ensemble_profile": (c_int32, [c_void_p, c_int32, c_void_p]),
    "wrc_ensemble_last_error": (ctypes.c_char_p, [c_void_p]),
    "wrc_ensemble_destroy": (None, [c_void_p]),
    "wrc_server_estimate": (c_int32, [POINTER(WrcConfig), POINTER(c_double)]),
    "wrc_server_create": (c_int32, [POINTER(WrcServerConfig), POINTER(c_void_p)]),
    "wrc_server_submit": (c_int32, [c_void_p, POINTER(WrcConfig), c_int32, c_void_p, c_void_p, c_void_p,
                                    c_void_p, c_int64, c_double, POINTER(c_int64)]),
    "wrc_server_query": (c_int32, [c_void_p, c_int64, POINTER(WrcRequestInfo)]),
    "wrc_server_result_active": (c_int32, [c_void_p, c_int64, c_void_p, c_void_p, c_int64]),
    "wrc_server_request_error": (c_int32, [c_void_p, c_int64, c_void_p, c_int64]),
    "wrc_server_wait": (c_int32, [c_void_p, c_int64, c_double]),
    "wrc_server_release": (c_int32, [c_void_p, c_int64]),
    "wrc_server_stats": (c_int32, [c_void_p, c_void_p]),
    "wrc_server_last_error": (ctypes.c_char_p, [c_void_p]),
    "wrc_server_destroy": (None, [c_void_p]),
}

_lib = None


class WrcError(RuntimeError):
    def __init__(self, fn: str, status: int, message: str):
        super().__init__(f"{fn} -> {STATUS.get(status, status)}: {message}")
        self.status = status
        self.message = message


def load(path: str | None = None) -> ctypes.CDLL:
    """Load libwrc.so (built by ``paper_1604_08159_gb300.build``)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"{p} is missing: run paper_1604_08159_gb300.build.build() (nvcc) first")
    lib = ctypes.CDLL(p)
    for name, (res, args) in SIGNATURES.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    if path is None:
        _lib = lib
    return lib


def _ptr(x):
    """(pointer, device_ptr flag) of a numpy array or a CUDA tensor; (None, 0) for None."""
    if x is None:
        return None, 0
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("host arrays must be C-contiguous")
        return x.ctypes.data, 0
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("device tensors must be contiguous")
        return x.data_ptr(), 1 if x.is_cuda else 0
    raise TypeError(f"unsupported buffer type {type(x)}")


def _check(fn: str, st: int, run=None):
    if st != WRC_OK:
        msg = load().wrc_last_error(run)
        raise WrcError(fn, st, msg.decode() if msg else "")


def _flag(*ptrs):
    flags = {f for _, f in ptrs if _ is not None}
    if len(flags) > 1:
        raise ValueError("mix of host and device buffers in one call")
    return flags.pop() if flags else 0


def make_config(params) -> WrcConfig:
    """WrcConfig from a ``workloads.RunParams``-like object."""
    return WrcConfig(params.n0, params.J, params.m, params.sgs, params.prec, getattr(params, "p", 2), params.eps,
                     params.re, params.cs, params.s_apriori, params.rayleigh_r, params.dt,
                     getattr(params, "scheme", 0), getattr(params, "model", 0), getattr(params, "cpt", 0.0),
                     getattr(params, "coriolis", 0.0), getattr(params, "gx", 0.0), getattr(params, "gy", 0.0))


# ---- entry points -------------------------------------------------------------

def wrc_create(cfg: WrcConfig, stream: int | None = None) -> int:
    h = c_void_p()
    _check("wrc_create", load().wrc_create(byref(cfg), c_void_p(stream or 0), byref(h)))
    return h.value


def wrc_init_vortices(run, xc, yc, gamma, s):
    arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in (xc, yc, gamma, s)]
    _check("wrc_init_vortices", load().wrc_init_vortices(run, arrs[0].size, *[a.ctypes.data for a in arrs]), run)


def wrc_init_field(run, omega):
    p, f = _ptr(omega)
    _check("wrc_init_field", load().wrc_init_field(run, p, f), run)


def wrc_set_grid(run, active, omega):
    pa, fa = _ptr(active)
    po, fo = _ptr(omega)
    _check("wrc_set_grid", load().wrc_set_grid(run, pa, po, _flag((pa, fa), (po, fo))), run)


def wrc_threshold(run, eps: float):
    _check("wrc_threshold", load().wrc_threshold(run, eps), run)


def wrc_step(run, nsteps: int = 1):
    _check("wrc_step", load().wrc_step(run, nsteps), run)


def wrc_sync(run, timeout_ms=-1):
    _check("wrc_sync", load().wrc_sync(run, int(timeout_ms)), run)


def wrc_set_wait_limit(run, seconds):
    _check("wrc_set_wait_limit", load().wrc_set_wait_limit(run, float(seconds)), run)


def wrc_query_krylov_form(run):
    """Thread-block cluster size (1, 2 or 4) of the run's next Krylov launch."""
    cl = c_int32(0)
    _check("wrc_query_krylov_form", load().wrc_query_krylov_form(run, byref(cl)), run)
    return int(cl.value)


def wrc_query_counts(run, J: int):
    na, ng = c_int64(), c_int64()
    per = np.zeros(J + 1, dtype=np.int64)
    _check("wrc_query_counts", load().wrc_query_counts(run, byref(na), byref(ng), per.ctypes.data), run)
    return na.value, ng.value, per


def wrc_query_active(run, idx_out=None, omega_out=None, cap: int = 0):
    pi, fi = _ptr(idx_out)
    po, fo = _ptr(omega_out)
    _check("wrc_query_active", load().wrc_query_active(run, pi, po, cap, _flag((pi, fi), (po, fo))), run)


def wrc_scalar_init(run, kappa: float, field):
    p, f = _ptr(field)
    _check("wrc_scalar_init", load().wrc_scalar_init(run, float(kappa), p, f), run)


def wrc_query_scalar(run, idx_out=None, r_out=None, cap: int = 0):
    pi, fi = _ptr(idx_out)
    pr, fr = _ptr(r_out)
    _check("wrc_query_scalar", load().wrc_query_scalar(run, pi, pr, cap, _flag((pi, fi), (pr, fr))), run)


def wrc_exner_init(run, u, v, pi):
    ps = [_ptr(x) for x in (u, v, pi)]
    _check("wrc_exner_init", load().wrc_exner_init(run, ps[0][0], ps[1][0], ps[2][0], _flag(*ps)), run)


def wrc_exner_init_vortices(run, xc, yc, gamma, s, pi0: float):
    arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in (xc, yc, gamma, s)]
    _check("wrc_exner_init_vortices",
           load().wrc_exner_init_vortices(run, arrs[0].size, *[a.ctypes.data for a in arrs], float(pi0)), run)


def wrc_query_exner(run, idx_out=None, u_out=None, v_out=None, pi_out=None, cap: int = 0):
    ps = [_ptr(x) for x in (idx_out, u_out, v_out, pi_out)]
    _check("wrc_query_exner", load().wrc_query_exner(run, *[p for p, _ in ps], cap, _flag(*ps)), run)


def wrc_query_masks(run, active=None, ghost=None, significant=None):
    ps = [_ptr(x) for x in (active, ghost, significant)]
    _check("wrc_query_masks", load().wrc_query_masks(run, ps[0][0], ps[1][0], ps[2][0], _flag(*ps)), run)


def wrc_query_details(run, d_out, cap: int):
    p, f = _ptr(d_out)
    _check("wrc_query_details", load().wrc_query_details(run, p, cap, f), run)


def wrc_query_stencil_levels(run, jx_out, jy_out, cap: int):
    px, fx = _ptr(jx_out)
    py, fy = _ptr(jy_out)
    _check("wrc_query_stencil_levels",
           load().wrc_query_stencil_levels(run, px, py, cap, _flag((px, fx), (py, fy))), run)


def wrc_query_field(run, which: int, out):
    p, f = _ptr(out)
    _check("wrc_query_field", load().wrc_query_field(run, which, p, f), run)


def wrc_freeze(run):
    _check("wrc_freeze", load().wrc_freeze(run), run)


def wrc_apply_operator(run, q, w, g_out=None):
    ps = [_ptr(x) for x in (q, w, g_out)]
    _check("wrc_apply_operator", load().wrc_apply_operator(run, ps[0][0], ps[1][0], ps[2][0], _flag(*ps)), run)


def wrc_query_krylov(run, m: int):
    beta, hl = c_double(), c_double()
    k = c_int32()
    H = np.zeros((m + 1) * m)
    y = np.zeros(m)
    _check("wrc_query_krylov",
           load().wrc_query_krylov(run, byref(beta), byref(k), byref(hl), H.ctypes.data, y.ctypes.data), run)
    return {"beta": beta.value, "k": k.value, "h_last": hl.value, "H": H.reshape(m + 1, m), "y": y}


def wrc_diagnostics(run):
    out = np.zeros(9)
    _check("wrc_diagnostics", load().wrc_diagnostics(run, out.ctypes.data), run)
    keys = ("E", "Z", "P", "circulation", "t", "nstep", "n_active", "n_ghost", "krylov_err")
    return dict(zip(keys, out.tolist()))


def wrc_query_stats(run):
    out = np.zeros(4, dtype=np.int64)
    _check("wrc_query_stats", load().wrc_query_stats(run, out.ctypes.data), run)
    return {"launches": int(out[0]), "steps": int(out[1]), "host_syncs": int(out[2]), "n_active": int(out[3])}


def wrc_profile(run, enable):
    """enable: False/0 off, True/1 event timing of the Krylov launches, 2 that
    and the phase trace, 3 stage timing (wrc_query_stages)."""
    _check("wrc_profile", load().wrc_profile(run, int(enable)), run)


def wrc_query_stages(run):
    """Steps timed and the total ms of each stage since wrc_profile(run, 3)."""
    out = np.zeros(1 + len(STAGES))
    _check("wrc_query_stages", load().wrc_query_stages(run, out.ctypes.data, out.size), run)
    return int(out[0]), dict(zip(STAGES, out[1:].tolist()))


def wrc_query_profile(run):
    out = np.zeros(4)
    _check("wrc_query_profile", load().wrc_query_profile(run, out.ctypes.data), run)
    return {"launches": int(out[0]), "ms": float(out[1]), "bytes": float(out[2]), "flops": float(out[3])}


def wrc_query_phase_trace(run):
    """Per grid barrier of the last traced Krylov launch: (first arrival,
    last arrival, last block, release of block 0) in microseconds."""
    cap = 4 * 128
    out = np.zeros(cap)
    n = c_int32()
    _check("wrc_query_phase_trace", load().wrc_query_phase_trace(run, out.ctypes.data, cap, byref(n)), run)
    return out[:4 * n.value].reshape(n.value, 4)


def wrc_last_error(run) -> str:
    m = load().wrc_last_error(run)
    return m.decode() if m else ""


def wrc_destroy(run):
    if run:
        load().wrc_destroy(run)


# ---- convenience wrapper -------------------------------------------------------

class Run:
    """One run on the current CUDA device (numpy in and out by default)."""

    def __init__(self, params, stream: int | None = None):
        self.params = params
        self.NJ = params.n0 << params.J
        self.J = params.J
        self.m = params.m
        self.h = wrc_create(make_config(params), stream)

    def close(self):
        if self.h:
            wrc_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def init_vortices(self, v):
        wrc_init_vortices(self.h, v.xc, v.yc, v.gamma, v.s)

    def init_field(self, omega):
        wrc_init_field(self.h, np.ascontiguousarray(omega, dtype=np.float64) if isinstance(omega, np.ndarray) else omega)

    def set_grid(self, active, omega):
        wrc_set_grid(self.h, np.ascontiguousarray(active, dtype=np.uint8), np.ascontiguousarray(omega, dtype=np.float64))

    def threshold(self, eps):
        wrc_threshold(self.h, eps)

    def step(self, n=1):
        wrc_step(self.h, n)

    def sync(self, timeout_ms=-1):
        wrc_sync(self.h, timeout_ms)

    def set_wait_limit(self, seconds):
        wrc_set_wait_limit(self.h, seconds)

    def krylov_form(self):
        return wrc_query_krylov_form(self.h)

    def counts(self):
        return wrc_query_counts(self.h, self.J)

    def active(self):
        na = self.counts()[0]
        idx = np.zeros(na, dtype=np.int32)
        om = np.zeros(na)
        wrc_query_active(self.h, idx, om, na)
        return idx, om

    def scalar_init(self, kappa, field):
        """Enable the passive scalar (vapour mixing ratio) from a lattice field."""
        wrc_scalar_init(self.h, kappa, np.ascontiguousarray(field, dtype=np.float64) if isinstance(field, np.ndarray)
                        else field)

    def scalar(self):
        na = self.counts()[0]
        idx = np.zeros(na, dtype=np.int32)
        r = np.zeros(na)
        wrc_query_scalar(self.h, idx, r, na)
        return idx, r

    def exner_init(self, u, v, pi):
        """Velocity-Exner initial condition from lattice fields u, v, pi."""
        arrs = [np.ascontiguousarray(a, dtype=np.float64) if isinstance(a, np.ndarray) else a for a in (u, v, pi)]
        wrc_exner_init(self.h, *arrs)

    def exner_init_vortices(self, vortices, pi0=1.0):
        wrc_exner_init_vortices(self.h, vortices.xc, vortices.yc, vortices.gamma, vortices.s, pi0)

    def exner(self):
        """(idx, u, v, pi) at the active points of a velocity-Exner run."""
        na = self.counts()[0]
        idx = np.zeros(na, dtype=np.int32)
        u, v, p = np.zeros(na), np.zeros(na), np.zeros(na)
        wrc_query_exner(self.h, idx, u, v, p, na)
        return idx, u, v, p

    def masks(self):
        n2 = self.NJ * self.NJ
        a, g, s = (np.zeros(n2, dtype=np.uint8) for _ in range(3))
        wrc_query_masks(self.h, a, g, s)
        return [x.reshape(self.NJ, self.NJ).astype(bool) for x in (a, g, s)]

    def details(self, count):
        d = np.zeros(count)
        wrc_query_details(self.h, d, count)
        return d

    def stencil_levels(self):
        na = self.counts()[0]
        jx = np.zeros(na, dtype=np.uint8)
        jy = np.zeros(na, dtype=np.uint8)
        wrc_query_stencil_levels(self.h, jx, jy, na)
        return jx, jy

    def field(self, which):
        out = np.zeros(self.NJ * self.NJ)
        wrc_query_field(self.h, which, out)
        return out.reshape(self.NJ, self.NJ)

    def freeze(self):
        wrc_freeze(self.h)

    def apply_operator(self, q):
        q = np.ascontiguousarray(q, dtype=np.float64)
        w = np.zeros_like(q)
        g = np.zeros_like(q)
        wrc_apply_operator(self.h, q, w, g)
        return w, g

    def krylov(self):
        return wrc_query_krylov(self.h, self.m)

    def diagnostics(self):
        return wrc_diagnostics(self.h)

    def stats(self):
        return wrc_query_stats(self.h)

    def profile(self, enable=True):
        wrc_profile(self.h, enable)

    def profile_record(self):
        return wrc_query_profile(self.h)

    def stages(self):
        return wrc_query_stages(self.h)

    def phase_trace(self):
        return wrc_query_phase_trace(self.h)


def wrc_lattice_diagnostics_noalloc(omega_lattice, psi_lattice, NJ: int, out, stream: int | None = None):
    """Device tensors in and out; allocates nothing on the device."""
    po, fo = _ptr(omega_lattice)
    pp, fp = _ptr(psi_lattice)
    pq, fq = _ptr(out)
    if not (fo and fp and fq):
        raise ValueError("wrc_lattice_diagnostics_noalloc takes device arrays")
    st = load().wrc_lattice_diagnostics_noalloc(po, pp, NJ, pq, c_void_p(stream or 0))
    if st != WRC_OK:
        raise WrcError("wrc_lattice_diagnostics_noalloc", st, "invalid argument or CUDA error")


# ---- batched ensemble ------------------------------------------------------------

def _echeck(fn: str, st: int, ens=None):
    if st != WRC_OK:
        msg = load().wrc_ensemble_last_error(ens)
        raise WrcError(fn, st, msg.decode() if msg else "")


def wrc_ensemble_create(cfgs, stream: int | None = None) -> int:
    arr = (WrcConfig * len(cfgs))(*cfgs)
    h = c_void_p()
    _echeck("wrc_ensemble_create", load().wrc_ensemble_create(len(cfgs), arr, c_void_p(stream or 0), byref(h)))
    return h.value


def wrc_ensemble_member(ens, member: int) -> int:
    h = c_void_p()
    _echeck("wrc_ensemble_member", load().wrc_ensemble_member(ens, member, byref(h)), ens)
    return h.value


def wrc_ensemble_step(ens, nsteps: int = 1):
    _echeck("wrc_ensemble_step", load().wrc_ensemble_step(ens, nsteps), ens)


def wrc_ensemble_set_shape(ens, threads_per_block: int, points_per_thread: int):
    _echeck("wrc_ensemble_set_shape", load().wrc_ensemble_set_shape(ens, threads_per_block, points_per_thread), ens)


def wrc_ensemble_tune(ens, steps_per_candidate: int = 1):
    out = np.zeros(2, dtype=np.int32)
    _echeck("wrc_ensemble_tune", load().wrc_ensemble_tune(ens, steps_per_candidate, out.ctypes.data), ens)
    return int(out[0]), int(out[1])


def wrc_ensemble_stats(ens):
    out = np.zeros(6, dtype=np.int64)
    _echeck("wrc_ensemble_stats", load().wrc_ensemble_stats(ens, out.ctypes.data), ens)
    keys = ("members", "n_active", "steps", "blocks", "threads_per_block", "points_per_thread")
    return dict(zip(keys, (int(x) for x in out)))


def wrc_ensemble_profile(ens, enable: bool):
    ms = c_double()
    _echeck("wrc_ensemble_profile", load().wrc_ensemble_profile(ens, 1 if enable else 0, byref(ms)), ens)
    return ms.value


def wrc_ensemble_last_error(ens) -> str:
    m = load().wrc_ensemble_last_error(ens)
    return m.decode() if m else ""


def wrc_ensemble_destroy(ens):
    if ens:
        load().wrc_ensemble_destroy(ens)


class Member(Run):
    """A member of an Ensemble: the Run interface on a borrowed handle."""

    def __init__(self, params, handle):
        self.params = params
        self.NJ = params.n0 << params.J
        self.J = params.J
        self.m = params.m
        self.h = handle

    def close(self):
        self.h = None          # owned by the ensemble


class Ensemble:
    """Members advanced together (one batched Krylov launch per step)."""

    def __init__(self, params_list, stream: int | None = None):
        self.params = list(params_list)
        self.h = wrc_ensemble_create([make_config(p) for p in self.params], stream)
        self.members = [Member(p, wrc_ensemble_member(self.h, i)) for i, p in enumerate(self.params)]

    def step(self, n=1):
        wrc_ensemble_step(self.h, n)

    def tune(self, steps_per_candidate=1):
        return wrc_ensemble_tune(self.h, steps_per_candidate)

    def set_shape(self, threads_per_block, points_per_thread):
        wrc_ensemble_set_shape(self.h, threads_per_block, points_per_thread)

    def stats(self):
        return wrc_ensemble_stats(self.h)

    def profile(self, enable=True):
        return wrc_ensemble_profile(self.h, enable)

    def sync(self):
        for m in self.members:
            m.sync()

    def close(self):
        if self.h:
            for m in self.members:
                m.close()
            wrc_ensemble_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---- request server -------------------------------------------------------------

def _scheck(fn: str, st: int, srv=None):
    if st != WRC_OK:
        msg = load().wrc_server_last_error(srv)
        raise WrcError(fn, st, msg.decode() if msg else "")


def wrc_server_estimate(cfg: WrcConfig) -> float:
    b = c_double()
    st = load().wrc_server_estimate(byref(cfg), byref(b))
    if st != WRC_OK:
        raise WrcError("wrc_server_estimate", st, "invalid configuration")
    return b.value


def wrc_server_create(policy: int = SERVE_BATCHED, max_slots: int = 256, hbm_budget_bytes: float = 150e9,
                      threads_per_block: int = 0, points_per_thread: int = 0) -> int:
    cfg = WrcServerConfig(policy, max_slots, threads_per_block, points_per_thread, hbm_budget_bytes)
    h = c_void_p()
    _scheck("wrc_server_create", load().wrc_server_create(byref(cfg), byref(h)))
    return h.value


def wrc_server_submit(srv, cfg: WrcConfig, xc, yc, gamma, s, nsteps: int, arrival_s: float = 0.0) -> int:
    arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in (xc, yc, gamma, s)]
    rid = c_int64()
    _scheck("wrc_server_submit", load().wrc_server_submit(
        srv, byref(cfg), arrs[0].size, *[a.ctypes.data for a in arrs], nsteps, arrival_s, byref(rid)), srv)
    return rid.value


def wrc_server_query(srv, rid: int) -> WrcRequestInfo:
    info = WrcRequestInfo()
    _scheck("wrc_server_query", load().wrc_server_query(srv, rid, byref(info)), srv)
    return info


def wrc_server_result_active(srv, rid: int, cap: int):
    idx = np.empty(cap, dtype=np.int32)
    om = np.empty(cap, dtype=np.float64)
    _scheck("wrc_server_result_active",
            load().wrc_server_result_active(srv, rid, idx.ctypes.data, om.ctypes.data, cap), srv)
    return idx, om


def wrc_server_request_error(srv, rid: int) -> str:
    buf = ctypes.create_string_buffer(1024)
    _scheck("wrc_server_request_error", load().wrc_server_request_error(srv, rid, buf, 1024), srv)
    return buf.value.decode()


def wrc_server_wait(srv, rid: int = -1, timeout_s: float = 600.0):
    _scheck("wrc_server_wait", load().wrc_server_wait(srv, rid, timeout_s), srv)


def wrc_server_release(srv, rid: int):
    _scheck("wrc_server_release", load().wrc_server_release(srv, rid), srv)


def wrc_server_stats(srv) -> dict:
    out = np.zeros(12, dtype=np.float64)
    _scheck("wrc_server_stats", load().wrc_server_stats(srv, out.ctypes.data), srv)
    keys = ("submitted", "done", "failed", "queued", "resident", "peak_resident", "charged_bytes",
            "peak_charged_bytes", "iterations", "updates", "clock_s", "fatal")
    return dict(zip(keys, out.tolist()))


def wrc_server_last_error(srv) -> str:
    msg = load().wrc_server_last_error(srv)
    return msg.decode() if msg else ""


def wrc_server_destroy(srv):
    load().wrc_server_destroy(srv)


class Server:
    """Request server: runs submitted with arrival times are admitted by slot
    and HBM budget and advanced together (continuous batching), or one at a
    time (FIFO)."""

    def __init__(self, policy: int = SERVE_BATCHED, max_slots: int = 256, hbm_budget_bytes: float = 150e9,
                 threads_per_block: int = 0, points_per_thread: int = 0):
        self.h = wrc_server_create(policy, max_slots, hbm_budget_bytes, threads_per_block, points_per_thread)

    def submit(self, params, vortices, nsteps: int, arrival_s: float = 0.0) -> int:
        return wrc_server_submit(self.h, make_config(params), vortices.xc, vortices.yc, vortices.gamma,
                                 vortices.s, nsteps, arrival_s)

    def query(self, rid: int) -> WrcRequestInfo:
        return wrc_server_query(self.h, rid)

    def result(self, rid: int):
        """(lattice indices, omega) of a finished request's final active set."""
        info = self.query(rid)
        if info.state != REQ_DONE:
            raise WrcError("result", -7, wrc_server_request_error(self.h, rid) or "request not done")
        return wrc_server_result_active(self.h, rid, int(info.n_active))

    def error(self, rid: int) -> str:
        return wrc_server_request_error(self.h, rid)

    def wait(self, rid: int = -1, timeout_s: float = 600.0):
        wrc_server_wait(self.h, rid, timeout_s)

    def release(self, rid: int):
        wrc_server_release(self.h, rid)

    def stats(self) -> dict:
        return wrc_server_stats(self.h)

    def close(self):
        if self.h:
            wrc_server_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
