"""Benchmark: active-point updates/s of the Krylov-projected DD
wavelet-collocation step on GB300.

One step = one pass of the whole hot path (reconstruction, streamfunction,
velocity and Smagorinsky forcing, Krylov projection with the phi_1 update,
grid adaptation) over the active grid of the 1024^2 Fujiwhara pair workload
(coarsest 32^2, J = 5, eps = 1e-4, m = 30, dynamic Smagorinsky C_s = 0.17,
Re = 5000, dt = 1e-2, FP64).  One active-point update = one active point
advanced one full step.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank advances an independent replica (seed
offset by rank; no collective on the data path) and rank 0 prints the
whole-job line.  ``--impl reference`` times the FP64 CPU oracle on the host
cores instead (rank 0 only).

Rank 0 also adds two measurements of the batched forms: ``serving`` (a
sample of the Poisson-arrival serving trace through the continuous-batching
request server, p50/p99 time-to-result and throughput, against the plain
per-run FP64 FIFO) and ``ensemble`` (256 uneven members advanced together,
against members run alone in FP64).
"""

from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_1604_08159_gb300 import workloads as W  # noqa: E402

METRIC = "active-point updates/s"
UNIT = "updates/s"
FALLBACK_HBM_GBS = 6800.0
# FP64 rate of one GB300 (nominal, 1.25 TFLOP/s): the FP64 path's arithmetic
# ceiling, far below its HBM ceiling at this step's arithmetic intensity.
FP64_PEAK_GFLOPS = 1250.0
L2_FLUSH_BYTES = 256 << 20
REFERENCE_MAX_STEPS = 60


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


WORKLOADS = {
    # the headline configuration: 1024^2 pair, dynamic Smagorinsky, FP64
    "fujiwhara_1024": lambda rank: W.fujiwhara_1024(seed=2 + rank),
    # 4096^2 three-vortex configuration, mixed precision (for profiling)
    "three_vortex_4096": lambda rank: W.three_vortex_4096(seed=3 + rank),
}


def workload_for(rank: int, name: str = "fujiwhara_1024"):
    return WORKLOADS[name](rank)


def combine_ranks(dev_ms: float, upd: int, device):
    """Whole-job numbers over the ranks of an initialised process group: the
    slowest rank's device time (MAX) and the updates of all ranks (SUM).  A
    single process returns its own numbers."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return dev_ms, upd
    t = torch.tensor([dev_ms], dtype=torch.float64, device=device)
    u = torch.tensor([float(upd)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t[0]), int(u[0])


def oracle_config(p):
    from oracle import wrc_oracle as O
    return O.Config(n0=p.n0, J=p.J, eps=p.eps, re=p.re, dt=p.dt, m=p.m, sgs=p.sgs_name(), cs=p.cs,
                    s_apriori=p.s_apriori, rayleigh_r=p.rayleigh_r)


def time_oracle(wl, nsteps: int, warmup: int = 0):
    """Time the oracle (as it stands) for nsteps steps of the workload from
    its initial state; returns (updates/s, wall s, cores used, per-step N_a)."""
    from oracle import wrc_oracle as O
    cfg = oracle_config(wl.params)
    v = wl.vortices
    st = O.initial_state(cfg, v.xc, v.yc, v.gamma, v.s)
    for _ in range(warmup):
        st, _ = O.step(cfg, st)
    upd = 0
    t0 = time.perf_counter()
    c0 = os.times()
    for _ in range(nsteps):
        upd += int(st.active.sum())
        st, _ = O.step(cfg, st)
    wall = time.perf_counter() - t0
    c1 = os.times()
    cpu = (c1.user - c0.user) + (c1.system - c0.system)
    cores = max(1, int(round(cpu / wall))) if wall > 0 else 1
    return upd / wall, wall, cores, upd


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons, each stamped with
    the host time it arrived; the summary keeps the samples that fall inside
    the marked region (the timed steps)."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    PERIOD_MS = 20

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.lines = []            # (host time, csv line)
        self.region = None
        self._first = threading.Event()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.perf_counter(), line))
            self._first.set()

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", str(self.PERIOD_MS)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
            return self
        self.reader = threading.Thread(target=self._read, daemon=True)
        self.reader.start()
        self._first.wait(timeout=5.0)      # sampling is running before the region starts
        return self

    def mark(self, t0: float, t1: float):
        self.region = (t0, t1)

    def __exit__(self, *exc):
        if self.proc is None:
            return
        time.sleep(2e-3 * self.PERIOD_MS)  # one more period, so the region's end is covered
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            self.proc.wait()
        self.reader.join(timeout=5)

    def summary(self):
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        rows = []
        for t, line in self.lines:
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                rows.append((t, float(f[1]), float(f[2]), f[5:9]))
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        window = "timed region"
        if self.region is not None:
            t0, t1 = self.region
            # a sample reports the period that ends when it arrives
            sel = [r for r in rows if t0 < r[0] <= t1 + 1e-3 * self.PERIOD_MS]
            if not sel:
                sel = [min(rows, key=lambda r: abs(r[0] - t1))]
                window = "nearest sample to the timed region's end"
        else:
            sel, window = rows, "whole run"
        reasons = set()
        for r in sel:
            for name, val in zip(names, r[3]):
                if val.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(r[1] for r in sel), "sm_max_mhz": sel[-1][2],
                "reasons": sorted(reasons), "samples": len(sel), "period_ms": self.PERIOD_MS,
                "window": window}


# Algorithmic cost per step of the stages that have a simple model (bulk word
# size es; N = NJ^2 lattice points, na active points):
#   reconstruct  two inverse transforms per step, each writing every lattice
#                value and reading it and the mask once: 2 (2 es + 1) N bytes
#   poisson      two real 2-D FFTs of N points (forward, inverse) at the usual
#                2.5 N log2 N flops each: 5 N log2 N FP64 flops
#   velocity     meta, one psi word and U, V per active point: (4 + 3 es) na bytes
#   krylov       the Krylov launch's own model (wrc_query_profile)
#   adapt        the lattice masks read and written once each (significance,
#                next grid, ghosts, stencil levels, compaction keys), the
#                lattice-to-index map, and the new compact arrays:
#                13 N + (4 + es) na bytes
# The subgrid forcing and the host gap are reported by time only.
STAGE_BOUND = {"reconstruct": "hbm", "poisson": "alu", "velocity": "hbm", "sgs": "alu (FP64 over the halo list)",
               "krylov": "alu", "adapt": "hbm (small launches: latency)", "host": "host synchronisation"}


def stage_report(sms, nsteps, p, na, hbm_gbs):
    N = float(p.NJ) ** 2
    es = 4.0 if p.prec == W.PREC_MIXED else 8.0
    per = {k: v / max(1, nsteps) for k, v in sms.items()}
    total = sum(per.values())
    k = p.m
    krylov_flops = na * (30.0 * (k + 1) + 3.0 * k + sum(8.0 * (j + 1) + 4.0 for j in range(k)))
    model = {"reconstruct": ("bytes", 2.0 * (2.0 * es + 1.0) * N),
             "poisson": ("flops", 5.0 * N * math.log2(N)) if es == 8.0 else None,
             "velocity": ("bytes", (4.0 + 3.0 * es) * na),
             "krylov": ("flops", krylov_flops) if es == 8.0 else None,
             "adapt": ("bytes", 13.0 * N + (4.0 + es) * na)}
    out = {"steps": nsteps, "mean_active_points": na, "launch": "direct (graphs off while stages are timed)",
           "step_ms": total}
    for name in sms:   # the library's stage order
        ms = per.get(name, 0.0)
        row = {"ms_per_step": ms, "share": ms / total if total > 0 else 0.0, "bound": STAGE_BOUND[name]}
        m = model.get(name)
        if m is not None and ms > 0:
            kind, amount = m
            if kind == "bytes":
                a = amount / (ms * 1e-3) / 1e9
                row.update({"algorithmic_bytes": amount, "achieved": a, "unit": "GB/s", "peak": hbm_gbs,
                            "frac": a / hbm_gbs})
            else:
                a = amount / (ms * 1e-3) / 1e9
                row.update({"algorithmic_flops": amount, "achieved": a, "unit": "GFLOP/s",
                            "peak": FP64_PEAK_GFLOPS, "frac": a / FP64_PEAK_GFLOPS})
        out[name] = row
    return out


def hbm_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        try:
            d = json.load(open(path))
            for key in ("hbm_gbs", "hbm_GBs", "hbm"):
                if key in d:
                    v = d[key]
                    return float(v["value"] if isinstance(v, dict) else v), "measured"
        except (ValueError, KeyError, TypeError):
            pass
    return FALLBACK_HBM_GBS, "fallback"


def measure_serving(args):
    """Replay a sample of the serving trace (Poisson arrivals at 50/s of 2-3
    vortex runs, finest 128^2-4096^2) through the request server four times,
    so that batching and precision are measured apart: continuous batching in
    the mixed mode (the trace's precision) and in FP64, and the plain per-run
    form (FIFO, one run at a time) in both precisions.  Time-to-result is
    measured by the server from each request's arrival to its result on the
    host.  The mixed results' error is stated per request against the same
    request's FP64 per-run result (relative L2 of omega over the points
    active in both, and the count of points active in only one)."""
    import dataclasses

    from paper_1604_08159_gb300 import binding as B

    trace = W.serving_trace()[:args.serve_requests]
    scale = args.serve_step_scale

    def replay(policy, fp64, keep):
        with B.Server(policy=policy, max_slots=256, hbm_budget_bytes=150e9) as srv:
            t0 = srv.stats()["clock_s"] + 0.05
            ids = []
            for t, p, v, ns in trace:
                p = dataclasses.replace(p, prec=W.PREC_FP64 if fp64 else W.PREC_MIXED)
                ids.append(srv.submit(p, v, max(1, int(round(ns * scale))), t0 + t))
            srv.wait(timeout_s=3600)
            infos = [srv.query(i) for i in ids]
            st = srv.stats()
            results = [srv.result(i) if (keep and info.state == B.REQ_DONE) else None
                       for i, info in zip(ids, infos)]
        done = [i for i in infos if i.state == B.REQ_DONE]
        lat = np.array([i.t_done - i.t_arrival for i in done]) if done else np.zeros(1)
        upd = sum(i.updates for i in done)
        span = max(i.t_done for i in done) - min(i.t_arrival for i in infos) if done else 0.0
        return {"done": len(done), "failed": len(infos) - len(done),
                "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
                "throughput": upd / span if span > 0 else 0.0, "unit": UNIT,
                "requests_per_s": len(done) / span if span > 0 else 0.0, "makespan_s": span,
                "peak_resident": int(st["peak_resident"]), "peak_hbm_gb": st["peak_charged_bytes"] / 1e9}, results

    batched, res_bm = replay(B.SERVE_BATCHED, fp64=False, keep=True)
    batched64, res_b64 = replay(B.SERVE_BATCHED, fp64=True, keep=True)
    fifo_mixed, _ = replay(B.SERVE_FIFO, fp64=False, keep=False)
    fifo, res_f64 = replay(B.SERVE_FIFO, fp64=True, keep=True)

    def errors(res):
        rel, flips = [], []
        for a, b in zip(res, res_f64):
            if a is None or b is None:
                continue
            r, f = compare_results(a[0], a[1], b[0], b[1])
            rel.append(r)
            flips.append(f / max(1, b[0].size))
        if not rel:
            return None
        return {"requests": len(rel), "rel_l2_max": float(np.max(rel)), "rel_l2_median": float(np.median(rel)),
                "grid_diff_frac_max": float(np.max(flips)), "per_request_rel_l2": [float(x) for x in rel]}

    sizes = sorted({p.NJ for _, p, _, _ in trace})
    ratio = lambda a, b: a["throughput"] / b["throughput"] if b["throughput"] > 0 else None
    return {"sample": f"first {len(trace)} requests of the 50 req/s serving trace (seed 5), each run's step "
                      f"count scaled by {scale} (full trace: 200-2000 steps); lattices {sizes}",
            "batched_mixed": batched, "batched_fp64": batched64, "fifo_mixed": fifo_mixed, "fifo_fp64": fifo,
            "throughput_ratio": ratio(batched, fifo),
            "batching_gain_fp64": ratio(batched64, fifo), "batching_gain_mixed": ratio(batched, fifo_mixed),
            "precision_gain_batched": ratio(batched, batched64),
            "error_vs_fifo_fp64": {"batched_mixed": errors(res_bm), "batched_fp64": errors(res_b64),
                                   "measure": "relative L2 of omega over points active in both results; "
                                              "grid differences as a fraction of the FP64 active count"}}


def measure_ensemble(args):
    """The uneven ensemble (256 two-vortex members, finest 256^2-2048^2)
    advanced together -- one cooperative Krylov launch per step for all
    members, graph-replayed phases, autotuned block shape -- in the mixed
    mode and in FP64, against the plain per-run form (each member alone) in
    both precisions on a sample of the members, so that batching and
    precision are measured apart.  The batched Krylov launches are timed
    with events and set against the algorithmic bytes of the members' Krylov
    steps (the HBM fraction of the batched launch, whose working set exceeds
    L2).  Each mixed member's error is stated against its own FP64 batched
    result after the same steps."""
    import dataclasses

    import torch

    from paper_1604_08159_gb300 import binding as B

    peak, peak_src = hbm_peak()
    nsteps = args.ens_steps

    # every arm ends at the same step count (the tuner advances the members
    # by one step per shape it times: at most 9), so that the members' final
    # states can be compared
    final_steps = 2 + 9 + 1 + nsteps

    def batched(prec):
        members = W.ensemble_members(n=args.ens_members, prec=prec)
        stream = torch.cuda.Stream()
        with B.Ensemble([p for p, _ in members], stream=stream.cuda_stream) as ens:
            for m, (_, v) in zip(ens.members, members):
                m.init_vortices(v)
            ens.step(2)
            shape = ens.tune(1)
            ens.step(1)
            ens.sync()
            torch.cuda.synchronize()
            ens.profile(True)
            ens.profile(True)                  # clears the record: only the timed steps count
            upd = 0
            t0 = time.perf_counter()
            for _ in range(nsteps):
                upd += ens.stats()["n_active"]
                ens.step(1)
            ens.sync()
            torch.cuda.synchronize()
            wall = time.perf_counter() - t0
            kms = ens.profile(False)
            rest = final_steps - ens.stats()["steps"]
            if rest > 0:
                ens.step(rest)
            ens.sync()
            finals = [m.active() for m in ens.members]
        es = 4.0 if prec == W.PREC_MIXED else 8.0
        m = members[0][0].m
        kbytes = krylov_bytes_per_update(m, es) * upd
        kgbs = kbytes / (kms * 1e-3) / 1e9 if kms > 0 else 0.0
        return {"value": upd / wall, "unit": UNIT, "ms_per_ensemble_step": 1e3 * wall / nsteps,
                "block_shape": list(shape), "mean_active_points_total": upd / nsteps,
                "krylov_launch": {"bound": "hbm", "achieved": kgbs, "peak": peak, "unit": "GB/s",
                                  "frac": kgbs / peak, "peak_source": peak_src,
                                  "ms_per_step": kms / nsteps,
                                  "algorithmic_bytes_per_update": krylov_bytes_per_update(m, es),
                                  "working_set_bytes": (m + 1) * es * upd / nsteps}}, finals

    def per_run(prec):
        sample = W.ensemble_members(n=args.ens_members, prec=prec)[:args.ens_solo_sample]
        stream = torch.cuda.Stream()
        s_upd, s_wall = 0, 0.0
        for p, v in sample:
            with B.Run(p, stream=stream.cuda_stream) as run:
                run.init_vortices(v)
                run.step(2)
                run.sync()
                t1 = time.perf_counter()
                for _ in range(nsteps):
                    s_upd += run.stats()["n_active"]
                    run.step(1)
                run.sync()
                s_wall += time.perf_counter() - t1
        return s_upd / s_wall if s_wall > 0 else 0.0

    bm, fin_m = batched(W.PREC_MIXED)
    b64, fin_64 = batched(W.PREC_FP64)
    rel, flips = [], []
    for (ai, ao), (bi, bo) in zip(fin_m, fin_64):
        r, f = compare_results(ai, ao, bi, bo)
        rel.append(r)
        flips.append(f / max(1, bi.size))
    pm = per_run(W.PREC_MIXED)
    p64 = per_run(W.PREC_FP64)
    return {"members": args.ens_members, "steps": nsteps,
            "batched_mixed": bm, "batched_fp64": b64,
            "per_run_mixed": pm, "per_run_fp64": p64, "unit": UNIT,
            "per_run_sample": f"first {args.ens_solo_sample} members, each alone, {nsteps} steps after 2",
            "throughput_ratio": bm["value"] / p64 if p64 > 0 else None,
            "batching_gain_fp64": b64["value"] / p64 if p64 > 0 else None,
            "batching_gain_mixed": bm["value"] / pm if pm > 0 else None,
            "precision_gain_batched": bm["value"] / b64["value"] if b64["value"] > 0 else None,
            "mixed_error_vs_fp64": {"members": len(rel), "rel_l2_max": float(np.max(rel)),
                                    "rel_l2_median": float(np.median(rel)),
                                    "grid_diff_frac_max": float(np.max(flips)),
                                    "per_member_rel_l2": [float(x) for x in rel],
                                    "measure": f"each member after {final_steps} steps, mixed against FP64 "
                                               "(both batched), over points active in both"}}


def measure_scalar(args, wl):
    """The passive scalar of the water-vapour section on the same workload:
    r_v = 1 for y > 0, else 0 (the paper's initial condition), diffusivity
    1/Re, advanced with omega by every step on the grid that adapts to both
    fields.  Device time per step by CUDA events on the run's stream, after
    warm-up steps; updates count the active points (each advancing both
    fields)."""
    import numpy as np
    import torch

    from paper_1604_08159_gb300 import binding as B

    p = wl.params
    NJ = p.NJ
    y = -np.pi + (2.0 * np.pi / NJ) * np.arange(NJ)
    field = np.repeat((y > 0).astype(np.float64)[:, None], NJ, axis=1)   # [k, i]
    stream = torch.cuda.Stream()
    with B.Run(p, stream=stream.cuda_stream) as run:
        run.init_vortices(wl.vortices)
        na_omega = run.stats()["n_active"]
        run.scalar_init(1.0 / p.re, field)
        run.step(3)
        run.sync()
        n = max(1, min(args.steps, 10))
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        upd = 0
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(n):
            upd += run.stats()["n_active"]
            run.step(1)
        e1.record(stream)
        run.sync()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / n
    return {"initial_condition": "r_v = 1 for y > 0 else 0 (water-vapour section), kappa = 1/Re",
            "steps": n, "ms_per_step": ms, "mean_active_points": upd / n,
            "active_points_without_scalar": na_omega, "value": upd / (ms * 1e-3 * n),
            "unit": UNIT + " (both fields advanced per update)"}


def measure_exner(args):
    """The compressible velocity-Exner form (Eqs. 1-2) on the 1024^2 pair
    (``workloads.fujiwhara_exner_1024``): initial condition from the vortex
    parameters (the library's Poisson solve for the velocity, pi = 1), 3
    warm-up steps, then device time per step by CUDA events on the run's
    stream; an update advances the three fields at one active point."""
    import torch

    from paper_1604_08159_gb300 import binding as B

    wl = W.fujiwhara_exner_1024()
    stream = torch.cuda.Stream()
    with B.Run(wl.params, stream=stream.cuda_stream) as run:
        run.exner_init_vortices(wl.vortices, wl.extra["pi0"])
        run.step(3)
        run.sync()
        n = max(1, min(args.steps, 10))
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        upd = 0
        ks = []
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(n):
            upd += run.stats()["n_active"]
            run.step(1)
        e1.record(stream)
        run.sync()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / n
        kr = run.krylov()
        _, u, v, p = run.exner()
    return {"workload": wl.name, "scheme": "rosenbrock (exact Jacobian)", "cpt": wl.params.cpt,
            "coriolis": wl.params.coriolis, "steps": n, "ms_per_step": ms, "mean_active_points": upd / n,
            "krylov_k": kr["k"], "max_abs_pi_minus_1": float(abs(p - 1.0).max()),
            "value": upd / (ms * 1e-3 * n), "unit": UNIT + " (u, v and pi advanced per update)"}


def measure_variants(args):
    """The next rows of the 1024^2 pair's step, each timed alone: the
    exponential Rosenbrock-Euler step with the full Jacobian (a
    reconstruction and a Poisson solve per Krylov vector) and the DD orders
    2p = 6 and 8.  Same workload and initial condition; 3 warm-up steps, then
    device time per step by CUDA events on the run's stream."""
    import dataclasses

    import torch

    from paper_1604_08159_gb300 import binding as B

    wl = W.fujiwhara_1024()
    out = {}
    for name, change in (("rosenbrock", {"scheme": W.SCHEME_ROSENBROCK}), ("dd_order_6", {"p": 3}),
                         ("dd_order_8", {"p": 4})):
        prm = dataclasses.replace(wl.params, **change)
        stream = torch.cuda.Stream()
        with B.Run(prm, stream=stream.cuda_stream) as run:
            run.init_vortices(wl.vortices)
            run.step(3)
            run.sync()
            n = max(1, min(args.steps, 10))
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            upd = 0
            torch.cuda.synchronize()
            e0.record(stream)
            for _ in range(n):
                upd += run.stats()["n_active"]
                run.step(1)
            e1.record(stream)
            run.sync()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / n
            kr = run.krylov()
        out[name] = {"change": change, "steps": n, "ms_per_step": ms, "mean_active_points": upd / n,
                     "krylov_k": kr["k"], "value": upd / (ms * 1e-3 * n), "unit": UNIT}
    return out


KRYLOV_SOURCES = ("csrc/krylov_impl.cuh", "csrc/krylov.cu", "csrc/operator.cuh", "csrc/common.cuh",
                  "csrc/kernels.h")
# DRAM bytes per launch of the Krylov kernel on the 1024^2 pair, from one ncu
# capture (dram__bytes_read.sum + dram__bytes_write.sum), valid only for the
# kernel sources whose SHA-256 is recorded with it.
KRYLOV_TRAFFIC = {"sources_sha256": "64d894531698a095396417b05a59368f59e9683214113e97e53b3efff5e424de",
                  "bytes_per_launch": 2660864,
                  "capture": "ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum, clustered form "
                             "(the one timed), 1024^2 pair, third launch"}


def krylov_traffic():
    """DRAM bytes per Krylov launch from the recorded ncu capture, or None if
    there is none or the kernel's sources changed since it was taken."""
    import hashlib
    if not KRYLOV_TRAFFIC:
        return None
    h = hashlib.sha256()
    for f in KRYLOV_SOURCES:
        h.update(open(os.path.join(ROOT, "paper_1604_08159_gb300", f), "rb").read())
    return KRYLOV_TRAFFIC["bytes_per_launch"] if h.hexdigest() == KRYLOV_TRAFFIC["sources_sha256"] else None


def krylov_bytes_per_update(m: int, es: float) -> float:
    """Algorithmic bytes of the Krylov part per active-point update: m + 1
    operator applications reading q, U, V and writing w (4 words each), at
    Arnoldi step j a fused Gram-Schmidt pass reading j + 1 basis vectors and
    w twice and writing w (2(j + 1) + 3 words), the combination reading m
    vectors and omega and writing omega (m + 2 words): es (m^2 + 9m + 6)
    bytes, with es the bulk word size (8 in FP64, 4 in the mixed mode)."""
    return es * (m * m + 9.0 * m + 6.0)


def compare_results(a_idx, a_om, b_idx, b_om):
    """Relative L2 difference of omega over the lattice points active in
    both results, and the number of points active in only one of them."""
    common, ia, ib = np.intersect1d(a_idx, b_idx, assume_unique=True, return_indices=True)
    x, y = a_om[ia], b_om[ib]
    den = float(np.linalg.norm(y))
    rel = float(np.linalg.norm(x - y) / den) if den > 0 else 0.0
    flips = int(a_idx.size + b_idx.size - 2 * common.size)
    return rel, flips


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    wl = workload_for(0, args.workload)
    warm = min(args.warmup, 1)
    # one oracle step of the 1024^2 pair takes ~1.3 s on the host cores (of
    # the 4096^2 workload ~40-80 s): the sample is capped at 60 steps, and at
    # 2 steps at 4096^2, so that the run ends within a few minutes
    cap = REFERENCE_MAX_STEPS if wl.params.NJ < 4096 else 2
    nsteps = max(1, min(args.steps, cap))
    val, wall, cores, upd = time_oracle(wl, nsteps, warmup=warm)
    line = {
        "impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
        "steps": nsteps, "warmup": warm, "ms_per_step": 1e3 * wall / nsteps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": wl.name, "NJ": wl.params.NJ, "n0": wl.params.n0,
                                        "J": wl.params.J, "eps": wl.params.eps, "m": wl.params.m,
                                        "sgs": wl.params.sgs_name()},
        "cpu_baseline": {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{nsteps} oracle steps of {wl.name} after {warm} warm-up step(s)"
                                   + (f" ({args.steps} requested)" if nsteps != args.steps else "")},
        "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_1604_08159_gb300 import binding as B
    from paper_1604_08159_gb300 import build as BLD

    ws, rank, local = dist_env()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device (there is no CPU path)")
    torch.cuda.set_device(local)
    if ws > 1:
        backend = "nccl" if dist.is_nccl_available() else "gloo"
        dist.init_process_group(backend=backend)
    if rank == 0:
        BLD.build()
    if ws > 1:
        dist.barrier()
    B.load()

    wl = workload_for(rank, args.workload)
    p = wl.params
    stream = torch.cuda.Stream()
    run = B.Run(p, stream=stream.cuda_stream)
    run.init_vortices(wl.vortices)
    sampler = ClockSampler(local)
    sampler.__enter__()                  # sampling runs from the warm-up on
    run.step(args.warmup)
    run.sync()

    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    upd = 0
    l0 = run.stats()["launches"]
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    try:
        t0 = time.perf_counter()
        with torch.cuda.stream(stream):
            for q in range(args.steps):
                flush.zero_()                      # L2 flush between timed steps (outside the events)
                starts[q].record(stream)
                upd += run.stats()["n_active"]
                run.step(1)
                ends[q].record(stream)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        wall = t1 - t0
        sampler.mark(t0, t1)
    finally:
        sampler.__exit__(None, None, None)
    launches = run.stats()["launches"] - l0      # library kernels only (the flush is torch's)
    run.sync()
    dev_ms = sum(s.elapsed_time(e) for s, e in zip(starts, ends))

    # dominant kernel: the Krylov part of the step (cooperative Arnoldi kernel,
    # phi_1, update), timed with events on the run's stream in a window of
    # steps right after the timed region
    run.profile(True)
    prof_steps = min(args.steps, 5)
    run.step(prof_steps)
    rec = run.profile_record()
    run.profile(False)
    peak, peak_src = hbm_peak()
    sec = rec["ms"] * 1e-3
    es = 4.0 if p.prec == W.PREC_MIXED else 8.0
    # the library counts 8-byte words; the mixed mode's basis and stencil
    # vectors are 4 bytes (the byte model's half)
    kbytes = rec["bytes"] * es / 8.0
    achieved_gbs = kbytes / sec / 1e9 if sec > 0 else 0.0
    achieved_gflops = rec["flops"] / sec / 1e9 if sec > 0 else 0.0
    cluster = run.krylov_form()

    # every stage of the step, timed by the library's stage events in a
    # window of direct-launched steps (graphs are off while stages are timed)
    stages = None
    if not args.no_stages:
        run.profile(3)
        sa = 0
        for _ in range(prof_steps):
            sa += run.stats()["n_active"]
            run.step(1)
        nst, sms = run.stages()
        run.profile(False)
        stages = stage_report(sms, nst, p, sa / max(1, nst), peak)

    # late window: the same run advanced further untimed (the vortices have
    # merged further and the grid has grown), then timed as the main region
    late = None
    if args.late_steps > 0:
        run.step(args.late_steps)
        run.sync()
        l_starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        l_ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        l_upd = 0
        torch.cuda.synchronize()
        with torch.cuda.stream(stream):
            for q in range(args.steps):
                flush.zero_()
                l_starts[q].record(stream)
                l_upd += run.stats()["n_active"]
                run.step(1)
                l_ends[q].record(stream)
        torch.cuda.synchronize()
        l_ms = sum(a.elapsed_time(b) for a, b in zip(l_starts, l_ends))
        run.profile(True)
        run.step(prof_steps)
        lrec = run.profile_record()
        run.profile(False)
        lsec = lrec["ms"] * 1e-3
        lgbs = lrec["bytes"] * es / 8.0 / lsec / 1e9 if lsec > 0 else 0.0
        na_late = l_upd / args.steps
        late = {"after_steps": args.warmup + args.steps + 2 * prof_steps + args.late_steps,
                "sim_time": run.diagnostics()["t"], "steps": args.steps, "value": l_upd / (l_ms * 1e-3),
                "unit": UNIT, "ms_per_step": l_ms / args.steps, "mean_active_points": na_late,
                "krylov_working_set_bytes": (p.m + 1) * es * na_late,
                "roofline": {"bound": "hbm", "achieved": lgbs, "peak": peak, "unit": "GB/s", "frac": lgbs / peak,
                             "avg_launch_us": 1e3 * lrec["ms"] / max(1, lrec["launches"])}}

    # end to end through the C-ABI with host buffers (pinned), a fresh run
    e2e = None
    if not args.no_e2e:
        v = wl.vortices
        prm = [torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).pin_memory()
               for a in (v.xc, v.yc, v.gamma, v.s)]
        run2 = B.Run(p, stream=stream.cuda_stream)
        idx_h = torch.empty(p.NJ * p.NJ, dtype=torch.int32).pin_memory()
        om_h = torch.empty(p.NJ * p.NJ, dtype=torch.float64).pin_memory()
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        B.wrc_init_vortices(run2.h, *[a.numpy() for a in prm])
        e2e_upd, d2h = 0, 0
        for _ in range(args.steps):
            na = run2.stats()["n_active"]
            e2e_upd += na
            run2.step(1)
            na2 = run2.stats()["n_active"]
            B.wrc_query_active(run2.h, idx_h, om_h, p.NJ * p.NJ)
            d2h += 12 * na2
        torch.cuda.synchronize()
        e2e_wall = time.perf_counter() - t1
        run2.close()
        e2e = {"value": e2e_upd / e2e_wall, "unit": UNIT,
               "h2d_bytes_per_step": int(32 * v.n / args.steps),
               "d2h_bytes_per_step": int(d2h / args.steps)}

    # the mixed mode's error against FP64: the same workload advanced the same
    # steps from its initial condition in both precisions on the GPU (the
    # FP64 path is held to 1e-10 of the oracle by the parity tests)
    accuracy = None
    if p.prec == W.PREC_MIXED and rank == 0:
        import dataclasses
        res = []
        for prec in (W.PREC_MIXED, W.PREC_FP64):
            with B.Run(dataclasses.replace(p, prec=prec), stream=stream.cuda_stream) as r2:
                r2.init_vortices(wl.vortices)
                r2.step(args.steps)
                r2.sync()
                res.append(r2.active())
        rel, flips = compare_results(res[0][0], res[0][1], res[1][0], res[1][1])
        accuracy = {"steps": args.steps, "rel_l2_vs_fp64": rel, "grid_differences": flips,
                    "grid_diff_frac": flips / max(1, res[1][0].size),
                    "measure": "omega after the same steps from the same initial condition, mixed against FP64 "
                               "(both on the GPU), over the points active in both"}

    serving = None
    if not args.no_serving and rank == 0:
        serving = measure_serving(args)
    ensemble = None
    if not args.no_ensemble and rank == 0:
        ensemble = measure_ensemble(args)
    scalar = None
    if not args.no_scalar and rank == 0:
        scalar = measure_scalar(args, wl)
    exner = None
    if not args.no_exner and rank == 0:
        exner = measure_exner(args)
    variants = None
    if not args.no_variants and rank == 0 and args.workload == "fujiwhara_1024":
        variants = measure_variants(args)

    # max over ranks
    t_dev, upd = combine_ranks(dev_ms, upd, "cuda")
    value = upd / (t_dev * 1e-3)

    line = None
    if rank == 0:
        cpu = None
        if not args.no_cpu_baseline:
            csteps = args.cpu_steps if args.cpu_steps is not None else (1 if p.NJ >= 4096 else 2)
            cval, cwall, cores, cupd = time_oracle(wl, csteps)
            cpu = {"value": cval, "unit": UNIT, "cores": cores, "kind": "oracle",
                   "sample": f"{csteps} oracle step(s) of {wl.name} from t=0 ({cupd} updates, {cwall:.1f} s)"}
        # the whole step against HBM: b (m^2 + 9m + 12) bytes per active-point
        # update (Krylov part and adaptation) plus ~30 b per lattice point
        # (reconstruction, FFT solve, velocity, SGS) per step, b the bulk bytes
        na_step = upd / max(1, args.steps * ws)
        step_bytes = es * ((p.m * p.m + 9 * p.m + 12) * na_step + 30.0 * p.NJ * p.NJ)
        step_gbs = step_bytes / (t_dev / args.steps * 1e-3) / 1e9
        step_hbm = {"achieved": step_gbs, "peak": peak, "unit": "GB/s", "frac": step_gbs / peak,
                    "bytes_per_step": step_bytes,
                    "bytes_model": f"{int(es)} (m^2 + 9m + 12) bytes per active point + {int(30 * es)} bytes per "
                                   "lattice point, per step",
                    "peak_source": f"{peak_src} HBM copy bandwidth (MEASURED_PEAKS.json hbm_gbs)",
                    "target_frac": 0.6}
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_dev / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64" if p.prec == W.PREC_MIXED else "f64",
            "data": "synthetic",
            "config": {"workload": wl.name, "NJ": p.NJ, "n0": p.n0, "J": p.J, "eps": p.eps, "m": p.m,
                       "sgs": p.sgs_name(), "cs": p.cs, "re": p.re, "dt": p.dt,
                       "mean_active_points": upd / max(1, args.steps * ws),
                       "l2": "flushed between timed steps (256 MiB write outside the step events)",
                       "wall_s": wall},
            "roofline": {"bound": "hbm", "kernel": "k_krylov_step (Arnoldi, phi_1 and the update: the Krylov "
                                                    "part of a step)",
                         "achieved": achieved_gbs, "peak": peak, "unit": "GB/s", "frac": achieved_gbs / peak,
                         "peak_source": f"{peak_src} HBM copy bandwidth (MEASURED_PEAKS.json hbm_gbs)",
                         "traffic": krylov_traffic() if args.workload == "fujiwhara_1024" else None,
                         "bytes_per_launch": kbytes / max(1, rec["launches"]),
                         "bytes_model": f"{int(es)} (m^2 + 9m + 6) bytes per active point (operator applications, "
                                        "fused Gram-Schmidt passes, combination)",
                         "launches": rec["launches"], "avg_launch_us": 1e3 * rec["ms"] / max(1, rec["launches"]),
                         "cluster_size": cluster, "target_frac": 0.6,
                         "fp64": {"achieved": achieved_gflops, "peak": FP64_PEAK_GFLOPS, "unit": "GFLOP/s",
                                  "frac": achieved_gflops / FP64_PEAK_GFLOPS,
                                  "peak_source": "nominal FP64 rate of GB300 (1.25 TFLOP/s; no measured FP64 peak)",
                                  "flops_per_launch": rec["flops"] / max(1, rec["launches"])}},
            "step_hbm": step_hbm,
            "late": late,
            "accuracy": accuracy,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": launches,
            "clocks": sampler.summary(),
            "serving": serving,
            "ensemble": ensemble,
            "scalar": scalar,
            "exner": exner,
            "variants": variants,
            "stages": stages,
        }
        print(json.dumps(line), flush=True)
    run.close()
    if ws > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=60)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--cpu-steps", type=int, default=None,
                    help="oracle steps of the cpu_baseline sample (default 2, 1 at 4096^2)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="fujiwhara_1024")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-ensemble", action="store_true")
    ap.add_argument("--no-scalar", action="store_true")
    ap.add_argument("--no-exner", action="store_true")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--no-stages", action="store_true")
    ap.add_argument("--ens-members", type=int, default=256)
    ap.add_argument("--ens-steps", type=int, default=50)
    ap.add_argument("--late-steps", type=int, default=1000)
    ap.add_argument("--ens-solo-sample", type=int, default=32)
    ap.add_argument("--serve-requests", type=int, default=48)
    ap.add_argument("--serve-step-scale", type=float, default=0.1)
    ap.add_argument("--serve-full", action="store_true",
                    help="the whole serving trace (400 requests) at full step counts (takes many minutes)")
    args = ap.parse_args()
    if args.serve_full:
        args.serve_requests, args.serve_step_scale = 400, 1.0
    if args.warmup < 3 and args.impl == "ours":
        log("warm-up raised to 3 steps")
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
