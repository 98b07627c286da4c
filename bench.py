#!/usr/bin/env python3
"""Throughput of the multi-moment vortex method right-hand side on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Workload: two co-rotating Gaussian patches, N = 65536 particles (2 x 32768,
patch radius 2, centres (+-3, 0), circulations ~ exp(-r^2) normalised to 1
per patch), order M = 6 (28 moments), core sigma = lambda_0 = 0.1, Re = 2000,
RK4 with dt = 0.05; mixed precision (FP32 pair jets and contractions, FP64
state, tables and per-particle finish).  One step = one RK4 step = four
right-hand sides = 4 N^2 ordered pair interactions (the self pair included:
the finish kernel evaluates it from the jet at the origin).

value      pair-interactions/s of the device-timed steps (state resident in HBM,
           L2 flushed by a 256 MiB write before every timed step, outside the
           timed region).
e2e        the same metric through the C ABI with host buffers: set_state from
           pinned host memory, one step, get_state to pinned host memory.
roofline   the all-pairs kernels of one right-hand side (~95% of the step;
           the autotuner's choice: the direct form, or the list form's list
           build, tree, far-field and near-pair kernels) against the FP32 FMA
           peak measured in the same run (mmvm_alu_peak: a full-occupancy
           grid of independent FMA chains; nominal 152 SMs x 128 lanes x 2
           flop x 2.07 GHz = 80.5 TFLOP/s); the flops of one launch are the
           work it did on each path (counted by the kernels: near pairs, far
           pairs source by source, expansions evaluated) times that path's
           flops (flops_per_pair, far_flops_per_pair, m2p_flops).
near_pairs_per_s, pairs_by_path_per_rhs  how the N^2 pairs of a right-hand
           side were evaluated: through the full jet (near), the point-vortex
           jet source by source, or inside expansions of far groups / tree
           nodes (at FP32 rounding: the far field is the Gaussian-free tail).
fp64       the plain FP64 form of the same right-hand side on the first 16384
           particles of the workload (one right-hand side, device-timed),
           beside mixed precision without and with the far field.
mixed_vs_fp64_100_steps  the same comparison over 100 RK4 steps of the
           recipe at N = 4096 (--prec-n): rates of the three forms, the gain
           of the precision split and of the far field apart, and the
           per-particle error of both mixed forms against FP64.
single_m10 one particle at order 10 (66 moments), 500 FP64 RK4 steps: RHS/s,
           coefficient terms/s and the error against the oracle's trajectory.
random_disk_n4096  N = 4096, M = 4 random disk, up to 200 mixed RK4 steps:
           throughput over the finite steps and the error against FP64.
served     the served stream (independent random-disk solves: n log-uniform in
           [64, 8192], M in {2, 4, 8}, Re uniform in [100, 5000], 50-500 RK4
           steps of 0.01) through the continuous-batching server: a burst
           (every request at t = 0) gives the saturation throughput, then
           Poisson arrivals at 0.7x and at 1.2x the saturation request rate
           give p50/p99 latency below and above saturation (submit -> result
           on the host; a request whose state leaves
           the finite range stops there with MMVM_E_NUMERIC and is counted
           apart); the smallest requests are
           re-run in the plain FP64 form (context API) for their error, and
           a few in FP64 through the server for the mixed/FP64 ratio.
single_m60 one particle at order 60 (1891 moments), Lamb-Oseen core plus a
           quadrupole, eps in {1e-3, 1e-2, 0.1} x Re in {1e3, 1e4}: six
           instances, 2000 RK4 steps of 0.01 each, FP64 separable self term
           (six contexts on their own streams); RHS evaluations/s, the
           multiply-adds of the separable passes against the measured FP64
           peak, sampled rows against the oracle at t = 0, and the step at
           which the trajectory leaves the bounded range against the size of
           a perturbation of the initial state and against the time step
           (order 48 as the control).
cpu_baseline the FP64 numpy oracle on sampled target rows against all sources,
           one host core; cpu_baseline_all_cores and --impl reference: one
           single-threaded oracle process per host core, each on its own rows.
N > 1 GPUs (torchrun): independent replicas of the workload, one per GPU.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")
os.environ.setdefault("OMP_NUM_THREADS", "1")
os.environ.setdefault("MKL_NUM_THREADS", "1")

import numpy as np  # noqa: E402

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import mmvm_inputs  # noqa: E402

METRIC = "moment-ODE pair-interactions/s"
UNIT = "pair-interactions/s"
SM_COUNT = 152
FP32_LANES = 128
SM_MAX_GHZ = 2.07
FP32_PEAK_TFLOPS = SM_COUNT * FP32_LANES * 2 * SM_MAX_GHZ / 1e3
FP64_SUBSET = 16384


def workload(n: int = 65536):
    return mmvm_inputs.two_patches(n=n, order=6, sigma=0.1, Re=2000.0, dt=0.05, steps=100)


def config_dict(wl, extra=None):
    d = {"workload": f"two co-rotating Gaussian patches, N={wl.n}, M=6, sigma=0.1, Re=2000, "
                     "RK4 dt=0.05 (all-pairs)",
         "n": wl.n, "order": wl.order, "moments_per_particle": wl.K, "lambda0": wl.lam0,
         "Re": 1.0 / wl.nu, "dt": wl.dt,
         "precision": "mixed: FP32 pair jet/contraction, FP64 state/tables/finish/RK4",
         "far_field": "on: pairs whose Gaussian tail is below FP32 rounding take the point-vortex "
                      "jet, source by source or inside expansions of far groups / tree nodes "
                      "(pairs_by_path_per_rhs; near_pairs_per_s counts the full-jet pairs)",
         "pairs_per_step": 4 * wl.n * wl.n,
         "l2": "flushed (256 MiB write) before every timed step, outside the timed region"}
    if extra:
        d.update(extra)
    return d


def flops_per_pair(M: int) -> int:
    """Floating-point operations of one near-field pair in the all-pairs kernel.

    K = (M+1)(M+2)/2 source moments, BMAX = 2M correlation orders,
    NJ = M + BMAX jet orders:
      edge columns      beta1 in {0, 1}: 2 BMAX K multiply-adds     = 4 BMAX K
      Laplacian columns (BMAX-1) K + tri(BMAX-1) (M+1) multiply-adds, x 2
      jet order n       Laplacian chain and projection 4 (n-1),
                        entries alpha1 <= M+1: 2 min(n+1, M+2), seeds 8
      edge terms        I_n, zbar^n, scaling (per order)            ~ 16
      Hermite fns       two three-term recurrences                  ~ 6 (NJ - 1)
      setup             separation, |b|^2, masks                    ~ 30 (plus 2 exp)
    """
    K = (M + 1) * (M + 2) // 2
    bmax = 2 * M if M > 0 else 1
    nj = M + bmax
    edge = 4 * bmax * K
    lap = 2 * ((bmax - 1) * K + (bmax - 1) * bmax // 2 * (M + 1)) if bmax >= 2 else 0
    jet = sum(4 * (n - 1) + 2 * min(n + 1, M + 2) + 8 for n in range(1, nj + 1))
    return edge + lap + jet + 16 * nj + 6 * (nj - 1) + 30


def flops_per_pair_parts(M: int):
    """flops_per_pair split by the list form's kernels: (edge part: the jet,
    its edge contraction and the set-up; Laplacian part: the Hermite
    functions and the separable sums); the two add up to flops_per_pair."""
    K = (M + 1) * (M + 2) // 2
    bmax = 2 * M if M > 0 else 1
    nj = M + bmax
    edge = 4 * bmax * K
    lap = 2 * ((bmax - 1) * K + (bmax - 1) * bmax // 2 * (M + 1)) if bmax >= 2 else 0
    jet = sum(4 * (n - 1) + 2 * min(n + 1, M + 2) + 8 for n in range(1, nj + 1))
    return edge + jet + 16 * nj + 30, lap + 6 * (nj - 1)


def far_flops_per_pair(M: int) -> int:
    """Floating-point operations of one far-field (point-vortex multipole) pair.

    u = 1/(b_hi + b_lo) to first order in b_lo                  ~ 30
    rho_q = (q-1)! u^q, q = 2 .. 3M (complex product + scale)   8 (3M - 1)
    Y[nb] += A'_n rho_{n+nb}, 0 <= n <= M, 1 <= nb <= 2M        8 (M+1) 2M
    (the fold of Y into Psi is once per target and tile, not per pair)
    """
    if M == 0:
        return 30 + 8 * 2
    return 30 + 8 * (3 * M - 1) + 8 * (M + 1) * 2 * M


M2P_ORDER = [8, 10, 12, 14, 15, 17, 18, 19, 21]  # m2p_order(M) of the CUDA code


def m2p_flops(M: int) -> int:
    """Floating-point operations of one tile-expansion evaluation (one target
    against one far source tile summed about the tile centre):
    u = 1/w (~30), rho_q up to order 2M + NA - 1 (8 each), Y[nb] += B_j
    rho_{j+nb} for 1 <= nb <= 2M, j < NA (8 each), fold into the two edge
    columns per order and the (hi, lo) flush (~8 per output), NA = M + P + 1
    terms."""
    na = M + M2P_ORDER[M] + 1
    nb = 2 * (2 * M if M > 0 else 1)
    return 30 + 8 * (2 * M + na - 2) + 8 * 2 * max(M, 1) * na + 8 * nb


# ---------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (FileNotFoundError, OSError):
            self.proc = None
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [ln for ln in out.splitlines() if ln.strip()]

    def summary(self):
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in getattr(self, "lines", []):
            p = [v.strip() for v in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax.append(float(p[2]))
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- oracle
def oracle_rate(wl, rows: int, seed: int = 0):
    """Time the FP64 oracle on `rows` target rows against all sources."""
    from oracle.rhs import rhs_regrouped

    sel = np.random.default_rng(seed).choice(wl.n, rows, replace=False)
    t0 = time.perf_counter()
    ox, oM = rhs_regrouped(wl.x, wl.moments, 0.0, wl.order, wl.lam0, wl.nu, rows=sel)
    dt = time.perf_counter() - t0
    return rows * wl.n / dt, dt, sel, ox, oM


def _oracle_rows_child(args):
    """One process of the all-cores oracle timing: its own sample of rows."""
    n, rows, seed, keep = args
    os.environ["OPENBLAS_NUM_THREADS"] = "1"
    from oracle.rhs import rhs_regrouped

    wl = workload(n)
    rng = np.random.default_rng(seed)
    # untimed: the oracle's first call builds its coefficient caches
    rhs_regrouped(wl.x, wl.moments, 0.0, wl.order, wl.lam0, wl.nu, rows=rng.choice(wl.n, 1))
    sel = rng.choice(wl.n, rows, replace=False)
    t0 = time.perf_counter()
    ox, oM = rhs_regrouped(wl.x, wl.moments, 0.0, wl.order, wl.lam0, wl.nu, rows=sel)
    secs = time.perf_counter() - t0
    return (secs, sel, ox, oM) if keep else secs


def oracle_rate_all_cores(wl, rows_per_proc: int, procs: int, seed: int = 0, keep=False):
    """The oracle as it stands, one single-threaded process per host core, each
    on its own sampled target rows against all sources (rows are
    independent): pair-interactions/s = all rows x n / the slowest process's
    compute time.  A spawn pool, so no process inherits a CUDA context.
    keep: also return the rows and the oracle's values on them."""
    import multiprocessing as mp

    ctx = mp.get_context("spawn")
    with ctx.Pool(procs) as pool:
        res = pool.map(_oracle_rows_child,
                       [(wl.n, rows_per_proc, seed + 7919 * i, keep) for i in range(procs)])
    secs = [r[0] for r in res] if keep else res
    value = procs * rows_per_proc * wl.n / max(secs)
    if not keep:
        return value, max(secs)
    return (value, max(secs), np.concatenate([r[1] for r in res]),
            np.concatenate([r[2] for r in res]), np.concatenate([r[3] for r in res]))


def error_vs_oracle(wl, gx, gM, rows, ox, oM, procs):
    """Per-particle error of the right-hand side at t = 0 against the oracle:
    the random rows already evaluated, plus rows aimed at the all-pairs
    kernel's path switches (evaluated here, untimed)."""
    from tests.parity_util import (oracle_rows_parallel, rhs_error_rows, switch_rows,
                                   vel_error_rows)

    kinds = switch_rows(wl.x, wl.moments, wl.order, wl.lam0)
    srows = np.array(sorted({j for v in kinds.values() for j in v}))
    sx, sM = oracle_rows_parallel(wl.x, wl.moments, 0.0, wl.order, wl.lam0, wl.nu, srows, procs)
    out = {"t": 0.0, "norm": "per particle: weighted moment norm (convergence theorem) and "
                             "Euclidean velocity norm, relative to the particle's own value "
                             "floored at 1e-3 of the largest row; max over the rows",
           "rows_random": int(len(rows)), "rows_at_path_switches": int(len(srows)),
           "xdot_rel": max(vel_error_rows(gx[rows], ox), vel_error_rows(gx[srows], sx)),
           "dM_rel_weighted": max(rhs_error_rows(gM[rows], oM, wl.order, wl.lam0),
                                  rhs_error_rows(gM[srows], sM, wl.order, wl.lam0))}
    pos = {j: i for i, j in enumerate(srows)}
    out["by_kind"] = {k: {"rows": len(v),
                          "xdot_rel": vel_error_rows(gx[v], sx[[pos[j] for j in v]]),
                          "dM_rel_weighted": rhs_error_rows(gM[v], sM[[pos[j] for j in v]],
                                                            wl.order, wl.lam0)}
                      for k, v in kinds.items()}
    return out


def cpu_cores_used() -> int:
    v = os.environ.get("OPENBLAS_NUM_THREADS") or os.environ.get("OMP_NUM_THREADS") or "1"
    try:
        return int(v)
    except ValueError:
        return 1


def run_reference(args, wl):
    rows = args.ref_rows
    procs = args.oracle_procs or os.cpu_count() or 1
    vals, secs = [], []
    for s in range(args.steps):
        v, dt = oracle_rate_all_cores(wl, rows, procs, seed=s)[:2]
        vals.append(v)
        secs.append(dt)
    value = len(vals) * procs * rows * wl.n / sum(secs)
    sample = (f"{procs} processes x {rows} random target rows x all {wl.n} sources per "
              f"step, one right-hand side at t=0 (FP64 numpy oracle, one thread per process)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * sum(secs) / len(secs), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_dict(wl, {"oracle_rows_per_step": rows}),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": procs,
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- ours
def _served_requests(count):
    return mmvm_inputs.served_stream(count=count, rate=1.0)


def _wait_all(srv, tickets):
    out = {}
    pending = set(tickets)
    while pending:
        for t in list(pending):
            r = srv.poll(t)
            if r is not None:
                out[t] = r
                pending.discard(t)
        time.sleep(0.0005)
    return out


def _ok(r):
    return r is not None and not isinstance(r[0], str)


def _run_stream(mm, reqs, precision, arrivals=None):
    """Submit reqs (at their arrival times, seconds from start, or all at once)
    and collect (result or error, latency_ms) per request; returns results and
    the makespan in seconds."""
    results = [None] * len(reqs)
    with mm.Server(precision=precision) as srv:
        t0 = time.perf_counter()
        tickets = {}
        order = sorted(range(len(reqs)), key=lambda i: arrivals[i] if arrivals else 0.0)
        nxt = 0
        while nxt < len(order) or tickets:
            now = time.perf_counter() - t0
            while nxt < len(order) and (arrivals is None or arrivals[order[nxt]] <= now):
                i = order[nxt]
                w = reqs[i].workload
                tickets[srv.submit(w.x, w.moments, w.order, w.lam0, w.nu, w.dt, w.steps)] = i
                nxt += 1
            for t in list(tickets):
                try:
                    r = srv.poll(t)
                except mm.MMVMError as e:
                    results[tickets.pop(t)] = ("error", str(e), getattr(e, "info", {}))
                    continue
                if r is not None:
                    results[tickets.pop(t)] = r
            time.sleep(0.0005)
        makespan = time.perf_counter() - t0
        stats = srv.stats()
    return results, makespan, stats


def _lat_stats(lat):
    lat = np.asarray(lat, dtype=float)
    if not len(lat):
        return {"count": 0, "p50_ms": None, "p99_ms": None, "mean_ms": None}
    return {"count": int(len(lat)), "p50_ms": float(np.percentile(lat, 50)),
            "p99_ms": float(np.percentile(lat, 99)), "mean_ms": float(lat.mean())}


def run_served(args, mm):
    """Served-stream measurement (see the module docstring).

    * saturation: the first --serve-burst requests submitted at t = 0 (the
      request rate and pair-interactions/s the server sustains);
    * Poisson arrivals of the whole stream at 0.7x and 1.2x that request
      rate: latency (submit -> result on the host) percentiles over the
      requests that completed, apart over the diverged ones (stopped with
      MMVM_E_NUMERIC at the step where their state left the finite range),
      and over all;
    * batching gain: the burst's requests one at a time through contexts
      (same precision, same steps as served) against the burst's makespan.
    """
    reqs = _served_requests(args.serve_requests)
    work = [4 * r.workload.n ** 2 * r.workload.steps for r in reqs]
    mixed = mm.MMVM_MIXED_FP32
    nb = min(args.serve_burst, len(reqs))
    # warm-up (untimed): the server's and the contexts' per-order variant
    # choices are made once per process
    warm = []
    for order in sorted({r.workload.order for r in reqs}):
        w = mmvm_inputs.random_disk(n=256, order=order, steps=2, seed=7 + order)
        warm.append(mmvm_inputs.Request(len(warm), 0.0, w))
    _run_stream(mm, warm, mixed)
    seen = set()
    for r in reqs[:nb]:
        w = r.workload
        key = (w.order, int(math.log2(w.n)))
        if key not in seen:
            seen.add(key)
            with mm.Context(w.order, w.lam0, w.nu, mixed) as c:
                c.set_state(w.x, w.moments, 0.0)
    burst, span_b, st_b = _run_stream(mm, reqs[:nb], mixed)
    ok_b = [i for i, r in enumerate(burst) if _ok(r)]

    def done_work(res, rr):  # pair interactions computed (a diverged request stops early)
        tot = 0
        for i, r in enumerate(res):
            if r is not None:
                steps = r[2].get("steps", 0) if isinstance(r[2], dict) else 0
                tot += 4 * rr[i].workload.n ** 2 * steps
        return tot

    sat_rate = nb / span_b

    def poisson(factor):
        """The stream's own exponential gaps rescaled to factor x the
        saturation request rate."""
        rate = factor * sat_rate
        arrivals = [r.arrival / rate for r in reqs]
        res, span, st = _run_stream(mm, reqs, mixed, arrivals)
        ok = [i for i, r in enumerate(res) if _ok(r)]
        div = [i for i, r in enumerate(res) if r is not None and not _ok(r)
               and "NUMERIC" in r[1]]
        lat_ok = [res[i][2]["latency_ms"] for i in ok]
        lat_div = [res[i][2].get("latency_ms", np.nan) for i in div]
        out = {"rate_per_s": rate, "of_saturation": factor, "makespan_s": span,
               "value": done_work(res, reqs) / span, "unit": UNIT,
               "completed": _lat_stats(lat_ok), "diverged": _lat_stats(lat_div),
               "all_finished": _lat_stats(lat_ok + lat_div),
               "queue_p50_ms": float(np.percentile([res[i][2]["queue_ms"] for i in ok], 50))
               if ok else None,
               "max_batch": st["max_batch"], "errors_other": len(reqs) - len(ok) - len(div)}
        # flat keys of the completed requests (the served-solve latency)
        out["p50_ms"] = out["completed"]["p50_ms"]
        out["p99_ms"] = out["completed"]["p99_ms"]
        return out

    pois_under = poisson(0.7)
    pois_over = poisson(1.2)
    # batching gain: the burst's requests one at a time through contexts, each
    # for the steps the server ran for it
    t0 = time.perf_counter()
    solo_work = 0
    for i, r in enumerate(burst):
        w = reqs[i].workload
        steps = r[2].get("steps", 0) if r is not None and isinstance(r[2], dict) else 0
        if steps <= 0:
            continue
        with mm.Context(w.order, w.lam0, w.nu, mixed) as c:
            c.set_state(w.x, w.moments, 0.0)
            c.step(w.dt, steps)
            c.get_state()
        solo_work += 4 * w.n ** 2 * steps
    solo_s = time.perf_counter() - t0
    # errors of the served mixed results against the plain FP64 form (context API)
    from tests.parity_util import state_error

    small = sorted(ok_b, key=lambda i: work[i])[:args.serve_check]
    errs = []
    for i in small:
        w = reqs[i].workload
        with mm.Context(w.order, w.lam0, w.nu, mm.MMVM_FP64,
                        flags=mm.MMVM_FLAG_NO_FAR_FIELD) as c64:
            c64.set_state(w.x, w.moments, 0.0)
            c64.step(w.dt, w.steps)
            x64, m64, t64 = c64.get_state()
        lam_t = math.sqrt(w.lam0 ** 2 + 4 * w.nu * t64)
        x, m, _ = burst[i]
        errs.append({"n": w.n, "order": w.order, "steps": w.steps,
                     "x_rel_lambda": float(np.abs(x - x64).max() / lam_t),
                     "M_rel_weighted": state_error(m, m64, w.order, lam_t)})
    # the same few requests in FP64 through the server, against mixed
    sub = sorted(ok_b, key=lambda i: work[i])[:args.serve_fp64]
    r64, span64, _ = _run_stream(mm, [reqs[i] for i in sub], mm.MMVM_FP64)
    r32, span32, _ = _run_stream(mm, [reqs[i] for i in sub], mixed)
    sub_work = sum(work[i] for i in sub)
    return {
        "workload": f"{len(reqs)} random-disk solves: n log-uniform [64, 8192], M in {{2,4,8}}, "
                    "Re U[100,5000], 50-500 RK4 steps of 0.01 (moments 1% per moment in the "
                    "weighted norm), mixed precision with the far field",
        "requests": len(reqs),
        "pair_interactions": float(sum(work)),
        "saturation": {"requests": nb, "makespan_s": span_b,
                       "value": done_work(burst, reqs[:nb]) / span_b,
                       "unit": UNIT, "requests_per_s": sat_rate,
                       "completed": len(ok_b), "max_batch": st_b["max_batch"],
                       "ticks": st_b["ticks"]},
        "poisson": pois_under,
        "poisson_over_saturation": pois_over,
        "batching_gain": {"requests": nb, "served_makespan_s": span_b,
                          "one_at_a_time_s": solo_s,
                          "one_at_a_time_value": solo_work / solo_s if solo_s else None,
                          "gain": solo_s / span_b,
                          "note": "the saturation burst's requests run one after another "
                                  "through mixed-precision contexts (set_state, the steps the "
                                  "server ran, get_state) against the served makespan"},
        "note": "requests whose state leaves the finite range (the truncated moment ODE of "
                "dense mixed-sign random disks at M >= 4) stop at that step with "
                "MMVM_E_NUMERIC; p50_ms/p99_ms are over the requests that completed, the "
                "diverged ones and all finished requests are listed apart",
        "error_vs_fp64": errs,
        "fp64_same_requests": {"requests": len(sub), "pair_interactions": float(sub_work),
                               "fp64_value": sub_work / span64, "mixed_value": sub_work / span32,
                               "mixed_over_fp64": span64 / span32},
    }


def run_scaling(args, mm, stream, device):
    """One right-hand side of the two-patch recipe at growing N, in the list
    form with the tree far field: (a) the core shrinking as
    sigma = 0.1 sqrt(65536 / N) (every particle keeps about the same number
    of sources within the near-field radius, so the near work grows like N
    and the far field decides the rest), (b) the benchmark's fixed
    sigma = 0.1 (the near field is a fixed fraction of the N^2 pairs).
    Device time of the all-pairs launches and of the whole right-hand side,
    and the pairs by path."""
    import torch

    sizes = [int(v) for v in args.scaling.split(",") if v.strip()]
    out = []
    nv = mm.pair_variant_counts(6)[0]
    saved = {k: os.environ.get(k) for k in ("MMVM_PAIR_VARIANT", "MMVM_FAR_TREE")}
    os.environ["MMVM_PAIR_VARIANT"] = str(nv + 4)  # the list form's split, barrier-free variant
    os.environ["MMVM_FAR_TREE"] = "1"
    try:
        for kind in ("sigma_scaled", "sigma_fixed"):
            for n in sizes:
                if kind == "sigma_fixed" and n > args.scaling_fixed_max:
                    continue
                sigma = 0.1 * math.sqrt(65536.0 / n) if kind == "sigma_scaled" else 0.1
                wl = mmvm_inputs.two_patches(n=n, order=6, sigma=sigma, Re=2000.0, dt=0.05)
                with mm.Context(6, wl.lam0, wl.nu, mm.MMVM_MIXED_FP32, device=device) as c:
                    mm.mmvm_set_stream(c.handle, stream.cuda_stream)
                    c.set_state(wl.x, wl.moments, 0.0)
                    mm.mmvm_enable_timing(c.handle, True)
                    d_dx = torch.empty((n, 2), dtype=torch.float64, device=stream.device)
                    d_dm = torch.empty((n, wl.K), dtype=torch.float64, device=stream.device)
                    mm.mmvm_rhs_device(c.handle, d_dx.data_ptr(), d_dm.data_ptr())  # warm-up
                    torch.cuda.synchronize(stream.device)
                    mm.mmvm_pair_time(c.handle)
                    w0 = mm.mmvm_pair_work(c.handle)
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    mm.mmvm_rhs_device(c.handle, d_dx.data_ptr(), d_dm.data_ptr())
                    e1.record(stream)
                    e1.synchronize()
                    rhs_ms = e0.elapsed_time(e1)
                    pair_ms, _ = mm.mmvm_pair_time(c.handle)
                    w1 = mm.mmvm_pair_work(c.handle)
                    ok = bool(torch.isfinite(d_dm).all().item())
                work = [int(b - a) for a, b in zip(w0, w1)]
                out.append({"n": n, "sigma": sigma, "kind": kind, "rhs_ms": rhs_ms,
                            "pair_ms": pair_ms, "value": n * n / (rhs_ms / 1e3), "unit": UNIT,
                            "near_pairs": work[0], "far_pairs_source_by_source": work[1],
                            "expansions": work[2], "pairs_in_expansions": work[3],
                            "finite": ok})
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    return {"workload": "two co-rotating patches, M=6, one right-hand side per N (list form, "
                        "tree far field)", "runs": out}


def coefficient_terms(M: int) -> int:
    """(k, l, i, q) terms of the single-particle coefficient sums of
    eq:FinalSingleI/II per right-hand side at order M (every k, l with
    |k|, |l| <= M): what the literal form evaluates, 9.45e8 at M = 60."""
    ks = np.array([(n - k2, k2) for n in range(M + 1) for k2 in range(n + 1)])
    k1, k2 = ks[:, 0][:, None], ks[:, 1][:, None]
    l1, l2 = ks[:, 0][None, :], ks[:, 1][None, :]
    n1 = np.where(k1 >= 1, (np.minimum(l1, k1 - 1) + 1) * (np.minimum(l2, k2) + 1), 0)
    n2 = np.where(k2 >= 1, (np.minimum(l1, k1) + 1) * (np.minimum(l2, k2 - 1) + 1), 0)
    return int(n1.sum() + n2.sum())


def separable_fmas(M: int) -> int:
    """Multiply-adds of one separable single-particle RHS at order M (the
    loop bounds of the CUDA passes: Psi, pass 1 (q), pass 2 (l2), pass 3 (i))."""
    tot = 0
    for bn in range(1, 2 * M + 1):  # Psi[beta]: m of the parity of beta
        for b2 in range(bn + 1):
            b1 = bn - b2
            tot += sum(1 for m1 in range(b1 & 1, M + 1, 2) for m2 in range(b2 & 1, M - m1 + 1, 2))
    for k2 in range(M + 1):
        for l2 in range(M + 1):
            for b1 in range(2 * M + 1):
                tot += sum(1 for q in range(min(l2, k2) + 1) if b1 + k2 + l2 - 2 * q + 1 <= 2 * M)
                if k2 >= 1:
                    tot += sum(1 for q in range(min(l2, k2 - 1) + 1)
                               if 1 <= b1 + k2 + l2 - 2 * q - 1 <= 2 * M)
    tot += 2 * (M + 1) * (2 * M + 1) * sum(M - l1 + 1 for l1 in range(M + 1))
    for kn in range(M + 1):
        for k2 in range(kn + 1):
            k1 = kn - k2
            for l1 in range(M + 1):
                if k1 >= 1:
                    tot += min(l1, k1 - 1) + 1
                if k2 >= 1:
                    tot += min(l1, k1) + 1
    return tot


def divergence_sweep(mm, M=60, eps=0.1, Re=1e3, dt=0.01, max_steps=400, chunk=5,
                     deltas=(0.0, 1e-14, 1e-11, 1e-8, 1e-5)):
    """Where does the order-60 FP64 trajectory leave the bounded range, and
    how does that step move with the size of a perturbation of the initial
    state?  Every moment of order >= 2 of the quadrupole state gets delta
    times a fixed random draw in the weighted norm of the convergence
    theorem (relative to the circulation); delta = 0 is the unperturbed FP64
    run, whose only perturbation is rounding (~1e-16).  The divergence step
    is the first checkpoint (every `chunk` steps) where the weighted norm of
    the state exceeds 1e3 times its initial value or is not finite.  A step
    that moves by a fixed amount per decade of delta says the blow-up is an
    instability seeded at the perturbation's size: a wider floating-point
    format (a smaller delta) moves it by that many steps per decade of
    precision, no more."""
    from tests.parity_util import weights

    base = mmvm_inputs.single_quadrupole(order=M, eps=eps, sigma0=1.0, Re=Re, dt=dt)
    w = weights(M, 1.0)
    xi = np.random.default_rng(5).standard_normal(base.K)
    xi[:3] = 0.0  # circulation and first moments unchanged
    out = []
    for d in deltas:
        m0 = base.moments.copy()
        m0[0] += d * xi / np.sqrt(w)
        n0 = float(np.sqrt((m0[0] ** 2 * w).sum()))
        step, growth = None, []
        with mm.Context(M, base.lam0, base.nu, mm.MMVM_FP64) as c:
            c.set_state(base.x, m0, 0.0)
            done = 0
            while done < max_steps:
                c.step(dt, chunk)
                done += chunk
                _, m, _ = c.get_state()
                nrm = float(np.sqrt((m[0] ** 2 * w).sum())) if np.isfinite(m).all() else np.inf
                if d == 0.0:
                    growth.append(round(math.log10(max(nrm / n0, 1e-300)), 3)
                                  if np.isfinite(nrm) else None)
                if not np.isfinite(nrm) or nrm > 1e3 * n0:
                    step = done
                    break
        rec = {"delta": d, "divergence_step": step}
        if d == 0.0:
            rec["log10_norm_growth_every_%d_steps" % chunk] = growth
        out.append(rec)
    steps = [(r["delta"], r["divergence_step"]) for r in out if r["delta"] > 0
             and r["divergence_step"] is not None]
    slope = None
    if len(steps) >= 2:
        x = np.log10([d for d, _ in steps])
        y = np.array([st for _, st in steps], dtype=float)
        slope = float(np.polyfit(x, y, 1)[0])
    return {"workload": f"order {M}, Lamb-Oseen core + quadrupole eps={eps}, Re={Re:g}, RK4 "
                        f"dt={dt}, FP64 separable self term",
            "runs": out, "steps_per_decade_of_delta": slope,
            "criterion": "weighted norm above 1e3 x its initial value, or not finite, at a "
                         f"checkpoint every {chunk} steps"}


def divergence_vs_dt(mm, M=60, Re=1e3, t_end=5.0, eps_list=(0.1, 1e-2),
                     dts=(0.01, 0.005, 0.0025, 0.00125), check_t=0.05):
    """Does the order-60 FP64 trajectory leave the bounded range because of
    RK4's stability limit (a stiff mode that a smaller step would resolve)
    or because the truncated system itself has a growing mode?  The same
    state is run with the step halved three times; the divergence time (the
    first check, every check_t time units, where the weighted norm exceeds
    1e3 times its initial value or is not finite) is listed per step.  A
    time that does not move with the step rules out the integrator.  Order 48
    from the same states is the control."""
    from tests.parity_util import weights

    out = []
    for order in (M, 48):
        w = weights(order, 1.0)
        for eps in eps_list:
            rec = {"order": order, "eps": eps, "divergence_time": {}}
            for dt in dts:
                base = mmvm_inputs.single_quadrupole(order=order, eps=eps, sigma0=1.0, Re=Re,
                                                     dt=dt)
                n0 = float(np.sqrt((base.moments[0] ** 2 * w).sum()))
                chunk = max(1, int(round(check_t / dt)))
                t_div, done = None, 0
                with mm.Context(order, base.lam0, base.nu, mm.MMVM_FP64) as c:
                    c.set_state(base.x, base.moments, 0.0)
                    while done * dt < t_end - 1e-9:
                        c.step(dt, chunk)
                        done += chunk
                        _, m, _ = c.get_state()
                        nrm = float(np.sqrt((m[0] ** 2 * w).sum())) \
                            if np.isfinite(m).all() else np.inf
                        if not np.isfinite(nrm) or nrm > 1e3 * n0:
                            t_div = round(done * dt, 6)
                            break
                rec["divergence_time"][str(dt)] = t_div
            out.append(rec)
    return {"workload": f"Lamb-Oseen core + quadrupole, Re={Re:g}, FP64 separable self term, "
                        f"RK4 to t={t_end} with dt in {list(dts)}",
            "runs": out,
            "criterion": "weighted norm above 1e3 x its initial value, or not finite, at a "
                         f"check every {check_t} time units; null: bounded to t_end"}


def run_single_high(args, mm):
    """Single particle at order 60 (see the module docstring)."""
    from oracle.rhs import lam_at, self_rhs_rows

    M, dt, steps = 60, 0.01, args.high_steps
    ctxs = []
    for eps in (1e-3, 1e-2, 0.1):
        for Re in (1e3, 1e4):
            w = mmvm_inputs.single_quadrupole(order=M, eps=eps, sigma0=1.0, Re=Re, dt=dt)
            c = mm.Context(M, w.lam0, w.nu, mm.MMVM_FP64)
            c.set_state(w.x, w.moments, 0.0)
            ctxs.append((c, w))
    w0 = ctxs[-1][1]
    gx, gM = ctxs[-1][0].rhs()
    for c, _ in ctxs:  # graph capture and warm-up
        c.step(dt, 2)
    for c, _ in ctxs:
        c.synchronize()
    # in chunks of 100 steps, noting when each trajectory leaves the finite range
    finite_until = [None] * len(ctxs)
    t0 = time.perf_counter()
    done = 0
    while done < steps:
        k = min(100, steps - done)
        for c, _ in ctxs:
            c.step(dt, k)
        done += k
        for i, (c, _) in enumerate(ctxs):
            c.synchronize()
            if finite_until[i] is None and not np.isfinite(c.get_state()[1]).all():
                finite_until[i] = done - k
    secs = time.perf_counter() - t0
    finals = [c.get_state() for c, _ in ctxs]
    for c, _ in ctxs:
        c.close()
    n_rhs = 4 * steps * len(ctxs)
    fmas = separable_fmas(M)
    peak64 = mm.mmvm_alu_peak(0, mm.MMVM_FP64) / 1e12
    achieved = 2.0 * fmas * n_rhs / secs / 1e12
    rng = np.random.default_rng(0)
    rows = sorted(set(range(10)) | set(rng.integers(10, w0.K, args.high_rows).tolist()))
    v, a = self_rhs_rows(w0.moments[0], lam_at(0.0, w0.lam0, w0.nu), M, rows)
    d = np.abs(gM[0, rows] - v)
    ok = a > 0
    return {
        "workload": "one particle, order 60 (1891 moments), Lamb-Oseen core + quadrupole on "
                    "(2,0)/(0,2)/(1,1), eps {1e-3,1e-2,0.1} x Re {1e3,1e4}: 6 instances x "
                    f"{steps} RK4 steps of {dt}, FP64 separable self term",
        "rhs_per_s": n_rhs / secs, "unit": "RHS evaluations/s", "seconds": secs,
        "steps_per_s_per_instance": steps / secs,
        "fmas_per_rhs": fmas,
        "coefficient_terms_per_rhs": coefficient_terms(60),
        "coefficient_terms_per_s": coefficient_terms(60) * n_rhs / secs,
        "coefficient_terms_note": "(k, l, i, q) terms of eq:FinalSingleI/II the literal form "
                                  "evaluates per RHS; the separable passes do fmas_per_rhs "
                                  "multiply-adds for them",
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak64, "unit": "TFLOP/s",
                     "frac": achieved / peak64,
                     "peak_note": "of measured: FP64 FMA peak measured in this run"},
        "error_vs_oracle_t0": {"rows": len(rows),
                               "max_abs_over_term_sum": float((d[ok] / a[ok]).max()),
                               "rows_without_terms_exact": bool(np.all(d[~ok] == 0.0))},
        "invariants": {"M00_unchanged": all(f[1][0, 0] == w.moments[0, 0]
                                            for f, (_, w) in zip(finals, ctxs))},
        "finite_steps": [steps if f is None else f for f in finite_until],
        "divergence_vs_perturbation": divergence_sweep(mm),
        "divergence_vs_dt": divergence_vs_dt(mm),
        "note": "the FP64 trajectories at order 60 leave the finite range early (the last "
                "finite 100-step mark is listed per instance: eps 1e-3, 1e-3, 1e-2, 1e-2, 0.1, "
                "0.1 with Re 1e3, 1e4): once every moment is populated the per-row condition "
                "number of the coefficient sums reaches 1e16-1e18 at orders >= 40, so FP64 "
                "rounding of the state seeds the top moments far above their size; the timing "
                "covers all steps (non-finite arithmetic runs at the same speed)",
    }


def _timed_steps(mm, ctx, dt, nsteps, stream):
    """Device time (ms) of nsteps RK4 steps of a context on `stream`."""
    import torch

    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    ctx.step(dt, nsteps)
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1)


def run_precision(args, mm, stream, device):
    """The precision pattern measured like for like: the same two-patch
    recipe (N = args.prec_n, M = 6, sigma = 0.1, Re = 2000, dt = 0.05), the
    same 100 RK4 steps, in (i) the plain FP64 form, (ii) mixed precision with
    every pair through the full jet (MMVM_FLAG_NO_FAR_FIELD) and (iii) mixed
    precision with the far field (point-vortex far sources and tile
    expansions).  (ii)/(i) is the gain of the precision split alone, (iii)/(ii)
    the gain of the far-field evaluation; errors are per particle against (i)
    after the 100 steps."""
    from tests.parity_util import position_error, state_error

    wl = mmvm_inputs.two_patches(n=args.prec_n, order=6, sigma=0.1, Re=2000.0, dt=0.05)
    steps = args.prec_steps
    out = {"workload": f"two co-rotating Gaussian patches, N={wl.n}, M=6, sigma=0.1, Re=2000, "
                       f"{steps} RK4 steps of {wl.dt}", "n": wl.n, "steps": steps}
    res = {}
    for name, prec, flags in (("fp64", mm.MMVM_FP64, 0),
                              ("mixed_no_far_field", mm.MMVM_MIXED_FP32, mm.MMVM_FLAG_NO_FAR_FIELD),
                              ("mixed", mm.MMVM_MIXED_FP32, 0)):
        with mm.Context(6, wl.lam0, wl.nu, prec, flags=flags, device=device) as c:
            mm.mmvm_set_stream(c.handle, stream.cuda_stream)
            c.set_state(wl.x, wl.moments, 0.0)
            c.step(wl.dt, 1)  # graph capture, warm-up
            c.set_state(wl.x, wl.moments, 0.0)
            w0 = mm.mmvm_pair_work(c.handle)
            ms = _timed_steps(mm, c, wl.dt, steps, stream)
            w1 = mm.mmvm_pair_work(c.handle)
            x, m, t = c.get_state()
        pairs = 4 * steps * wl.n * wl.n
        res[name] = (x, m, t)
        out[name] = {"value": pairs / (ms / 1e3), "unit": UNIT, "ms": ms,
                     "work": dict(zip(("near_pairs", "far_pairs_source_by_source",
                                       "tile_expansions", "pairs_in_tile_expansions"),
                                      [int(b - a) for a, b in zip(w0, w1)]))}
    x64, m64, t64 = res["fp64"]
    lam = math.sqrt(wl.lam0 ** 2 + 4 * wl.nu * t64)
    for name in ("mixed_no_far_field", "mixed"):
        x, m, t = res[name]
        out[name]["moments_rel_per_particle_vs_fp64"] = state_error(m, m64, 6, lam)
        out[name]["centroid_err_in_core_sizes_vs_fp64"] = position_error(x, x64, lam)
    out["precision_gain"] = out["mixed_no_far_field"]["value"] / out["fp64"]["value"]
    out["far_field_gain"] = out["mixed"]["value"] / out["mixed_no_far_field"]["value"]
    out["mixed_over_fp64"] = out["mixed"]["value"] / out["fp64"]["value"]
    out["note"] = ("precision_gain = (ii)/(i): FP32 jets and contractions against FP64, same "
                   "all-pairs algorithm; far_field_gain = (iii)/(ii): the point-vortex far field "
                   "and tile expansions, same precision; errors: max over particles of the "
                   "weighted moment norm relative to the particle's FP64 moments, and the "
                   "centroid distance in core sizes")
    return out


def run_single_m10(args, mm, stream):
    """Single particle, order 10 (66 moments), Lamb-Oseen core + quadrupole
    eps = 0.1 on (2,0)/(0,2)/(1,1), Re = 1000, 500 FP64 RK4 steps of 0.01:
    RHS evaluations/s, coefficient terms/s, and (cpu leg) the per-particle
    error against the oracle's 500-step trajectory."""
    wl = mmvm_inputs.single_quadrupole(order=10, eps=0.1, sigma0=1.0, Re=1000.0)
    steps = args.m10_steps
    with mm.Context(10, wl.lam0, wl.nu, mm.MMVM_FP64) as c:
        mm.mmvm_set_stream(c.handle, stream.cuda_stream)
        c.set_state(wl.x, wl.moments, 0.0)
        c.step(wl.dt, 2)
        c.set_state(wl.x, wl.moments, 0.0)
        ms = _timed_steps(mm, c, wl.dt, steps, stream)
        x, m, t = c.get_state()
    n_rhs = 4 * steps
    return {"workload": "one particle, order 10 (66 moments), Lamb-Oseen + quadrupole eps=0.1, "
                        f"Re=1000, {steps} FP64 RK4 steps of {wl.dt}",
            "rhs_per_s": n_rhs / (ms / 1e3), "unit": "RHS evaluations/s", "ms": ms,
            "coefficient_terms_per_rhs": coefficient_terms(10),
            "coefficient_terms_per_s": coefficient_terms(10) * n_rhs / (ms / 1e3),
            "_final": (wl, m, t)}


def single_m10_error(res):
    """Error of the order-10 trajectory against the oracle's (cpu leg)."""
    from oracle.rhs import lam_at, rk4
    from tests.parity_util import state_error

    wl, m, t = res.pop("_final")
    steps = round(t / wl.dt)
    t0 = time.perf_counter()
    ox, oM, ot = rk4(wl.x, wl.moments, 0.0, wl.dt, steps, 10, wl.lam0, wl.nu)
    res["oracle_seconds"] = time.perf_counter() - t0
    res["error_vs_oracle"] = {"steps": steps, "t": ot,
                              "moments_rel_weighted": state_error(m, oM, 10,
                                                                  lam_at(ot, wl.lam0, wl.nu))}


def run_random_disk(args, mm, stream, device):
    """The random-disk configuration (N = 4096, M = 4, sigma = 0.5, Re = 500,
    dt = 0.01, up to 200 RK4 steps) in mixed precision with the far field:
    throughput over the steps whose state stays finite (checked every 10
    steps), and the per-particle error against the plain FP64 form over the
    same steps."""
    from tests.parity_util import position_error, state_error

    wl = mmvm_inputs.random_disk()
    steps, chunk = args.disk_steps, 10
    with mm.Context(wl.order, wl.lam0, wl.nu, mm.MMVM_MIXED_FP32, device=device) as c:
        mm.mmvm_set_stream(c.handle, stream.cuda_stream)
        c.set_state(wl.x, wl.moments, 0.0)
        c.step(wl.dt, 1)
        c.set_state(wl.x, wl.moments, 0.0)
        done, ms_tot, last = 0, 0.0, None
        while done < steps:
            k = min(chunk, steps - done)
            ms_tot += _timed_steps(mm, c, wl.dt, k, stream)
            x, m, t = c.get_state()
            if not (np.isfinite(x).all() and np.isfinite(m).all()):
                break
            done += k
            last = (x, m, t)
    out = {"workload": f"random disk N={wl.n}, M={wl.order}, R=10, sigma={wl.lam0}, Re=500, "
                       f"dt={wl.dt}, {steps} RK4 steps (mixed precision, far field on)",
           "steps_requested": steps, "finite_steps": done,
           "value": 4 * wl.n * wl.n * done / (ms_tot / 1e3) if done else None, "unit": UNIT}
    if done:
        with mm.Context(wl.order, wl.lam0, wl.nu, mm.MMVM_FP64, device=device) as c64:
            mm.mmvm_set_stream(c64.handle, stream.cuda_stream)
            c64.set_state(wl.x, wl.moments, 0.0)
            c64.step(wl.dt, done)
            x64, m64, t64 = c64.get_state()
        x, m, t = last
        lam = math.sqrt(wl.lam0 ** 2 + 4 * wl.nu * t)
        out["error_vs_fp64"] = {"steps": done, "t": t,
                                "moments_rel_per_particle": state_error(m, m64, wl.order, lam),
                                "centroid_err_in_core_sizes": position_error(x, x64, lam)}
    out["note"] = ("the state of this dense mixed-sign random disk leaves the finite range "
                   "(the truncated moment ODE cannot follow the straining cores); throughput "
                   "and error cover the steps before the first non-finite 10-step chunk")
    return out


TRAFFIC_FILE = os.path.join(ROOT, "profiles", "pair_kernel_traffic.json")
KERNEL_SOURCES = ("common.cuh", "pair_kernel.cuh", "pair_launch.cuh", "pair_variants.h",
                  "pair_inst.cu", "pair_list.cuh", "pair_list_variants.h", "pair_list_inst.cu")


def kernel_source_hash() -> str:
    """sha256 of the all-pairs kernel's code (the DRAM traffic recorded by ncu
    belongs to one version of it): the sources with // comments and blank
    lines dropped, so that editing a comment keeps the record."""
    import hashlib

    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_1010_2475_gb300", "csrc", f)) as fh:
            lines = (ln.split("//", 1)[0].rstrip() for ln in fh.read().splitlines())
            h.update("\n".join(ln for ln in lines if ln).encode())
    return h.hexdigest()


def recorded_traffic(n: int, variant: int, chunks: int):
    """DRAM bytes per launch from the ncu capture in profiles/, or None when
    the capture was taken on other kernel sources or another launch shape."""
    try:
        with open(TRAFFIC_FILE) as f:
            rec = json.load(f)
    except (OSError, ValueError):
        return None
    if rec.get("source_hash") != kernel_source_hash() or rec.get("n") != n:
        return None
    for c in rec.get("captures", []):
        if c.get("variant") == variant and c.get("chunks") == chunks:
            return c.get("dram_bytes_per_launch")
    return None


def max_over_ranks(ms: float, dist, device) -> float:
    """The slowest rank's time (every rank gets it)."""
    import torch

    t = torch.tensor([ms], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_value(world: int, pairs_per_step: int, steps: int, max_ms: float) -> float:
    """Whole-job throughput of `world` independent replicas: every rank
    evaluates the full workload, the job takes the slowest rank's time."""
    return world * pairs_per_step * steps / (max_ms / 1e3)


def run_ours(args, wl, rank, world, local_rank):
    import torch

    import paper_1010_2475_gb300 as mm

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    # a dedicated stream: the library and the timing events must share it
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    fp32_peak = mm.mmvm_alu_peak(local_rank, mm.MMVM_MIXED_FP32) / 1e12
    ctx = mm.Context(wl.order, wl.lam0, wl.nu, mm.MMVM_MIXED_FP32, device=local_rank)
    mm.mmvm_set_stream(ctx.handle, stream.cuda_stream)
    ctx.set_state(wl.x, wl.moments, 0.0)
    mm.mmvm_enable_timing(ctx.handle, True)
    flush = torch.empty(256 * 2 ** 20 // 4, dtype=torch.float32, device=dev)
    pairs_step = 4 * wl.n * wl.n

    # accuracy of this run's arithmetic: right-hand side at t = 0 vs the oracle
    gx0, gM0 = ctx.rhs()
    for _ in range(args.warmup):
        ctx.step(wl.dt, 1)
    torch.cuda.synchronize(dev)
    mm.mmvm_pair_time(ctx.handle)
    mm.mmvm_pair_time_parts(ctx.handle)  # drop the warm-up's split
    work0 = mm.mmvm_pair_work(ctx.handle)
    if dist:
        dist.barrier()
    torch.cuda.synchronize(dev)
    launches0 = ctx.launches
    step_ms, pair_ms, pair_cnt = [], 0.0, 0
    with ClockSampler(local_rank) as clk:
        for _ in range(args.steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ctx.step(wl.dt, 1)
            e1.record(stream)
            e1.synchronize()
            step_ms.append(e0.elapsed_time(e1))
            ms, cnt = mm.mmvm_pair_time(ctx.handle)
            pair_ms += ms
            pair_cnt += cnt
    torch.cuda.synchronize(dev)
    launches = ctx.launches - launches0
    work1 = mm.mmvm_pair_work(ctx.handle)
    parts_ms, parts_cnt = mm.mmvm_pair_time_parts(ctx.handle)
    total_ms = sum(step_ms)
    if dist:
        total_ms = max_over_ranks(total_ms, dist, dev)
        dist.barrier()
    value = replica_value(world, pairs_step, args.steps, total_ms)

    # end to end through the C ABI with pinned host buffers
    K = wl.K
    hx = torch.empty((wl.n, 2), dtype=torch.float64, pin_memory=True).numpy()
    hm = torch.empty((wl.n, K), dtype=torch.float64, pin_memory=True).numpy()
    ox_ = torch.empty((wl.n, 2), dtype=torch.float64, pin_memory=True).numpy()
    om_ = torch.empty((wl.n, K), dtype=torch.float64, pin_memory=True).numpy()
    x_cur, m_cur, t_cur = ctx.get_state()
    hx[:] = x_cur
    hm[:] = m_cur
    e2e_s = []
    lib = mm.load_library()
    for _ in range(args.e2e_steps):
        t0 = time.perf_counter()
        ctx.set_state(hx, hm, t_cur)
        ctx.step(wl.dt, 1)
        tt = np.zeros(1)
        mm._check(lib.mmvm_get_state(ctx.handle, mm._dptr(ox_), mm._dptr(om_), mm._dptr(tt)))
        e2e_s.append(time.perf_counter() - t0)
        hx[:] = ox_
        hm[:] = om_
        t_cur = float(tt[0])
    e2e_val = world * pairs_step / statistics.mean(e2e_s) if e2e_s else None
    bytes_state = wl.n * (2 + K) * 8

    # plain FP64 form on a subset (one right-hand side, device-timed)
    fp64 = None
    if not args.skip_fp64:
        sub = wl.subset(min(FP64_SUBSET, wl.n))
        c64 = mm.Context(sub.order, sub.lam0, sub.nu, mm.MMVM_FP64, device=local_rank)
        mm.mmvm_set_stream(c64.handle, stream.cuda_stream)
        c64.set_state(sub.x, sub.moments, 0.0)
        c64.rhs()
        mm.mmvm_enable_timing(c64.handle, True)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        d_dx = torch.empty((sub.n, 2), dtype=torch.float64, device=dev)
        d_dm = torch.empty((sub.n, sub.K), dtype=torch.float64, device=dev)
        e0.record(stream)
        mm.mmvm_rhs_device(c64.handle, d_dx.data_ptr(), d_dm.data_ptr())
        e1.record(stream)
        e1.synchronize()
        rhs_ms = e0.elapsed_time(e1)
        p64_ms, _ = mm.mmvm_pair_time(c64.handle)
        c32 = mm.Context(sub.order, sub.lam0, sub.nu, mm.MMVM_MIXED_FP32, device=local_rank)
        mm.mmvm_set_stream(c32.handle, stream.cuda_stream)
        c32.set_state(sub.x, sub.moments, 0.0)
        c32.rhs()
        mm.mmvm_enable_timing(c32.handle, True)
        e0.record(stream)
        mm.mmvm_rhs_device(c32.handle, d_dx.data_ptr(), d_dm.data_ptr())
        e1.record(stream)
        e1.synchronize()
        rhs32_ms = e0.elapsed_time(e1)
        cnf = mm.Context(sub.order, sub.lam0, sub.nu, mm.MMVM_MIXED_FP32, device=local_rank,
                         flags=mm.MMVM_FLAG_NO_FAR_FIELD)
        mm.mmvm_set_stream(cnf.handle, stream.cuda_stream)
        cnf.set_state(sub.x, sub.moments, 0.0)
        cnf.rhs()
        e0.record(stream)
        mm.mmvm_rhs_device(cnf.handle, d_dx.data_ptr(), d_dm.data_ptr())
        e1.record(stream)
        e1.synchronize()
        rhsnf_ms = e0.elapsed_time(e1)
        fp64 = {"value": sub.n * sub.n / (rhs_ms / 1e3), "unit": UNIT,
                "workload": f"first {sub.n} particles of the workload, one right-hand side",
                "ms_per_rhs": rhs_ms, "pair_kernel_ms": p64_ms,
                "mixed_no_far_field_same_subset": sub.n * sub.n / (rhsnf_ms / 1e3),
                "mixed_same_subset": sub.n * sub.n / (rhs32_ms / 1e3),
                "precision_gain": rhs_ms / rhsnf_ms,
                "far_field_gain": rhsnf_ms / rhs32_ms,
                "mixed_over_fp64": rhs_ms / rhs32_ms}
        c64.close()
        c32.close()
        cnf.close()
    wall = {}
    t_sec = time.perf_counter()
    precision = run_precision(args, mm, stream, local_rank) if args.prec_steps > 0 else None
    wall["precision"] = time.perf_counter() - t_sec
    t_sec = time.perf_counter()
    single_m10 = run_single_m10(args, mm, stream) if args.m10_steps > 0 else None
    wall["single_m10"] = time.perf_counter() - t_sec
    t_sec = time.perf_counter()
    disk = run_random_disk(args, mm, stream, local_rank) if args.disk_steps > 0 else None
    wall["random_disk"] = time.perf_counter() - t_sec
    scaling = None
    if args.scaling:
        t_sec = time.perf_counter()
        scaling = run_scaling(args, mm, stream, local_rank)
        wall["scaling"] = time.perf_counter() - t_sec

    line = None
    pcfg = mm.mmvm_pair_config(ctx.handle)
    if rank == 0:
        avg_pair_s = pair_ms / max(pair_cnt, 1) / 1e3
        fpp = flops_per_pair(wl.order)
        ffp = far_flops_per_pair(wl.order)
        fm2p = m2p_flops(wl.order)
        near_l, far_l, m2p_l, m2p_pairs_l = [(b - a) / max(pair_cnt, 1)
                                             for a, b in zip(work0, work1)]
        flops_launch = near_l * fpp + far_l * ffp + m2p_l * fm2p
        achieved = flops_launch / avg_pair_s / 1e12
        per_kernel = None
        if parts_ms and parts_cnt:
            # list form: [list build + tree, far field, near kernels...]
            pcfg0 = mm.mmvm_pair_config(ctx.handle)
            fe, fl = flops_per_pair_parts(wl.order)
            names = ["near_list_kernel + tree_level_kernel",
                     "far_tree_kernel" if pcfg0["list_form"] == 2 else "far_pair_kernel"]
            flops = [0.0, far_l * ffp + m2p_l * fm2p]
            near_parts = len(parts_ms) - 2
            if near_parts == 1:
                names.append("near_pair_kernel (all columns)")
                flops.append(near_l * fpp)
            else:
                names.append("near_pair_kernel edge part")
                flops.append(near_l * fe)
                for k in range(near_parts - 1):
                    names.append(f"near_pair_kernel Laplacian part {k + 1}")
                    flops.append(near_l * fl / (near_parts - 1))
            per_kernel = []
            for nm, f, t in zip(names, flops, parts_ms):
                ms_rhs = t / parts_cnt
                tf = f / (ms_rhs / 1e3) / 1e12 if ms_rhs > 0 and f > 0 else None
                per_kernel.append({"kernel": nm, "ms_per_rhs": ms_rhs, "flops_per_rhs": f,
                                   "achieved_tflops": tf,
                                   "frac": tf / fp32_peak if tf is not None else None})
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": total_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": config_dict(wl, {"parallelism": f"replicas x{world}"}),
                "clocks": clk.summary(),
                "e2e": {"value": e2e_val, "unit": UNIT,
                        "h2d_bytes_per_step": bytes_state, "d2h_bytes_per_step": bytes_state + 8,
                        "steps": args.e2e_steps},
                "gpu_launches": launches,
                "pair_kernel_config": pcfg,
                "near_pairs_per_s": world * near_l * 4 * args.steps / (total_ms / 1e3),
                "pairs_by_path_per_rhs": {"near_full_jet": near_l,
                                          "far_point_vortex_source_by_source": far_l,
                                          "far_in_tile_expansions": m2p_pairs_l},
                "roofline": {"bound": "alu", "achieved": achieved, "peak": fp32_peak,
                             "unit": "TFLOP/s", "frac": achieved / fp32_peak,
                             "traffic": recorded_traffic(wl.n, pcfg["variant"], pcfg["chunks"]),
                             "traffic_note": "dram__bytes_read.sum + dram__bytes_write.sum of one "
                                             "launch (profiles/pair_kernel_traffic.json; null "
                                             "if the kernel sources or launch shape differ "
                                             "from the capture)",
                             "kernel": ("list form: near_list_kernel, tree_level_kernel, "
                                        "far_tree_kernel / far_pair_kernel, near_pair_kernel"
                                        if pcfg.get("list_form") else
                                        "pair_kernel (all-pairs jet + contraction)"),
                             "flops_per_pair": {"near": fpp, "far": ffp},
                             "flops_per_tile_expansion": fm2p,
                             "pairs_per_launch": {"near": near_l, "far_source_by_source": far_l,
                                                  "far_by_tile_expansion": m2p_pairs_l},
                             "tile_expansions_per_launch": m2p_l,
                             "flops_per_launch": flops_launch,
                             "launch_ms": avg_pair_s * 1e3,
                             "launches_timed": pair_cnt,
                             "peak_note": "of measured: FP32 FMA peak measured in this run "
                                          "(mmvm_alu_peak); nominal 152 SMs x 128 lanes x 2 "
                                          "flop x 2.07 GHz = %.1f TFLOP/s" % FP32_PEAK_TFLOPS,
                             "frac_of_nominal": achieved / FP32_PEAK_TFLOPS,
                             "per_kernel": per_kernel,
                             "per_kernel_note": "event-timed between the list form's launches; "
                                                "the Laplacian flops of a split near part are "
                                                "shared evenly between its kernels"},
                "fp64": fp64,
                "mixed_vs_fp64_100_steps": precision,
                "single_m10": single_m10,
                "random_disk_n4096": disk}
        if scaling is not None:
            line["scaling_n"] = scaling
        if args.serve_requests > 0:
            t_sec = time.perf_counter()
            line["served"] = run_served(args, mm)
            wall["served"] = time.perf_counter() - t_sec
        if args.high_steps > 0:
            t_sec = time.perf_counter()
            line["single_m60"] = run_single_high(args, mm)
            wall["single_m60"] = time.perf_counter() - t_sec
        if not args.skip_cpu:
            rate, secs, sel, ox, oM = oracle_rate(wl, args.oracle_rows)
            line["cpu_baseline"] = {
                "value": rate, "unit": UNIT, "cores": cpu_cores_used(), "kind": "oracle",
                "sample": f"{args.oracle_rows} random target rows x all {wl.n} sources, one "
                          f"right-hand side at t=0 ({secs:.1f} s, FP64 numpy oracle)"}
            procs = args.oracle_procs or os.cpu_count() or 1
            rows_all, ox_all, oM_all = [sel], [ox], [oM]
            if procs > 1:
                v_all, secs_all, rr, ox2, oM2 = oracle_rate_all_cores(wl, args.oracle_rows, procs,
                                                                     seed=99, keep=True)
                rows_all.append(rr)
                ox_all.append(ox2)
                oM_all.append(oM2)
                line["cpu_baseline_all_cores"] = {
                    "value": v_all, "unit": UNIT, "cores": procs, "kind": "oracle",
                    "sample": f"{procs} processes x {args.oracle_rows} random target rows x all "
                              f"{wl.n} sources, one right-hand side at t=0 ({secs_all:.1f} s)"}
            line["error_vs_oracle"] = error_vs_oracle(wl, gx0, gM0, np.concatenate(rows_all),
                                                      np.concatenate(ox_all),
                                                      np.concatenate(oM_all), procs)
            if single_m10 is not None:
                single_m10_error(single_m10)
        elif single_m10 is not None:
            single_m10.pop("_final", None)
        line["section_wall_s"] = wall
    ctx.close()
    if dist:
        dist.destroy_process_group()
    if line is not None:
        print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--oracle-rows", type=int, default=4,
                    help="random target rows per oracle process (one process per host core)")
    ap.add_argument("--ref-rows", type=int, default=2,
                    help="random target rows per oracle process per step of --impl reference")
    ap.add_argument("--oracle-procs", type=int, default=0,
                    help="processes of the all-cores oracle timing (0: one per host core)")
    ap.add_argument("--skip-fp64", action="store_true")
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--serve-requests", type=int, default=300,
                    help="requests of the served stream (0: skip the serving measurement)")
    ap.add_argument("--serve-burst", type=int, default=60,
                    help="first requests of the stream submitted at once (saturation, batching "
                         "gain)")
    ap.add_argument("--serve-check", type=int, default=3,
                    help="smallest served requests re-run in FP64 for their error")
    ap.add_argument("--serve-fp64", type=int, default=4,
                    help="smallest served requests run through an FP64 server as well")
    ap.add_argument("--high-steps", type=int, default=2000,
                    help="RK4 steps of the order-60 single-particle instances (0: skip)")
    ap.add_argument("--high-rows", type=int, default=8,
                    help="sampled rows of the order-60 RHS checked against the oracle")
    ap.add_argument("--prec-n", type=int, default=4096,
                    help="particles of the like-for-like precision comparison")
    ap.add_argument("--prec-steps", type=int, default=100,
                    help="RK4 steps of the precision comparison (0: skip)")
    ap.add_argument("--m10-steps", type=int, default=500,
                    help="FP64 RK4 steps of the order-10 single particle (0: skip)")
    ap.add_argument("--disk-steps", type=int, default=200,
                    help="RK4 steps of the N = 4096 random disk (0: skip)")
    ap.add_argument("--scaling", type=str, default="",
                    help="comma-separated N of the growing-N measurement (empty: skip)")
    ap.add_argument("--scaling-fixed-max", type=int, default=262144,
                    help="largest N of the fixed-sigma part of --scaling")
    ap.add_argument("--n", type=int, default=65536,
                    help="particles (the benchmark is 65536; smaller only for profiling)")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    wl = workload(args.n)
    if args.impl == "reference":
        if rank == 0:
            run_reference(args, wl)
        return
    if world > 1 or args.gpus > 1:
        args.skip_cpu = args.skip_cpu or rank != 0
    run_ours(args, wl, rank, world, local_rank)


if __name__ == "__main__":
    main()
