"""Serving (mmvm_server_*): continuous batching of independent simulations.

* Each result is the same alone and in a mix: the same requests run one at
  a time on one server and all together (with arrivals while others are on
  the GPU) on another, and the final states agree bit for bit (the split of
  a simulation's pairs into work items depends on its own size only, and
  every item is summed in a fixed order).
* Served results agree with the context API stepping the same simulation
  (mixed: 1e-5 relative on moments, the trajectory tolerance of the parity
  tests; FP64: 1e-12) and, for a small case, with the FP64 oracle.
* Admission by footprint: a budget that holds the largest simulation alone
  never holds them all at once; a request larger than the whole budget is
  refused.
* A request whose state diverges stops early with MMVM_E_NUMERIC.
"""
import math
import time

import numpy as np
import pytest

import mmvm_inputs
from oracle.rhs import lam_at, rk4
from tests.parity_util import state_error

pytestmark = pytest.mark.gpu

MIXED_TRAJ_TOL = 1e-5
FP64_TOL = 1e-12


@pytest.fixture(scope="module")
def mm():
    import paper_1010_2475_gb300 as mm

    mm.load_library()
    return mm


def _patches(n, order, Re, sigma, dt, seed):
    """Two-patch state (positive circulations) with small random moments of
    orders 2..M, M_k ~ 0.05 M_00 sigma^|k| / |k|! (the random-disk recipe of
    the served stream has near-zero circulations and large random moments;
    a few of its small instances blow up within a few steps, in the oracle
    too, which would test nothing here)."""
    wl = mmvm_inputs.two_patches(n=n, order=order, sigma=sigma, Re=Re, dt=dt,
                                 radius=0.6 + 0.08 * n ** 0.5, separation=3.0, seed=seed)
    if order >= 2:
        rng = np.random.default_rng(seed + 1)
        tot = np.concatenate([[s] * (s + 1) for s in range(order + 1)])[3:]
        scale = 0.05 * sigma ** tot / np.array([math.factorial(int(v)) for v in tot])
        wl.moments[:, 3:] = wl.moments[:, :1] * rng.standard_normal((n, wl.K - 3)) * scale
    return wl


def _requests():
    """Uneven simulations: particle counts across several tiles, every order
    of the served mix plus a lone high-order particle, different viscosities,
    core sizes and step counts."""
    spec = [  # (n, order, Re, sigma, steps, dt)
        (40, 2, 300.0, 0.5, 7, 0.01),
        (97, 4, 1500.0, 0.45, 5, 0.01),
        (150, 8, 800.0, 0.5, 3, 0.005),
        (260, 4, 4000.0, 0.5, 6, 0.01),
        (1, 10, 1000.0, 1.0, 9, 0.01),
        (600, 2, 120.0, 0.55, 4, 0.02),
        (333, 6, 2500.0, 0.5, 2, 0.01),
        (64, 4, 900.0, 0.5, 4, 0.01),     # shares a batch with the n = 97, M = 4 one
        (120, 8, 2000.0, 0.45, 2, 0.005),  # shares a batch with the n = 150, M = 8 one
    ]
    out = []
    for i, (n, order, Re, sigma, steps, dt) in enumerate(spec):
        if n == 1:
            wl = mmvm_inputs.single_quadrupole(order=order, eps=0.1, sigma0=sigma, Re=Re, dt=dt)
        else:
            wl = _patches(n, order, Re, sigma, dt, 900 + i)
        out.append((wl, steps))
    return out


def _submit(srv, wl, steps):
    return srv.submit(wl.x, wl.moments, wl.order, wl.lam0, wl.nu, wl.dt, steps, t0=0.0)


def _alone(mm, reqs, prec):
    res = []
    with mm.Server(precision=prec) as srv:
        for wl, steps in reqs:
            res.append(srv.wait(_submit(srv, wl, steps)))
    return res


def _mixed(mm, reqs, prec):
    with mm.Server(precision=prec) as srv:
        first = [_submit(srv, wl, s) for wl, s in reqs[:3]]
        # the rest arrive while the first ones are on the GPU
        while srv.stats()["ticks"] < 1:
            time.sleep(0.001)
        rest = [_submit(srv, wl, s) for wl, s in reqs[3:]]
        out = [srv.wait(t) for t in first + rest]
        st = srv.stats()
    return out, st


def test_same_alone_and_in_the_mix(mm):
    reqs = _requests()
    alone = _alone(mm, reqs, mm.MMVM_MIXED_FP32)
    mixed, st = _mixed(mm, reqs, mm.MMVM_MIXED_FP32)
    assert st["completed"] == len(reqs) and st["failed"] == 0
    assert st["max_active"] >= 3  # they really ran together
    assert st["max_batch"] >= 2  # and shared batches
    for (wl, steps), (xa, ma, ia), (xm, mm_, im) in zip(reqs, alone, mixed):
        assert ia["steps"] == im["steps"] == steps
        assert ia["t"] == im["t"]
        assert np.array_equal(xa, xm), f"positions differ for n={wl.n} M={wl.order}"
        assert np.array_equal(ma, mm_), f"moments differ for n={wl.n} M={wl.order}"


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_served_matches_context(mm, prec):
    p = mm.MMVM_MIXED_FP32 if prec == "mixed" else mm.MMVM_FP64
    tol = MIXED_TRAJ_TOL if prec == "mixed" else FP64_TOL
    reqs = _requests()
    with mm.Server(precision=p) as srv:
        tickets = [_submit(srv, wl, s) for wl, s in reqs]
        served = [srv.wait(t) for t in tickets]
    for (wl, steps), (x, m, info) in zip(reqs, served):
        with mm.Context(wl.order, wl.lam0, wl.nu, p, flags=mm.MMVM_FLAG_NO_FAR_FIELD) as ctx:
            ctx.set_state(wl.x, wl.moments, 0.0)
            ctx.step(wl.dt, steps)
            cx, cm, ct = ctx.get_state()
        assert abs(info["t"] - ct) <= 1e-15 * max(1.0, abs(ct))
        lam = lam_at(ct, wl.lam0, wl.nu)
        assert np.abs(x - cx).max() <= tol * lam
        assert state_error(m, cm, wl.order, lam) <= tol


def test_served_matches_oracle_small(mm):
    wl = _patches(24, 3, 700.0, 0.5, 0.01, 950)
    steps = 4
    with mm.Server(precision=mm.MMVM_MIXED_FP32) as srv:
        x, m, info = srv.wait(_submit(srv, wl, steps))
    ox, om, t = rk4(wl.x, wl.moments, 0.0, wl.dt, steps, wl.order, wl.lam0, wl.nu)
    assert info["t"] == t
    lam = lam_at(t, wl.lam0, wl.nu)
    assert np.abs(x - ox).max() <= MIXED_TRAJ_TOL * lam
    assert state_error(m, om, wl.order, lam) <= MIXED_TRAJ_TOL


def test_admission_by_footprint(mm):
    reqs = _requests()[:4]
    fps = [mm.mmvm_request_footprint(wl.order, mm.MMVM_MIXED_FP32, wl.n) for wl, _ in reqs]
    budget = max(fps)  # the largest fits alone; all four never fit together
    with mm.Server(precision=mm.MMVM_MIXED_FP32, hbm_budget_bytes=budget) as srv:
        tickets = [_submit(srv, wl, s) for wl, s in reqs]
        out = [srv.wait(t) for t in tickets]
        st = srv.stats()
    assert st["completed"] == len(reqs)
    assert st["peak_footprint_bytes"] <= budget
    assert st["max_active"] < len(reqs)
    # same results as without the budget
    alone = _alone(mm, reqs, mm.MMVM_MIXED_FP32)
    for (xa, ma, _), (xb, mb, _) in zip(alone, out):
        assert np.array_equal(xa, xb) and np.array_equal(ma, mb)


def test_submit_errors(mm):
    wl = _patches(50, 2, 500.0, 0.5, 0.01, 960)
    with mm.Server(precision=mm.MMVM_MIXED_FP32, hbm_budget_bytes=1 << 12) as srv:
        with pytest.raises(mm.MMVMError) as ei:  # bigger than the whole budget
            _submit(srv, wl, 3)
        assert ei.value.code == mm.MMVM_E_OOM
    with mm.Server(precision=mm.MMVM_MIXED_FP32) as srv:
        bad = wl.moments.copy()
        bad[7, 0] = 0.0
        with pytest.raises(mm.MMVMError) as ei:
            srv.submit(wl.x, bad, wl.order, wl.lam0, wl.nu, wl.dt, 3)
        assert ei.value.code == mm.MMVM_E_ZERO_CIRCULATION
        with pytest.raises(mm.MMVMError) as ei:  # a ticket that was never issued
            mm._check(mm.load_library().mmvm_poll(srv.handle, 12345, None, None, None))
        assert ei.value.code == mm.MMVM_E_INVALID_ARG
        t = _submit(srv, wl, 0)  # zero steps: the input state comes back
        x, m, info = srv.wait(t)
        assert np.array_equal(x, wl.x) and np.array_equal(m, wl.moments)


def test_divergent_request_stops_early(mm):
    """A state whose ODE leaves the finite range within a few steps (large
    absolute random moments at M = 8; the FP64 oracle gives NaN after three
    steps of 0.005 from this state) is stopped with MMVM_E_NUMERIC at the
    step where it diverged, and does not disturb a request beside it."""
    bad = mmvm_inputs.random_disk(n=150, order=8, radius=2.0 + 0.15 * 150 ** 0.5, sigma=0.5,
                                  amp=0.03, moment_scale="absolute", Re=800.0, dt=0.005,
                                  seed=902)
    good, gsteps = _requests()[0]
    with mm.Server(precision=mm.MMVM_MIXED_FP32) as srv:
        tb = srv.submit(bad.x, bad.moments, bad.order, bad.lam0, bad.nu, bad.dt, 400)
        tg = _submit(srv, good, gsteps)
        with pytest.raises(mm.MMVMError) as ei:
            srv.wait(tb)
        assert ei.value.code == mm.MMVM_E_NUMERIC
        assert 1 <= ei.value.info["steps"] < 400
        xg, mg, ig = srv.wait(tg)
    (xa, ma, ia), = _alone(mm, [(good, gsteps)], mm.MMVM_MIXED_FP32)
    assert np.array_equal(xg, xa) and np.array_equal(mg, ma)
