"""The coarse-grid tripole (Section 3.2.2) on the GPU against the paper's
Table 1 (Section 4.2, tests/golden/table1_tripole_errors.txt) and the
oracle.

The 6 x 6 grid runs with m = 0 and m = 2 (n = 36, FP64 contexts) and the
reference is one particle at order 24 carrying the expansion of the same
initial field (the separable self term); all three integrate with the
adaptive Dormand-Prince pair at 1e-8, the paper's tolerance, and their
vorticity is rebuilt on a uniform grid on [-6, 6]^2 by mmvm_vorticity.

Checked: the coarse-grid states against the oracle's after t = 1 (same
integrator, 1e-9); the reference against the oracle's order-24 run over a
short interval; and Table 1's claims over t = 1 .. 16: m = 2 about four times
more accurate than m = 0 early, still better by t = 16, errors growing with
t, magnitudes within a factor 2.5 of the table (0.5-0.7 of it with this
project's readings of the unstated grid details).
"""
import numpy as np
import pytest

import mmvm_inputs
from oracle.diagnostics import relative_errors, shifted_gaussians_expansion
from oracle.integrate import dopri5
from oracle.rhs import lam_at
from tests.parity_util import state_error
from tests.test_oracle_tripole import table1

pytestmark = pytest.mark.gpu

REF_ORDER = 24


@pytest.fixture(scope="module")
def mm():
    import paper_1010_2475_gb300 as mm

    mm.load_library()
    return mm


def _grid(half=6.0, npt=121):
    g = np.linspace(-half, half, npt)
    P1, P2 = np.meshgrid(g, g, indexing="ij")
    return np.stack([P1.ravel(), P2.ravel()], axis=1)


def _initial():
    wl0 = mmvm_inputs.tripole_coarse_grid(order=0)
    states = {m: mmvm_inputs.tripole_coarse_grid(order=m) for m in (0, 2)}
    ref = shifted_gaussians_expansion(wl0.x, wl0.moments[:, 0], REF_ORDER)
    return wl0, states, ref


def test_coarse_grid_and_reference_match_the_oracle(mm):
    wl0, states, ref = _initial()
    for m, wl in states.items():
        ox, om, ot, oa, orj = dopri5(wl.x, wl.moments, 0.0, 1.0, 0.01, m, wl.lam0, wl.nu,
                                     rtol=1e-8, atol=1e-8)
        with mm.Context(m, wl.lam0, wl.nu, mm.MMVM_FP64) as ctx:
            ctx.set_state(wl.x, wl.moments, 0.0)
            acc, rej = ctx.integrate(1.0, h0=0.01, rtol=1e-8, atol=1e-8)
            gx, gm, gt = ctx.get_state()
        assert (acc, rej) == (oa, orj)
        lam = lam_at(1.0, wl.lam0, wl.nu)
        assert np.abs(gx - ox).max() <= 1e-9 * lam
        if m >= 2:
            assert state_error(gm, om, m, lam) <= 1e-9
    T = 0.1
    ox, om, *_ = dopri5(np.zeros((1, 2)), ref, 0.0, T, 0.01, REF_ORDER, wl0.lam0, wl0.nu,
                        rtol=1e-8, atol=1e-8)
    with mm.Context(REF_ORDER, wl0.lam0, wl0.nu, mm.MMVM_FP64) as ctx:
        ctx.set_state(np.zeros((1, 2)), ref, 0.0)
        ctx.integrate(T, h0=0.01, rtol=1e-8, atol=1e-8)
        gx, gm, _ = ctx.get_state()
    assert np.all(gx == 0.0)
    assert state_error(gm, om, REF_ORDER, lam_at(T, wl0.lam0, wl0.nu)) <= 1e-9


def test_table_1(mm):
    wl0, states, ref = _initial()
    pts = _grid()
    paper = table1()
    ctxs = {}
    for m, wl in states.items():
        ctxs[m] = mm.Context(m, wl.lam0, wl.nu, mm.MMVM_FP64)
        ctxs[m].set_state(wl.x, wl.moments, 0.0)
    ctxs["ref"] = mm.Context(REF_ORDER, wl0.lam0, wl0.nu, mm.MMVM_FP64)
    ctxs["ref"].set_state(np.zeros((1, 2)), ref, 0.0)
    errs = {}
    try:
        for T in sorted(paper):
            fields = {}
            for k, c in ctxs.items():
                c.integrate(float(T), h0=0.01, rtol=1e-8, atol=1e-8)
                fields[k] = c.vorticity(pts)
            errs[T] = {m: relative_errors(fields[m], fields["ref"]) for m in (0, 2)}
    finally:
        for c in ctxs.values():
            c.close()
    for T, want in paper.items():
        e0, e2 = errs[T][0], errs[T][2]
        for got, w in zip((e0[0], e2[0], e0[1], e2[1]), want):
            assert w / 2.5 < got < w * 2.5, (T, errs[T])
        # Table 1: L2 ratio 3.7 (t <= 2), 3.5 (t = 4), 3.1 (t = 8), 2.1 (t = 16)
        assert e0[0] / e2[0] > (2.5 if T <= 4 else 1.5), (T, errs[T])
        assert e0[1] / e2[1] > (2.0 if T <= 4 else 1.3), (T, errs[T])
    ts = sorted(paper)
    for m in (0, 2):
        l2 = [errs[T][m][0] for T in ts]
        assert all(b > a for a, b in zip(l2, l2[1:]))
