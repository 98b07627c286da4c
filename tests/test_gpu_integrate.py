"""Adaptive Dormand-Prince 5(4) on the GPU (mmvm_integrate) against the
oracle's dopri5 (same tableau, error norm and controller, so the same step
sequence) and against the closed-form rotation of two order-0 vortices.

FP64: the two runs take the same accepted/rejected steps and agree to 1e-10
(relative, weighted norm for moments; positions relative to lambda).  Mixed
precision: within the trajectory tolerance of the parity tests (1e-5) of the
FP64 GPU run.
"""
import math

import numpy as np
import pytest

import mmvm_inputs
from oracle.integrate import dopri5
from oracle.rhs import lam_at
from tests.parity_util import state_error

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mm():
    import paper_1010_2475_gb300 as mm

    mm.load_library()
    return mm


def _state(n, order, seed):
    wl = mmvm_inputs.two_patches(n=n, order=order, sigma=0.5, Re=800.0, dt=0.01,
                                 radius=0.8, separation=2.5, seed=seed)
    if order >= 2:
        rng = np.random.default_rng(seed)
        wl.moments[:, 3:] = rng.normal(size=wl.moments[:, 3:].shape) * 0.01 \
            * wl.moments[:, :1] * wl.lam0 ** 2
    return wl


@pytest.mark.parametrize("n,order", [(24, 3), (40, 4), (1, 10)])
def test_fp64_matches_oracle_step_for_step(mm, n, order):
    if n == 1:
        wl = mmvm_inputs.single_quadrupole(order=order, eps=0.1, sigma0=1.0, Re=1000.0)
    else:
        wl = _state(n, order, 80 + order)
    T = 0.6 if n > 1 else 2.0
    ox, om, ot, oa, orj = dopri5(wl.x, wl.moments, 0.0, T, 0.02, order, wl.lam0, wl.nu,
                                 rtol=1e-9, atol=1e-9)
    with mm.Context(order, wl.lam0, wl.nu, mm.MMVM_FP64) as ctx:
        ctx.set_state(wl.x, wl.moments, 0.0)
        acc, rej = ctx.integrate(T, h0=0.02, rtol=1e-9, atol=1e-9)
        gx, gm, gt = ctx.get_state()
    assert gt == T and ot == T
    assert (acc, rej) == (oa, orj)
    lam = lam_at(T, wl.lam0, wl.nu)
    assert np.abs(gx - ox).max() <= 1e-10 * lam
    if order >= 2:
        assert state_error(gm, om, order, lam) <= 1e-10


def test_two_vortices_rotate_at_the_closed_form_rate(mm):
    G1, G2, d, lam0, nu, T = 1.0, 0.5, 1.2, 0.5, 0.0, 6.0
    x = np.array([[-d / 2, 0.0], [d / 2, 0.0]])
    mom = np.array([[G1], [G2]])
    with mm.Context(0, lam0, nu, mm.MMVM_FP64) as ctx:
        ctx.set_state(x, mom, 0.0)
        ctx.integrate(T, h0=0.01, rtol=1e-11, atol=1e-11)
        gx, gm, gt = ctx.get_state()
    theta = (G1 + G2) / (2 * math.pi * d * d) * (1.0 - math.exp(-d * d / (2 * lam0 * lam0))) * T
    c = (G1 * x[0] + G2 * x[1]) / (G1 + G2)
    rot = np.array([[math.cos(theta), -math.sin(theta)], [math.sin(theta), math.cos(theta)]])
    assert np.abs(gx - ((x - c) @ rot.T + c)).max() < 1e-8


def test_mixed_precision_follows_fp64(mm):
    wl = _state(2048, 4, 90)
    T = 0.3
    out = {}
    for name, prec in (("fp64", mm.MMVM_FP64), ("mixed", mm.MMVM_MIXED_FP32)):
        with mm.Context(4, wl.lam0, wl.nu, prec) as ctx:
            ctx.set_state(wl.x, wl.moments, 0.0)
            ctx.integrate(T, h0=0.02, rtol=1e-7, atol=1e-7)
            out[name] = ctx.get_state()
    lam = lam_at(T, wl.lam0, wl.nu)
    assert np.abs(out["mixed"][0] - out["fp64"][0]).max() <= 1e-5 * lam
    assert state_error(out["mixed"][1], out["fp64"][1], 4, lam) <= 1e-5


def test_step_limit_and_bad_arguments(mm):
    wl = _state(24, 2, 95)
    with mm.Context(2, wl.lam0, wl.nu, mm.MMVM_FP64) as ctx:
        ctx.set_state(wl.x, wl.moments, 0.0)
        with pytest.raises(mm.MMVMError) as ei:
            ctx.integrate(5.0, h0=1e-4, max_steps=3)
        assert ei.value.code == mm.MMVM_E_TIMEOUT
        t_after = ctx.get_state()[2]
        assert 0.0 < t_after < 5.0
        with pytest.raises(mm.MMVMError) as ei:
            ctx.integrate(t_after - 1.0)
        assert ei.value.code == mm.MMVM_E_INVALID_ARG
