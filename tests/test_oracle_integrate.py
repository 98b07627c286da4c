"""Pins of the oracle's adaptive Dormand-Prince 5(4) integrator
(oracle/integrate.py).

* Order 0 is the core-spreading vortex method (Section 3.2.2): two vortices
  of circulations G1, G2 at distance d rotate rigidly about their centre of
  vorticity at Omega(t) = (G1+G2)/(2 pi d^2) (1 - exp(-d^2 / (2 lambda(t)^2))),
  lambda(t)^2 = lambda_0^2 + 4 nu t.  The rotation angle int_0^T Omega dt is
  evaluated independently by adaptive quadrature.
* The same right-hand side integrated by scipy's Runge-Kutta 4(5)
  (an independent implementation with its own error norm and step control)
  agrees within a few times the tolerance.
* A fifth-order method takes about 10x more steps for 1e5x tighter
  tolerance (steps ~ tol^(-1/5)).
"""
import math

import numpy as np
import pytest
from scipy.integrate import quad, solve_ivp

from oracle.integrate import dopri5
from oracle.rhs import rhs_regrouped


def _pair(G1, G2, d):
    x = np.array([[-d / 2, 0.0], [d / 2, 0.0]])
    mom = np.array([[G1], [G2]])
    return x, mom


@pytest.mark.parametrize("nu", [0.0, 0.01])
def test_two_vortices_rotate_at_the_closed_form_rate(nu):
    G1, G2, d, lam0, T = 1.0, 0.5, 1.2, 0.5, 6.0
    x, mom = _pair(G1, G2, d)
    xe, me, t, acc, rej = dopri5(x, mom, 0.0, T, 0.01, 0, lam0, nu, rtol=1e-11, atol=1e-11)
    assert t == T and acc > 0
    omega = lambda s: (G1 + G2) / (2 * math.pi * d * d) * (
        1.0 - math.exp(-d * d / (2 * (lam0 * lam0 + 4 * nu * s))))
    theta, _ = quad(omega, 0.0, T, epsabs=1e-13, epsrel=1e-13)
    c = (G1 * x[0] + G2 * x[1]) / (G1 + G2)  # centre of vorticity
    rot = np.array([[math.cos(theta), -math.sin(theta)], [math.sin(theta), math.cos(theta)]])
    expect = (x - c) @ rot.T + c
    assert np.abs(xe - expect).max() < 1e-8
    assert np.all(me == mom)  # order 0: the circulations never change


def test_agrees_with_an_independent_rk45():
    rng = np.random.default_rng(4)
    n, order, lam0, nu = 5, 2, 0.6, 0.002
    x = rng.normal(size=(n, 2))
    mom = np.zeros((n, 6))
    mom[:, 0] = rng.choice([-1, 1], n) * (0.5 + rng.random(n))
    mom[:, 3:] = rng.normal(size=(n, 3)) * 0.01
    T = 0.4
    xe, me, t, acc, rej = dopri5(x, mom, 0.0, T, 0.01, order, lam0, nu, rtol=1e-10, atol=1e-10)

    def f(t, y):
        dx, dm = rhs_regrouped(y[:2 * n].reshape(n, 2), y[2 * n:].reshape(n, 6), t, order,
                               lam0, nu)
        return np.concatenate([dx.ravel(), dm.ravel()])

    sol = solve_ivp(f, (0.0, T), np.concatenate([x.ravel(), mom.ravel()]), method="RK45",
                    rtol=1e-10, atol=1e-10)
    ys = sol.y[:, -1]
    assert np.abs(xe.ravel() - ys[:2 * n]).max() < 1e-8
    assert np.abs(me.ravel() - ys[2 * n:]).max() < 1e-8


def test_step_count_scales_like_a_fifth_order_method():
    x, mom = _pair(1.0, 1.0, 1.0)
    steps = []
    for tol in (1e-6, 1e-11):
        *_, acc, rej = dopri5(x, mom, 0.0, 20.0, 0.01, 0, 0.4, 0.0, rtol=tol, atol=tol)
        steps.append(acc)
    ratio = steps[1] / steps[0]
    assert 6.0 < ratio < 16.0  # 10 = (1e5)^(1/5)
