"""Adaptive Dormand-Prince 5(4) integration of the MMVM moment ODE (oracle, FP64).

Test infrastructure only (see ``oracle/__init__.py``).

The paper integrates the moment system with an adaptive embedded
Runge-Kutta pair at relative and absolute tolerance 1e-8 (Section 4.3).
This is the Dormand-Prince 5(4) pair (the published tableau, first same as
last), with the state y = (x, M) flattened and lambda evaluated at every
stage time (eq:phi00):

* error of a step: e = h sum_i (b_i - b*_i) k_i; its size
  err = max_i |e_i| / (atol + rtol max(|y_i|, |y5_i|))  (a max norm);
* the step is kept when err <= 1; either way the next step size is
  h min(5, max(0.2, 0.9 err^(-1/5))) (at most h after a rejection);
* the last step is shortened to land on t_end.
"""
from __future__ import annotations

import numpy as np

from .rhs import rhs_regrouped

# Dormand-Prince 5(4): nodes, stage weights, 5th- and 4th-order weights
C = (0.0, 1 / 5, 3 / 10, 4 / 5, 8 / 9, 1.0, 1.0)
A = (
    (),
    (1 / 5,),
    (3 / 40, 9 / 40),
    (44 / 45, -56 / 15, 32 / 9),
    (19372 / 6561, -25360 / 2187, 64448 / 6561, -212 / 729),
    (9017 / 3168, -355 / 33, 46732 / 5247, 49 / 176, -5103 / 18656),
    (35 / 384, 0.0, 500 / 1113, 125 / 192, -2187 / 6784, 11 / 84),
)
B5 = (35 / 384, 0.0, 500 / 1113, 125 / 192, -2187 / 6784, 11 / 84, 0.0)
B4 = (5179 / 57600, 0.0, 7571 / 16695, 393 / 640, -92097 / 339200, 187 / 2100, 1 / 40)


def dopri5(x, mom, t0, t_end, h0, order, lam0, nu, rtol=1e-8, atol=1e-8, max_steps=100000,
           rhs=rhs_regrouped):
    """Integrate (x, mom) from t0 to t_end; returns (x, mom, t, accepted, rejected)."""
    x = np.array(x, dtype=np.float64)
    mom = np.array(mom, dtype=np.float64)
    n, K = mom.shape
    split = 2 * n

    def f(t, y):
        dx, dm = rhs(y[:split].reshape(n, 2), y[split:].reshape(n, K), t, order, lam0, nu)
        return np.concatenate([dx.ravel(), dm.ravel()])

    y = np.concatenate([x.ravel(), mom.ravel()])
    t, h = t0, h0
    k1 = f(t, y)
    accepted = rejected = 0
    while t < t_end and accepted + rejected < max_steps:
        last = t + h >= t_end
        if last:
            h = t_end - t
        ks = [k1]
        for s in range(1, 7):
            ys = y + h * sum(a * k for a, k in zip(A[s], ks))
            ks.append(f(t + C[s] * h, ys))
        y5 = y + h * sum(b * k for b, k in zip(B5, ks))  # equals the last stage state
        e = h * sum((b5 - b4) * k for b5, b4, k in zip(B5, B4, ks))
        sc = atol + rtol * np.maximum(np.abs(y), np.abs(y5))
        err = float(np.max(np.abs(e) / sc))
        fac = 0.9 * err ** (-0.2) if err > 0.0 else 5.0
        if err <= 1.0:
            t = t_end if last else t + h
            y = y5
            k1 = ks[6]  # first same as last
            accepted += 1
            h = h * min(5.0, max(0.2, fac))
        else:
            rejected += 1
            h = h * min(1.0, max(0.2, fac))
    return y[:split].reshape(n, 2), y[split:].reshape(n, K), t, accepted, rejected
