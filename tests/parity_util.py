"""Error norms shared by the GPU parity tests.

Moments are compared in the weighted norm of the convergence theorem of
Section 2.1.1 (weighted enstrophy E = int phi_00^{-1} omega^2): for one particle
||M||_w^2 = sum_k w_k M_k^2 with w_k = 2^{|k|} k1! k2! / lambda^{2|k|}, which is
(up to a constant) E of the Hermite expansion, since the Hermite functions are
orthogonal in that norm.
"""
import math

import numpy as np


def weights(order: int, lam: float) -> np.ndarray:
    w = []
    for n in range(order + 1):
        for k2 in range(n + 1):
            k1 = n - k2
            w.append(2.0 ** n * math.factorial(k1) * math.factorial(k2) / lam ** (2 * n))
    return np.array(w)


def wnorm(M: np.ndarray, order: int, lam: float) -> np.ndarray:
    """Per-particle weighted norm of an (n, K) moment array."""
    return np.sqrt((np.atleast_2d(M) ** 2 * weights(order, lam)[None, :]).sum(1))


def rhs_error(dM, dM_ref, order, lam):
    """max_j ||dM^j - dM_ref^j||_w / max_j ||dM_ref^j||_w."""
    return float(wnorm(dM - dM_ref, order, lam).max() / wnorm(dM_ref, order, lam).max())


def state_error(M, M_ref, order, lam):
    """max_j ||M^j - M_ref^j||_w / ||M_ref^j||_w (per particle relative)."""
    return float((wnorm(M - M_ref, order, lam) / wnorm(M_ref, order, lam)).max())


def vel_error(dx, dx_ref):
    return float(np.abs(dx - dx_ref).max() / np.abs(dx_ref).max())


def single_particle_condition(moments_row, order, lam):
    """Weighted condition number of the single-particle moment equation.

    kappa_w = ||sum_terms |term| ||_w / ||dM||_w over the terms of the
    regrouped self term (oracle/rhs.py).  Any FP64 evaluation has errors up to
    ~eps * kappa_w in the weighted norm; kappa_w grows like 2^n n! with the
    order (about 6, 14, 250, 5e3, 6e4 for M = 2, 4, 6, 8, 10 on the test
    states), which is why the FP64 tolerance is max(1e-12, 2 eps kappa_w).
    """
    from oracle.rhs import _finish_terms, self_velocity_jets

    m = np.atleast_2d(moments_row)
    S1, S2 = self_velocity_jets(m, lam, order)
    W = (S1[0], S2[0])
    ks, ls, cs, comps, offs = _finish_terms(order, lam)
    K = m.shape[1]
    absum = np.zeros(K)
    res = np.zeros(K)
    for k, l, c, comp, o in zip(ks, ls, cs, comps, offs):
        v = c * m[0, l] * W[comp][o]
        absum[k] += abs(v)
        res[k] += v
    return float(wnorm(absum, order, lam)[0] / wnorm(res, order, lam)[0])


def fp64_tolerance(kappa: float) -> float:
    return max(1e-12, 2.0 * 2.220446049250313e-16 * kappa)
