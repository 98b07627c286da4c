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
