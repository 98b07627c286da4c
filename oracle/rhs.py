"""Right-hand side and RK4 of the multi-moment vortex method (oracle, FP64).

Test infrastructure only (see ``oracle/__init__.py``).

State: centres x (n, 2) and moments M (n, K) (column order of
``coefficients.idx``), a shared core lambda(t)^2 = lambda_0^2 + 4 nu t
(eq:phi00).  The viscous term has no separate piece in these variables: it
is carried entirely by the core spreading lambda(t) (the cancellation noted
after eq:Galerkin), so the moment ODE is the purely quadratic system

    dM^j_k/dt = A(k) + B(k) + C(k)                          (eq:Final_CrossCoef)
    A(k) = c_k sum_{l,m} M^j_l M^j_m Gamma-tilde[k,l,m]           (self vortex)
    B(k) = c_k sum_{j' != j} sum_{l,m} M^j_l M^{j'}_m Gamma_B[k,l,m; s_jj']
    C(k) = xdot^j_1 M^j[k1-1,k2] + xdot^j_2 M^j[k1,k2-1]   (eq:last_termsimp)
    xdot^j = (1/M^j_00) sum_{j' != j} sum_{l,m} M^{j'}_l M^j_m (-1)^{|m|}
             H^B(l+m; s_jj')                                 (eq:xjdot_Final)

with s_jj' = x^j - x^{j'} and Gamma_B = Gamma^I + Gamma^II with H_1, H_2
replaced by the pair kernel H^B_1, H^B_2 at s_jj' (eq:FinalCrossI/II).  See
the package docstring for the readings of the printed labels.

Two evaluations are provided:

* ``rhs_literal`` builds the coefficient tensors Gamma-tilde and Gamma_B
  term by term exactly as printed and contracts them with the moments
  (small orders and particle counts only).
* ``rhs_regrouped`` sums over the velocity index m first,
  W_c[gamma] = sum_{j'} sum_m M^{j'}_m H^B_c(m + gamma; s_jj'), then applies
  the (i, q) sums of eq:FinalSingleI/II to W.  Because every H argument in
  Gamma^I/II is m plus an offset that does not depend on m, this is the same
  finite sum in a different order (the paper's own intermediate form,
  Appendix A.1, before the Gaussian self-convolution is substituted).  It is
  cross-checked against ``rhs_literal`` in the tests and is the form used for
  large problems (and for a subset of target rows against all sources).
"""
from __future__ import annotations

import math
from functools import lru_cache

import numpy as np

from .coefficients import (c_k, gamma_I_terms, gamma_II_terms, gamma_tensor, idx,
                           jet_table_at_zero, multi_indices, n_moments, self_tensor)
from .pair_jet import pair_jet


def lam_at(t: float, lam0: float, nu: float) -> float:
    """Core size at time t: lambda^2 = lambda_0^2 + 4 nu t (eq:phi00)."""
    return math.sqrt(lam0 * lam0 + 4.0 * nu * t)


def _transport(xdot: np.ndarray, mom: np.ndarray, order: int) -> np.ndarray:
    """C(k) = xdot_1 M[k1-1, k2] + xdot_2 M[k1, k2-1] (eq:last_termsimp)."""
    out = np.zeros_like(mom)
    for col, (k1, k2) in enumerate(multi_indices(order)):
        if k1 >= 1:
            out[:, col] += xdot[:, 0] * mom[:, idx(k1 - 1, k2)]
        if k2 >= 1:
            out[:, col] += xdot[:, 1] * mom[:, idx(k1, k2 - 1)]
    return out


def rhs_literal(x, mom, t, order, lam0, nu):
    """Literal A + B + C with explicit Gamma-tilde and Gamma_B tensors.

    Returns (dxdt (n,2), dMdt (n,K)).  Cost ~ n^2 K^3; for tests only.
    """
    x = np.asarray(x, dtype=np.float64)
    mom = np.asarray(mom, dtype=np.float64)
    n = x.shape[0]
    lam = lam_at(t, lam0, nu)
    P = max(3 * order - 1, 0)
    mi = multi_indices(order)
    sgn_m = np.array([(-1.0) ** (a + b) for a, b in mi])
    T_self = self_tensor(order, lam)
    dM = np.einsum("klm,jl,jm->jk", T_self, mom, mom)          # A
    xdot = np.zeros((n, 2))
    for j in range(n):
        for jp in range(n):
            if jp == j:
                continue
            s = x[j] - x[jp]
            J1, J2 = pair_jet(s[None, :], P, lam)
            J1 = J1[0]
            J2 = J2[0]
            T_B = gamma_tensor(order, lam, J1, J2)
            dM[j] += np.einsum("klm,l,m->k", T_B, mom[j], mom[jp])  # B
            # eq:xjdot_Final: sum_{l (source), m (target)} M^{j'}_l M^j_m (-1)^{|m|} H^B(l+m)
            for li, (l1, l2) in enumerate(mi):
                for mj, (m1, m2) in enumerate(mi):
                    col = idx(l1 + m1, l2 + m2)
                    w = mom[jp, li] * mom[j, mj] * sgn_m[mj]
                    xdot[j, 0] += w * J1[col]
                    xdot[j, 1] += w * J2[col]
        xdot[j] /= mom[j, 0]
    dM += _transport(xdot, mom, order)                          # C
    return xdot, dM


@lru_cache(maxsize=16)
def _finish_terms_unit(order: int):
    """(k, l, coef at lambda = 1, lambda power, comp, offset column) of the (i,q) sums.

    Every term of c_k * Gamma^I/II (eq:coefficient, eq:FinalSingleI/II) is a
    power of lambda times a number: c_k ~ lambda^{2|k|}, the bracketed ratios
    ~ lambda^{-2(i+1)-2q} (I) or lambda^{-2i-2(q+1)} (II); both give
    lambda^{2|k| - 2(i+q+1)}.
    """
    ks, ls, cs, pw, comps, offs = [], [], [], [], [], []
    for ki, (k1, k2) in enumerate(multi_indices(order)):
        ck = c_k(k1, k2, 1.0)
        for li, (l1, l2) in enumerate(multi_indices(order)):
            for comp, terms in ((0, gamma_I_terms(k1, k2, l1, l2, 1.0)),
                                (1, gamma_II_terms(k1, k2, l1, l2, 1.0))):
                for coef, (o1, o2) in terms:
                    # offset o = k + l - 2(i+q) - 1 in total order
                    iq1 = (k1 + k2 + l1 + l2 - (o1 + o2) - 1) // 2 + 1
                    ks.append(ki)
                    ls.append(li)
                    cs.append(ck * coef)
                    pw.append(2 * (k1 + k2) - 2 * iq1)
                    comps.append(comp)
                    offs.append(idx(o1, o2))
    return (np.array(ks, dtype=np.int64), np.array(ls, dtype=np.int64), np.array(cs),
            np.array(pw, dtype=np.int64), np.array(comps, dtype=np.int64),
            np.array(offs, dtype=np.int64))


def _finish_terms(order: int, lam: float):
    """(k, l, coef, comp, offset-column) of the (i,q) sums at core size lambda,
    with c_k folded in: dM_k gets sum_l M_l sum_terms coef * W_comp[offset]."""
    ks, ls, cs, pw, comps, offs = _finish_terms_unit(order)
    return ks, ls, cs * lam ** pw.astype(np.float64), comps, offs


@lru_cache(maxsize=16)
def _shift_index(order: int):
    """G[gamma, m] = column of m + gamma for |gamma| <= 2M-1, |m| <= M."""
    gam = multi_indices(max(2 * order - 1, 0))
    mi = multi_indices(order)
    return np.array([[idx(g1 + m1, g2 + m2) for (m1, m2) in mi] for (g1, g2) in gam],
                    dtype=np.int64)


def velocity_jets(x, mom, lam, order, rows, exclude_self=True, chunk=32):
    """W_c[j, gamma] = sum_{j' != j} sum_m M^{j'}_m H^B_c(m+gamma; x^j - x^{j'}).

    For the target rows ``rows`` against every source.  Returns (W1, W2), each
    (len(rows), n_gamma) with |gamma| <= 2M-1.
    """
    n = x.shape[0]
    P = max(3 * order - 1, 0)
    G = _shift_index(order)
    rows = np.asarray(rows)
    W1 = np.zeros((rows.size, G.shape[0]))
    W2 = np.zeros((rows.size, G.shape[0]))
    for start in range(0, rows.size, chunk):
        rr = rows[start:start + chunk]
        s = (x[rr][:, None, :] - x[None, :, :]).reshape(-1, 2)
        J1, J2 = pair_jet(s, P, lam)
        J1 = J1.reshape(rr.size, n, -1)
        J2 = J2.reshape(rr.size, n, -1)
        if exclude_self:
            for a, j in enumerate(rr):
                J1[a, j] = 0.0
                J2[a, j] = 0.0
        W1[start:start + rr.size] = _contract(J1, G, mom)
        W2[start:start + rr.size] = _contract(J2, G, mom)
    return W1, W2


def _contract(J: np.ndarray, G: np.ndarray, mom: np.ndarray) -> np.ndarray:
    """sum_{j', m} M^{j'}_m J[row, j', G[gamma, m]] -> (rows, n_gamma)."""
    out = np.zeros((J.shape[0], G.shape[0]))
    for mcol in range(G.shape[1]):
        # J[:, :, G[:, mcol]] is (rows, n, n_gamma); weight by M^{j'}_m
        out += np.einsum("rng,n->rg", J[:, :, G[:, mcol]], mom[:, mcol])
    return out


def self_velocity_jets(mom, lam, order):
    """W_c[j, gamma] = sum_m M^j_m H_c(m + gamma): the s = 0 (self) kernel."""
    P = max(3 * order - 1, 0)
    H1t, H2t = jet_table_at_zero(P, lam)
    G = _shift_index(order)
    return mom @ H1t[G].T, mom @ H2t[G].T


def rhs_regrouped(x, mom, t, order, lam0, nu, rows=None):
    """A + B + C through the velocity jet W (see module docstring).

    ``rows`` selects target particles (all sources are always used); returns
    (dxdt, dMdt) for those rows only.
    """
    x = np.asarray(x, dtype=np.float64)
    mom = np.asarray(mom, dtype=np.float64)
    n = x.shape[0]
    rows = np.arange(n) if rows is None else np.asarray(rows)
    lam = lam_at(t, lam0, nu)
    mi = multi_indices(order)
    sgn_m = np.array([(-1.0) ** (a + b) for a, b in mi])
    K = len(mi)
    if n > 1:
        W1x, W2x = velocity_jets(x, mom, lam, order, rows)
    else:
        W1x = np.zeros((rows.size, _shift_index(order).shape[0]))
        W2x = np.zeros_like(W1x)
    # eq:xjdot_Final: xdot^j = (1/M^j_00) sum_m (-1)^{|m|} M^j_m W^excl[m] (|m| <= M)
    mt = mom[rows]
    xdot = np.stack([(mt * sgn_m[None, :] * W1x[:, :K]).sum(1),
                     (mt * sgn_m[None, :] * W2x[:, :K]).sum(1)], axis=1) / mt[:, :1]
    S1, S2 = self_velocity_jets(mt, lam, order)
    W = np.stack([W1x + S1, W2x + S2], axis=0)                 # (2, rows, n_gamma)
    ks, ls, cs, comps, offs = _finish_terms(order, lam)
    contrib = cs[None, :] * mt[:, ls] * W[comps, :, offs].T    # (rows, terms)
    dM = np.zeros((rows.size, K))
    np.add.at(dM.T, ks, contrib.T)
    dM += _transport(xdot, mt, order)
    return xdot, dM


def rk4(x, mom, t, dt, nsteps, order, lam0, nu, rhs=rhs_regrouped):
    """Classic fourth-order Runge-Kutta on (x, M); lambda evaluated at stage times."""
    x = np.array(x, dtype=np.float64)
    mom = np.array(mom, dtype=np.float64)
    for _ in range(nsteps):
        k1x, k1m = rhs(x, mom, t, order, lam0, nu)
        k2x, k2m = rhs(x + 0.5 * dt * k1x, mom + 0.5 * dt * k1m, t + 0.5 * dt, order, lam0, nu)
        k3x, k3m = rhs(x + 0.5 * dt * k2x, mom + 0.5 * dt * k2m, t + 0.5 * dt, order, lam0, nu)
        k4x, k4m = rhs(x + dt * k3x, mom + dt * k3m, t + dt, order, lam0, nu)
        x = x + dt / 6.0 * (k1x + 2.0 * k2x + 2.0 * k3x + k4x)
        mom = mom + dt / 6.0 * (k1m + 2.0 * k2m + 2.0 * k3m + k4m)
        t = t + dt
    return x, mom, t


def self_rhs_rows(mom_row, lam, order, krows):
    """dM_k of a single particle (eq:moment_evolutionFinish: A(k) alone, no
    other particle, no centroid motion) for the moment rows ``krows`` only,
    with the absolute size of what is summed.

    For each k: sum_l M_l sum_{(i,q)} c_k coef_{I/II}(k,l,i,q) W_c[offset]
    (the (i,q) terms of eq:FinalSingleI/II), with the velocity jet
    W_c[gamma] = sum_m M_m H_c(m + gamma) (the paper's regrouped form; H_1, H_2
    are the exact closed forms of Appendix A.1).  Rows are independent, so a
    sample of them checks a high-order evaluation whose full term list
    (about M^6 / 50 terms) would not fit in memory.

    Returns (values, abs_sums): abs_sums[r] = sum over the same terms of
    |c_k coef M_l| * sum_m |M_m H_c(m + offset)|, the scale against which the
    rounding of any evaluation of that row is measured.
    """
    mom_row = np.asarray(mom_row, dtype=np.float64)
    P = max(3 * order - 1, 0)
    H1t, H2t = jet_table_at_zero(P, lam)
    G = _shift_index(order)
    W = (H1t[G] @ mom_row, H2t[G] @ mom_row)
    Wabs = (np.abs(H1t[G]) @ np.abs(mom_row), np.abs(H2t[G]) @ np.abs(mom_row))
    mi = multi_indices(order)
    vals, sums = [], []
    for kc in krows:
        k1, k2 = mi[kc]
        ck = c_k(k1, k2, lam)
        tot = 0.0
        ab = 0.0
        for lc, (l1, l2) in enumerate(mi):
            ml = mom_row[lc]
            if ml == 0.0:
                continue
            for comp, terms in ((0, gamma_I_terms(k1, k2, l1, l2, lam)),
                                (1, gamma_II_terms(k1, k2, l1, l2, lam))):
                for coef, (o1, o2) in terms:
                    g = idx(o1, o2)
                    f = ck * coef * ml
                    tot += f * W[comp][g]
                    ab += abs(f) * Wabs[comp][g]
        vals.append(tot)
        sums.append(ab)
    return np.array(vals), np.array(sums)
