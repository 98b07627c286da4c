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


# ---------------------------------------------------------------------------
# Per-particle norms (the error norm reading of the convergence theorem,
# Section 2.1.1: relative error per particle, maximum over particles)

ROW_FLOOR = 1e-3


def rhs_error_rows(dM, dM_ref, order, lam, floor=ROW_FLOOR):
    """max_j ||dM^j - dM_ref^j||_w / max(||dM_ref^j||_w, floor * max_k ||dM_ref^k||_w).

    Every particle is judged against its own right-hand side in the weighted
    norm; a row whose own right-hand side is below `floor` times the largest
    row of the sample is judged against that floor (its absolute error must
    stay below tol * floor * the largest row), so a vanishing row does not
    divide by zero.
    """
    num = wnorm(dM - dM_ref, order, lam)
    den = wnorm(dM_ref, order, lam)
    return float((num / np.maximum(den, floor * den.max())).max())


def vel_error_rows(dx, dx_ref, floor=ROW_FLOOR):
    """max_j |dx^j - dx_ref^j| / max(|dx_ref^j|, floor * max_k |dx_ref^k|)
    (Euclidean norm of the velocity of each particle)."""
    num = np.linalg.norm(np.atleast_2d(dx - dx_ref), axis=1)
    den = np.linalg.norm(np.atleast_2d(dx_ref), axis=1)
    return float((num / np.maximum(den, floor * den.max())).max())


def position_error(x, x_ref, lam):
    """max_j |x^j - x_ref^j| / lambda (centroid error in core sizes)."""
    return float(np.linalg.norm(np.atleast_2d(x - x_ref), axis=1).max() / lam)


# ---------------------------------------------------------------------------
# Rows where the all-pairs kernel switches path.  The library orders the
# centres along a Morton curve (keys of 16 bits per axis over the bounding
# box, stable sort) and decides near / far / tile expansion per pair of
# 32-particle groups from the boxes of the normalised centres
# zeta = x / sqrt(2 lambda^2) (FP32 hi parts).  The helpers below redo that
# bookkeeping on the host (selection only: no arithmetic of the method) so a
# test can aim its sampled rows at the groups where the switches happen.

X_FAR = (20.0, 32.0, 40.0, 50.0, 58.0, 66.0, 74.0, 80.0, 88.0)  # per order 0..8
M2P_THETA2 = 0.01


def _spread16(v):
    v = v.astype(np.uint64) & 0xFFFF
    v = (v | (v << 8)) & 0x00FF00FF
    v = (v | (v << 4)) & 0x0F0F0F0F
    v = (v | (v << 2)) & 0x33333333
    v = (v | (v << 1)) & 0x55555555
    return v


def morton_order(x):
    """Sorted position -> particle, as the library orders the centres."""
    lo = x.min(0)
    s = np.maximum(x.max(0) - lo, 1e-300)
    q = (np.clip((x - lo) / s, 0.0, 1.0) * 65535.0).astype(np.uint64)
    keys = _spread16(q[:, 0]) | (_spread16(q[:, 1]) << 1)
    return np.argsort(keys, kind="stable")


def group_geometry(x, lam, group=32):
    """(perm, boxes (G, 4) = (min1, max1, min2, max2), centres (G, 2),
    radii (G,)) of the sorted groups in normalised units."""
    perm = morton_order(x)
    z = (x[perm] / math.sqrt(2.0 * lam * lam)).astype(np.float32).astype(np.float64)
    G = (len(z) + group - 1) // group
    boxes = np.zeros((G, 4))
    cen = np.zeros((G, 2))
    rad = np.zeros(G)
    for g in range(G):
        zz = z[g * group:(g + 1) * group]
        boxes[g] = (zz[:, 0].min(), zz[:, 0].max(), zz[:, 1].min(), zz[:, 1].max())
        cen[g] = (0.5 * (boxes[g, 0] + boxes[g, 1]), 0.5 * (boxes[g, 2] + boxes[g, 3]))
        rad[g] = np.sqrt(((zz - cen[g]) ** 2).sum(1).max())
    return perm, boxes, cen, rad


def switch_rows(x, moments, order, lam, per_kind=8, seed=0):
    """Target rows aimed at the kernel's path switches (dict kind -> rows):

    * ``x_far_band``: groups with the most source groups whose box distance
      lies within 10 % of the near/far threshold x_far(M);
    * ``m2p_band``: groups with the most source groups just inside the tile
      expansion criterion (radius / distance between 0.09 and 0.1);
    * ``loose_box``: the groups with the largest boxes (the most sources of
      near tiles taken as far one by one);
    * ``small_circulation``: the smallest |M_00|.
    """
    rng = np.random.default_rng(seed)
    perm, boxes, cen, rad = group_geometry(x, lam)
    xf = X_FAR[order]
    G = boxes.shape[0]
    band = np.zeros(G, dtype=np.int64)
    m2p = np.zeros(G, dtype=np.int64)
    for t0 in range(0, G, 256):  # target groups in blocks (memory stays O(256 G))
        tb = boxes[t0:t0 + 256]
        dx = np.maximum(0.0, np.maximum(tb[:, None, 0] - boxes[None, :, 1],
                                        boxes[None, :, 0] - tb[:, None, 1]))
        dy = np.maximum(0.0, np.maximum(tb[:, None, 2] - boxes[None, :, 3],
                                        boxes[None, :, 2] - tb[:, None, 3]))
        d2 = dx * dx + dy * dy
        band[t0:t0 + 256] = ((d2 >= 0.9 * xf) & (d2 < 1.1 * xf)).sum(1)
        # distance from each target box to each source centre
        cx = np.maximum(0.0, np.maximum(tb[:, None, 0] - cen[None, :, 0],
                                        cen[None, :, 0] - tb[:, None, 1]))
        cy = np.maximum(0.0, np.maximum(tb[:, None, 2] - cen[None, :, 1],
                                        cen[None, :, 1] - tb[:, None, 3]))
        c2 = np.maximum(cx * cx + cy * cy, 1e-300)
        ratio2 = rad[None, :] ** 2 / c2
        m2p[t0:t0 + 256] = ((d2 >= xf) & (ratio2 <= M2P_THETA2)
                            & (ratio2 >= 0.81 * M2P_THETA2)).sum(1)
    size = (boxes[:, 1] - boxes[:, 0]) ** 2 + (boxes[:, 3] - boxes[:, 2]) ** 2
    n = x.shape[0]

    def rows_of(groups):
        out = []
        for g in groups:
            members = perm[g * 32:(g + 1) * 32]
            out.append(int(rng.choice(members)))
            if len(out) == per_kind:
                break
        return out

    return {
        "x_far_band": rows_of(np.argsort(-band, kind="stable")),
        "m2p_band": rows_of(np.argsort(-m2p, kind="stable")),
        "loose_box": rows_of(np.argsort(-size, kind="stable")),
        "small_circulation": [int(j) for j in np.argsort(np.abs(moments[:, 0]),
                                                         kind="stable")[:per_kind]],
        "last_partial_group": [int(j) for j in perm[((n - 1) // 32) * 32:]][:per_kind],
    }


# ---------------------------------------------------------------------------
# The oracle on many target rows, one single-threaded process per host core
# (rows are independent).  A spawn pool: no child inherits a CUDA context.

def _oracle_rows_child(args):
    x, mom, t, order, lam0, nu, rows = args
    from oracle.rhs import rhs_regrouped

    return rhs_regrouped(x, mom, t, order, lam0, nu, rows=rows)


def oracle_rows_parallel(x, mom, t, order, lam0, nu, rows, procs=None):
    """rhs_regrouped on `rows` (all sources), split over a spawn pool."""
    import multiprocessing as mp
    import os

    rows = np.asarray(rows)
    procs = max(1, min(procs or os.cpu_count() or 1, rows.size))
    if procs == 1:
        return _oracle_rows_child((x, mom, t, order, lam0, nu, rows))
    parts = np.array_split(rows, procs)
    with mp.get_context("spawn").Pool(procs) as pool:
        res = pool.map(_oracle_rows_child,
                       [(x, mom, t, order, lam0, nu, p) for p in parts if p.size])
    return np.concatenate([r[0] for r in res]), np.concatenate([r[1] for r in res])


# ---------------------------------------------------------------------------
# Per-particle scale of what a right-hand side sums.  A particle whose
# velocity or moment rate is the small difference of large pair terms cannot
# be evaluated to a relative accuracy better than the rounding of those terms
# (FP32: the jet of order n carries ~2 n u, u = 2^-24, of each term, up to
# ~3e-6 at n = 3M = 24); the absolute scale S_j below is the sum of the
# magnitudes of the pair terms (and of the self term), S_j >= |value_j|.
# The mixed-precision tests hold |error_j| / max(|value_j|, theta S_j) with
# theta = 1, i.e. each particle's error relative to its own rounding scale:
# for a particle whose sum does not cancel (S_j ~ |value_j|) this is its
# plain relative error.

def _abs_scale_rows_chunk(args):
    x, mom, t, order, lam0, nu, rows = args
    from oracle.coefficients import multi_indices
    from oracle.pair_jet import pair_jet
    from oracle.rhs import _finish_terms, _shift_index, lam_at, rhs_regrouped, self_velocity_jets

    lam = lam_at(t, lam0, nu)
    P = max(3 * order - 1, 0)
    G = _shift_index(order)
    mi = multi_indices(order)
    K = len(mi)
    n = x.shape[0]
    rows = np.asarray(rows)
    Wabs = np.zeros((2, rows.size, G.shape[0]))
    for a, j in enumerate(rows):
        s = x[j][None, :] - x
        J1, J2 = pair_jet(s, P, lam)
        for c, J in enumerate((J1, J2)):
            w = np.zeros((n, G.shape[0]))
            for m in range(K):
                w += J[:, G[:, m]] * mom[:, m][:, None]
            w[j] = 0.0  # the self pair: its own term below
            Wabs[c, a] = np.abs(w).sum(0)
    mt = mom[rows]
    S1, S2 = self_velocity_jets(mt, lam, order)
    Sabs = (np.abs(S1), np.abs(S2))
    # velocity: (1/M00) sum_m |M_m| |W_c[m]|, |m| <= M
    sx = np.stack([(np.abs(mt) * Wabs[0][:, :K]).sum(1), (np.abs(mt) * Wabs[1][:, :K]).sum(1)],
                  axis=1) / np.abs(mt[:, :1])
    # moments: |c coef M_l| (|W| + |W_self|) over the (i, q) terms, plus the transport terms
    xdot, _ = rhs_regrouped(x, mom, t, order, lam0, nu, rows=rows)
    ks, ls, cs, comps, offs = _finish_terms(order, lam)
    Wtot = np.stack([Wabs[0] + Sabs[0], Wabs[1] + Sabs[1]], axis=0)
    contrib = np.abs(cs[None, :] * mt[:, ls]) * Wtot[comps, :, offs].T
    sM = np.zeros((rows.size, K))
    np.add.at(sM.T, ks, contrib.T)
    for col, (k1, k2) in enumerate(mi):
        if k1 >= 1:
            sM[:, col] += np.abs(xdot[:, 0] * mt[:, mi.index((k1 - 1, k2))])
        if k2 >= 1:
            sM[:, col] += np.abs(xdot[:, 1] * mt[:, mi.index((k1, k2 - 1))])
    return np.linalg.norm(sx, axis=1), sM


def abs_scale_rows(x, mom, t, order, lam0, nu, rows, procs=None):
    """(sx (rows,), sM (rows, K)): per target row the sum of the magnitudes of
    the pair terms of its centroid velocity (Euclidean over the two
    components) and of its moment right-hand side (per moment), built from
    the oracle's pair jet; one spawn process per host core."""
    import multiprocessing as mp
    import os

    x = np.asarray(x, dtype=np.float64)
    mom = np.asarray(mom, dtype=np.float64)
    rows = np.asarray(rows)
    procs = max(1, min(procs or os.cpu_count() or 1, rows.size))
    if procs == 1:
        return _abs_scale_rows_chunk((x, mom, t, order, lam0, nu, rows))
    parts = [p for p in np.array_split(rows, procs) if p.size]
    with mp.get_context("spawn").Pool(procs) as pool:
        res = pool.map(_abs_scale_rows_chunk, [(x, mom, t, order, lam0, nu, p) for p in parts])
    return np.concatenate([r[0] for r in res]), np.concatenate([r[1] for r in res])


COND_THETA = 1.0


def vel_error_cond(dx, dx_ref, sx, theta=COND_THETA):
    """max_j |dx^j - dx_ref^j| / max(|dx_ref^j|, theta sx^j)."""
    num = np.linalg.norm(np.atleast_2d(dx - dx_ref), axis=1)
    den = np.linalg.norm(np.atleast_2d(dx_ref), axis=1)
    return float((num / np.maximum(den, theta * sx)).max())


def rhs_error_cond(dM, dM_ref, sM, order, lam, theta=COND_THETA):
    """max_j ||dM^j - dM_ref^j||_w / max(||dM_ref^j||_w, theta ||sM^j||_w)."""
    num = wnorm(dM - dM_ref, order, lam)
    den = wnorm(dM_ref, order, lam)
    return float((num / np.maximum(den, theta * wnorm(sM, order, lam))).max())


def cond_errors(gx, gM, ox, oM, x, mom, t, order, lam0, nu, rows, theta=COND_THETA, procs=None):
    """(velocity, moment) per-particle errors of sampled rows (gx, gM: the
    rows under test; ox, oM: their references) in the conditioning-aware
    norms above, with the scales of the oracle's pair terms."""
    from oracle.rhs import lam_at

    sx, sM = abs_scale_rows(x, mom, t, order, lam0, nu, rows, procs)
    lam = lam_at(t, lam0, nu)
    ev = vel_error_cond(gx, ox, sx, theta)
    em = rhs_error_cond(gM, oM, sM, order, lam, theta) if order >= 1 else 0.0
    return ev, em
