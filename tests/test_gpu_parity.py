"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Tolerances (derived in the design notes):
* FP64 mode: 1e-12 relative (weighted moment norm / velocity max norm) for a
  single right-hand side and after RK4 steps; where the weighted condition
  number of the moment equation kappa_w exceeds ~2e3 (single particle,
  M = 10) no FP64 evaluation can promise that, and the tolerance is
  2 eps kappa_w.
* Mixed FP32 mode: 5e-6 relative for a single right-hand side (rounding
  accumulated along the order-n recurrences of the jet, ~2 n u with n <= 3M
  and u = 2^-24, plus the tile sums); 1e-5 relative on moments after 100 RK4
  steps.
Every multi-particle error is per particle (the weighted norm of the
convergence theorem, Section 2.1.1, for the moments; the Euclidean norm for
the centroid velocity), maximum over particles.  FP64 results are held
relative to each particle's own value (floored at 1e-3 of the largest row);
mixed results relative to the particle's own rounding scale, the summed
magnitudes of its pair terms (a particle whose velocity is the small
difference of large pair terms cannot be evaluated in FP32 to better than
the rounding of those terms), computed from the oracle's pair jet
(tests/parity_util.py, cond_errors).
Sizes span several CTA tiles of targets and sources and end in ragged tails;
at the full benchmark sizes a sample of target rows is checked against the
oracle's sum over every source.
"""
import math

import numpy as np
import pytest

import mmvm_inputs
from oracle.rhs import lam_at, rhs_literal, rhs_regrouped, rk4
from tests.parity_util import (COND_THETA, cond_errors, fp64_tolerance, oracle_rows_parallel,
                               position_error, rhs_error, rhs_error_rows,
                               single_particle_condition, state_error, switch_rows, vel_error,
                               vel_error_rows)

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12
MIXED_RHS_TOL = 5e-6


def mixed_rhs_tol(order: int) -> float:
    """Single right-hand side, mixed precision: 5e-6 up to order 6; above,
    the FP32 rounding carried by the jet grows with its order n <= 3M
    (~2 n u per entry, u = 2^-24), so the bound grows in proportion to M."""
    return MIXED_RHS_TOL * max(1.0, order / 6.0)


@pytest.fixture(scope="module")
def mm():
    import paper_1010_2475_gb300 as mm

    mm.load_library()
    return mm


def _gpu_rhs(mm, wl, t, prec):
    with mm.Context(wl.order, wl.lam0, wl.nu, prec) as ctx:
        ctx.set_state(wl.x, wl.moments, t)
        return ctx.rhs()


@pytest.mark.parametrize("order", [0, 2, 4, 6, 10])
def test_single_particle_rhs_fp64(mm, order):
    wl = mmvm_inputs.single_quadrupole(order=order, eps=0.1, sigma0=1.0)
    rng = np.random.default_rng(order)
    wl.moments[0, 3:] += rng.normal(size=wl.K - 3) * 0.02 if wl.K > 3 else 0.0
    ox, oM = rhs_regrouped(wl.x, wl.moments, 1.5, order, wl.lam0, wl.nu)
    gx, gM = _gpu_rhs(mm, wl, 1.5, mm.MMVM_FP64)
    assert np.all(gx == 0.0)
    lam = lam_at(1.5, wl.lam0, wl.nu)
    if order >= 2:
        tol = fp64_tolerance(single_particle_condition(wl.moments[0], order, lam))
        assert rhs_error(gM, oM, order, lam) <= tol


@pytest.mark.parametrize("order,n", [(0, 2), (1, 5), (2, 37), (3, 70), (4, 131), (6, 97), (8, 40)])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_multi_particle_rhs(mm, order, n, prec):
    wl = mmvm_inputs.random_disk(n=n, order=order, radius=2.0 + 0.15 * n ** 0.5, sigma=0.45,
                                 amp=0.03, moment_scale="absolute", seed=100 + order)
    t = 0.7
    ox, oM = rhs_regrouped(wl.x, wl.moments, t, order, wl.lam0, wl.nu)
    p = mm.MMVM_FP64 if prec == "fp64" else mm.MMVM_MIXED_FP32
    gx, gM = _gpu_rhs(mm, wl, t, p)
    lam = lam_at(t, wl.lam0, wl.nu)
    if prec == "fp64":
        assert vel_error_rows(gx, ox) <= FP64_TOL
        if order >= 2:
            assert rhs_error_rows(gM, oM, order, lam) <= FP64_TOL
    else:
        ev, em = cond_errors(gx, gM, ox, oM, wl.x, wl.moments, t, order, wl.lam0, wl.nu,
                             np.arange(wl.n))
        assert ev <= mixed_rhs_tol(order)
        if order >= 2:
            assert em <= mixed_rhs_tol(order)


def test_literal_form_small(mm):
    """Tiny case against the literal Gamma-tensor form (no regrouping)."""
    wl = mmvm_inputs.random_disk(n=4, order=3, radius=1.5, sigma=0.6, amp=0.05, moment_scale="absolute", seed=5)
    ox, oM = rhs_literal(wl.x, wl.moments, 0.0, 3, wl.lam0, wl.nu)
    gx, gM = _gpu_rhs(mm, wl, 0.0, mm.MMVM_FP64)
    assert vel_error_rows(gx, ox) <= FP64_TOL
    assert rhs_error_rows(gM, oM, 3, wl.lam0) <= FP64_TOL


def test_near_coincident_and_far_pairs(mm):
    """Separations from 1e-7 core sizes to 1e4 core sizes (both jet paths)."""
    order = 4
    x = np.array([[0.0, 0.0], [1e-7, 2e-7], [0.3, -0.1], [2.0, 1.0], [40.0, -30.0],
                  [900.0, 1200.0]])
    rng = np.random.default_rng(9)
    K = (order + 1) * (order + 2) // 2
    mom = rng.normal(size=(6, K)) * 0.05
    mom[:, 0] = [1.0, -0.7, 0.4, 0.9, -1.1, 0.5]
    mom[:, 1:3] = 0.0
    lam0, nu, t = 0.2, 1e-3, 0.0
    ox, oM = rhs_regrouped(x, mom, t, order, lam0, nu)
    with mm.Context(order, lam0, nu, mm.MMVM_FP64) as ctx:
        ctx.set_state(x, mom, t)
        gx, gM = ctx.rhs()
    assert vel_error_rows(gx, ox) <= FP64_TOL
    assert rhs_error_rows(gM, oM, order, lam0) <= FP64_TOL


def _loose_group_workload(order):
    """A tight cluster of 32 particles (radius 0.1) and 32 spread from 0.3
    to 8 along a spiral around it: the spread group's box reaches into the
    cluster, so its list holds the cluster's sources, while its outer
    targets sit at x = |s|^2 / (2 lambda^2) up to ~800 from them, beyond the
    table form of the edge (x < 300): one warp then holds lanes on both
    forms of the per-order branch."""
    rng = np.random.default_rng(77)
    r_in = 0.1 * np.sqrt(rng.uniform(size=32))
    th_in = rng.uniform(0, 2 * np.pi, 32)
    r_out = np.linspace(0.3, 8.0, 32)
    th_out = np.linspace(0.0, 5 * np.pi, 32)
    x = np.concatenate([np.stack([r_in * np.cos(th_in), r_in * np.sin(th_in)], 1),
                        np.stack([r_out * np.cos(th_out), r_out * np.sin(th_out)], 1)])
    K = (order + 1) * (order + 2) // 2
    mom = rng.normal(size=(64, K)) * 0.02
    mom[:, 0] = rng.normal(size=64)
    mom[:, 1:3] = 0.0
    return x, mom


@pytest.mark.parametrize("order", [4, 6])
def test_near_list_lanes_on_both_edge_forms(mm, order, monkeypatch):
    """Every compiled variant against the oracle when a near-listed group
    mixes pairs below and above the table form's limit (mixed precision,
    far field on), and the FP64 form at 1e-12."""
    x, mom = _loose_group_workload(order)
    lam0, nu, t = 0.2, 1e-3, 0.0
    ox, oM = rhs_regrouped(x, mom, t, order, lam0, nu)
    dx = x[32:, None, :] - x[None, :32, :]
    xs = (dx ** 2).sum(-1) / (2 * lam0 ** 2)
    assert xs.max() > 600.0 and xs.min() < 5.0  # both forms occur in the pairs
    with mm.Context(order, lam0, nu, mm.MMVM_FP64) as ctx:
        ctx.set_state(x, mom, t)
        gx, gM = ctx.rhs()
    assert vel_error_rows(gx, ox) <= FP64_TOL
    assert rhs_error_rows(gM, oM, order, lam0) <= FP64_TOL
    nd, nl = mm.pair_variant_counts(order)
    assert nl >= 1
    for v in range(nd + nl):
        monkeypatch.setenv("MMVM_PAIR_VARIANT", str(v))
        with mm.Context(order, lam0, nu, mm.MMVM_MIXED_FP32) as ctx:
            ctx.set_state(x, mom, t)
            gx, gM = ctx.rhs()
            cfg = mm.mmvm_pair_config(ctx.handle)
        assert cfg["variant"] == v
        ev, em = cond_errors(gx, gM, ox, oM, x, mom, t, order, lam0, nu, np.arange(64))
        assert ev <= mixed_rhs_tol(order), cfg
        assert em <= mixed_rhs_tol(order), cfg


def test_rk4_fp64_matches_oracle(mm):
    wl = mmvm_inputs.random_disk(n=24, order=3, radius=2.0, sigma=0.5, amp=0.03, moment_scale="absolute", seed=3)
    dt, nsteps = 0.02, 5
    ox, oM, ot = rk4(wl.x, wl.moments, 0.0, dt, nsteps, 3, wl.lam0, wl.nu)
    with mm.Context(3, wl.lam0, wl.nu, mm.MMVM_FP64) as ctx:
        ctx.set_state(wl.x, wl.moments, 0.0)
        ctx.step(dt, nsteps)
        gx, gM, gt = ctx.get_state()
    assert gt == pytest.approx(ot, rel=1e-15)
    lam = lam_at(ot, wl.lam0, wl.nu)
    assert np.abs(gx - ox).max() / lam <= FP64_TOL
    assert state_error(gM, oM, 3, lam) <= FP64_TOL


def test_rk4_mixed_100_steps(mm):
    """Mixed precision: <= 1e-5 relative on moments after 100 RK4 steps.

    Two co-rotating patches of 24 particles (higher moments start at 0 and
    grow to ~2.5% of the circulation over the run)."""
    wl = mmvm_inputs.two_patches(n=48, order=4, sigma=0.35, seed=11)
    dt, nsteps = 0.05, 100
    ox, oM, ot = rk4(wl.x, wl.moments, 0.0, dt, nsteps, 4, wl.lam0, wl.nu)
    with mm.Context(4, wl.lam0, wl.nu, mm.MMVM_MIXED_FP32) as ctx:
        ctx.set_state(wl.x, wl.moments, 0.0)
        ctx.step(dt, nsteps)
        gx, gM, gt = ctx.get_state()
    lam = lam_at(ot, wl.lam0, wl.nu)
    assert state_error(gM, oM, 4, lam) <= 1e-5
    assert np.abs(gx - ox).max() / lam <= 1e-5


def test_mixed_trajectory_every_far_path_100_steps(mm):
    """The stated mixed-precision target on the benchmark recipe: two
    co-rotating patches, N = 8192, M = 6, sigma = 0.1, Re = 2000, 100 RK4
    steps of 0.05, mixed precision with every far path active (far sources
    of near tiles, far tiles source by source, tile expansions), against the
    plain FP64 form of the same 100 steps (the FP64 path is held to 1e-12 of
    the oracle on short trajectories above): <= 1e-5 per particle on the
    moments (weighted norm) and on the centroids (in core sizes)."""
    wl = mmvm_inputs.two_patches(n=8192, order=6, sigma=0.1, Re=2000.0, dt=0.05)
    nsteps = 100
    with mm.Context(6, wl.lam0, wl.nu, mm.MMVM_MIXED_FP32) as ctx:
        ctx.set_state(wl.x, wl.moments, 0.0)
        w0 = mm.mmvm_pair_work(ctx.handle)
        ctx.step(wl.dt, nsteps)
        gx, gM, gt = ctx.get_state()
        near, far_pp, n_m2p, m2p_pairs = [b - a for a, b in zip(w0, mm.mmvm_pair_work(ctx.handle))]
    assert near > 0 and far_pp > 0 and n_m2p > 0 and m2p_pairs > 0
    assert near + far_pp + m2p_pairs == 4 * nsteps * wl.n * wl.n
    with mm.Context(6, wl.lam0, wl.nu, mm.MMVM_FP64) as c64:
        c64.set_state(wl.x, wl.moments, 0.0)
        c64.step(wl.dt, nsteps)
        dx, dM, dt_ = c64.get_state()
    assert gt == dt_
    assert np.all(np.isfinite(gM)) and np.all(np.isfinite(dM))
    lam = lam_at(gt, wl.lam0, wl.nu)
    # the moments have grown from zero: every order is populated
    assert np.abs(dM[:, 3:]).max() > 1e-3 * np.abs(dM[:, :1]).max() * lam ** 2
    assert state_error(gM, dM, 6, lam) <= 1e-5
    assert position_error(gx, dx, lam) <= 1e-5


def test_single_particle_config_steps(mm):
    """Single particle, order 10 (the M=10 quadrupole case), 50 FP64 steps."""
    wl = mmvm_inputs.single_quadrupole(order=10, eps=0.1, sigma0=1.0, Re=1000.0)
    ox, oM, ot = rk4(wl.x, wl.moments, 0.0, 0.01, 50, 10, wl.lam0, wl.nu)
    with mm.Context(10, wl.lam0, wl.nu, mm.MMVM_FP64) as ctx:
        ctx.set_state(wl.x, wl.moments, 0.0)
        ctx.step(0.01, 50)
        gx, gM, gt = ctx.get_state()
    assert state_error(gM, oM, 10, lam_at(ot, wl.lam0, wl.nu)) <= FP64_TOL


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_random_disk_full_size_sampled_rows(mm, prec):
    """N = 4096, M = 4 random disk: sampled target rows against all sources."""
    wl = mmvm_inputs.random_disk()
    p = mm.MMVM_FP64 if prec == "fp64" else mm.MMVM_MIXED_FP32
    gx, gM = _gpu_rhs(mm, wl, 0.0, p)
    rows = np.random.default_rng(1).choice(wl.n, 12, replace=False)
    ox, oM = rhs_regrouped(wl.x, wl.moments, 0.0, wl.order, wl.lam0, wl.nu, rows=rows)
    if prec == "fp64":
        assert vel_error_rows(gx[rows], ox) <= FP64_TOL
        assert rhs_error_rows(gM[rows], oM, wl.order, wl.lam0) <= FP64_TOL
    else:
        ev, em = cond_errors(gx[rows], gM[rows], ox, oM, wl.x, wl.moments, 0.0, wl.order,
                             wl.lam0, wl.nu, rows)
        assert ev <= MIXED_RHS_TOL and em <= MIXED_RHS_TOL


@pytest.fixture(scope="module")
def two_patches_rows():
    """The benchmark workload and the oracle's right-hand side on 72 target
    rows against all 65536 sources (computed once, one oracle process per
    host core): 32 random rows and 40 rows aimed at the kernel's path
    switches (groups straddling the near/far threshold x_far(M), groups with
    source tiles just inside the tile-expansion criterion, the loosest group
    boxes, the smallest circulations, the last group)."""
    wl = mmvm_inputs.two_patches()
    kinds = {"random": [int(j) for j in np.random.default_rng(2).choice(wl.n, 32, replace=False)]}
    kinds.update(switch_rows(wl.x, wl.moments, wl.order, wl.lam0))
    rows = np.array(sorted({j for v in kinds.values() for j in v}))
    ox, oM = oracle_rows_parallel(wl.x, wl.moments, 0.0, wl.order, wl.lam0, wl.nu, rows)
    from tests.parity_util import abs_scale_rows

    sx, sM = abs_scale_rows(wl.x, wl.moments, 0.0, wl.order, wl.lam0, wl.nu, rows)
    return wl, rows, ox, oM, kinds, sx, sM


def _check_rows(gx, gM, wl, rows, ox, oM, kinds, sx, sM, tol):
    """Per-particle errors on the sampled rows (conditioning-aware norm),
    reported per kind of row."""
    from tests.parity_util import rhs_error_cond, vel_error_cond

    pos = {j: i for i, j in enumerate(rows)}
    bad = {}
    for kind, rr in kinds.items():
        ii = [pos[j] for j in rr]
        ev = vel_error_cond(gx[rr], ox[ii], sx[ii])
        em = rhs_error_cond(gM[rr], oM[ii], sM[ii], wl.order, wl.lam0)
        if not (ev <= tol and em <= tol):
            bad[kind] = (ev, em)
    assert not bad, f"rows above {tol}: {bad}"
    assert vel_error_cond(gx[rows], ox, sx) <= tol
    assert rhs_error_cond(gM[rows], oM, sM, wl.order, wl.lam0) <= tol


@pytest.mark.parametrize("variant", [None, 0, 8, 10, 11, 12, 13, 14, 15])
def test_two_patches_full_size_sampled_rows(mm, two_patches_rows, variant, monkeypatch):
    """N = 65536, M = 6 two patches (mixed precision), in the launch
    configurations bench.py times (the autotuner's choice; the direct form's
    fused variant 0 and split variants 8, 10, 11 and the list form's
    variants 12-15 forced): sampled rows vs the oracle."""
    wl, rows, ox, oM, kinds, sx, sM = two_patches_rows
    if variant is not None:
        monkeypatch.setenv("MMVM_PAIR_VARIANT", str(variant))
    with mm.Context(wl.order, wl.lam0, wl.nu, mm.MMVM_MIXED_FP32) as ctx:
        ctx.set_state(wl.x, wl.moments, 0.0)
        cfg = mm.mmvm_pair_config(ctx.handle)
        gx, gM = ctx.rhs()
    if variant is not None:
        assert cfg["variant"] == variant
    assert np.all(np.isfinite(gM)) and np.all(np.isfinite(gx))
    _check_rows(gx, gM, wl, rows, ox, oM, kinds, sx, sM, MIXED_RHS_TOL)
    # total impulse sum_j M00 xdot^j vanishes (pair antisymmetry) at any size
    imp = (wl.moments[:, :1] * gx).sum(0)
    assert np.abs(imp).max() <= 1e-6 * np.abs(wl.moments[:, :1] * gx).sum()


@pytest.mark.parametrize("variant", [0, 8, 10, 11, 12, 13, 14, 15])
def test_two_patches_ragged_size_every_path(mm, variant, monkeypatch):
    """N = 5003 (ragged for 32-source groups and 128/256/384-target CTAs), two
    patches, M = 6, mixed precision, far field on: every path of the pair
    kernel runs (near sources, far sources inside near tiles, far tiles
    source by source, tile expansions); sampled rows vs the oracle and the
    work counts add up to every ordered pair."""
    wl = mmvm_inputs.two_patches(n=5003, order=6, sigma=0.1, seed=77)
    rng = np.random.default_rng(7)
    wl.moments[:, 3:] = rng.normal(size=wl.moments[:, 3:].shape) * 1e-3 * wl.moments[:, :1] \
        * wl.lam0 ** 2
    monkeypatch.setenv("MMVM_PAIR_VARIANT", str(variant))
    with mm.Context(6, wl.lam0, wl.nu, mm.MMVM_MIXED_FP32) as ctx:
        ctx.set_state(wl.x, wl.moments, 0.0)
        assert mm.mmvm_pair_config(ctx.handle)["variant"] == variant
        gx, gM = ctx.rhs()
        near, far_pp, n_m2p, m2p_pairs = mm.mmvm_pair_work(ctx.handle)
    assert near > 0 and far_pp > 0 and n_m2p > 0
    assert near + far_pp + m2p_pairs == wl.n * wl.n
    picks = switch_rows(wl.x, wl.moments, 6, wl.lam0, per_kind=4)
    rows = np.array(sorted({0, wl.n - 1, *np.random.default_rng(8).choice(wl.n, 6, replace=False),
                            *(j for v in picks.values() for j in v)}))
    ox, oM = rhs_regrouped(wl.x, wl.moments, 0.0, 6, wl.lam0, wl.nu, rows=rows)
    ev, em = cond_errors(gx[rows], gM[rows], ox, oM, wl.x, wl.moments, 0.0, 6, wl.lam0, wl.nu,
                         rows)
    assert ev <= MIXED_RHS_TOL and em <= MIXED_RHS_TOL


def test_error_codes(mm):
    wl = mmvm_inputs.random_disk(n=8, order=2, seed=1)
    with mm.Context(2, wl.lam0, wl.nu, mm.MMVM_FP64) as ctx:
        bad = wl.moments.copy()
        bad[3, 0] = 0.0
        with pytest.raises(mm.MMVMError) as ei:
            ctx.set_state(wl.x, bad, 0.0)
        assert ei.value.code == mm.MMVM_E_ZERO_CIRCULATION
        bad = wl.moments.copy()
        bad[2, 4] = np.nan
        with pytest.raises(mm.MMVMError) as ei:
            ctx.set_state(wl.x, bad, 0.0)
        assert ei.value.code == mm.MMVM_E_NUMERIC
    with mm.Context(10, 1.0, 0.0, mm.MMVM_FP64) as ctx:
        K = 66
        with pytest.raises(mm.MMVMError) as ei:
            ctx.set_state(np.zeros((2, 2)), np.ones((2, K)), 0.0)
        assert ei.value.code == mm.MMVM_E_UNSUPPORTED


def test_far_field_matches_full_jet(mm):
    """Mixed precision with and without the far-field (point-vortex) tiles."""
    wl = mmvm_inputs.two_patches(n=4096, order=6, sigma=0.1)
    rng = np.random.default_rng(3)
    wl.moments[:, 3:] = rng.normal(size=wl.moments[:, 3:].shape) * 1e-3 * wl.moments[:, :1] \
        * wl.lam0 ** 2
    res = {}
    for name, flags in (("far", 0), ("full", mm.MMVM_FLAG_NO_FAR_FIELD)):
        with mm.Context(6, wl.lam0, wl.nu, mm.MMVM_MIXED_FP32, flags=flags) as ctx:
            ctx.set_state(wl.x, wl.moments, 0.0)
            res[name] = ctx.rhs()
    # every row, relative to the largest row
    assert vel_error(res["far"][0], res["full"][0]) <= 1e-6
    assert rhs_error(res["far"][1], res["full"][1], 6, wl.lam0) <= 1e-6
    # sampled rows, per particle (conditioning-aware): far field vs full jet and vs the oracle
    picks = switch_rows(wl.x, wl.moments, 6, wl.lam0, per_kind=4)
    rows = np.array(sorted({*np.random.default_rng(4).choice(wl.n, 16, replace=False),
                            *(j for v in picks.values() for j in v)}))
    ev, em = cond_errors(res["far"][0][rows], res["far"][1][rows], res["full"][0][rows],
                         res["full"][1][rows], wl.x, wl.moments, 0.0, 6, wl.lam0, wl.nu, rows)
    assert ev <= 2e-6 and em <= 2e-6
    ox, oM = oracle_rows_parallel(wl.x, wl.moments, 0.0, 6, wl.lam0, wl.nu, rows)
    ev, em = cond_errors(res["far"][0][rows], res["far"][1][rows], ox, oM, wl.x, wl.moments, 0.0,
                         6, wl.lam0, wl.nu, rows)
    assert ev <= MIXED_RHS_TOL and em <= MIXED_RHS_TOL


@pytest.mark.parametrize("order,kind", [(0, "patches"), (1, "disk"), (2, "disk"), (4, "disk"),
                                        (6, "patches"), (8, "disk")])
def test_tile_expansions_match_full_jet(mm, order, kind):
    """Far tiles summed through their expansion about the tile centre (and
    the rest source by source) against every pair through the full jet
    (2e-6), and sampled rows against the oracle (the mixed tolerance); the
    kernel must really have taken both far routes."""
    if kind == "patches":
        wl = mmvm_inputs.two_patches(n=8192, order=order, sigma=0.1, seed=500 + order)
        if order >= 2:
            rng = np.random.default_rng(order)
            wl.moments[:, 3:] = rng.normal(size=wl.moments[:, 3:].shape) * 1e-3 \
                * wl.moments[:, :1] * wl.lam0 ** 2
    else:
        wl = mmvm_inputs.random_disk(n=6000, order=order, radius=30.0, sigma=0.5,
                                     seed=510 + order)
    res = {}
    for name, flags in (("far", 0), ("full", mm.MMVM_FLAG_NO_FAR_FIELD)):
        with mm.Context(order, wl.lam0, wl.nu, mm.MMVM_MIXED_FP32, flags=flags) as ctx:
            ctx.set_state(wl.x, wl.moments, 0.0)
            res[name] = ctx.rhs()
            if name == "far":
                near, far_pp, n_m2p, m2p_pairs = mm.mmvm_pair_work(ctx.handle)
    assert n_m2p > 0 and m2p_pairs > 0 and far_pp > 0 and near > 0
    assert near + far_pp + m2p_pairs == wl.n * (wl.n - 1) + wl.n  # every ordered pair, self included
    # every row, relative to the largest row
    assert vel_error(res["far"][0], res["full"][0]) <= 2e-6
    if order >= 2:
        assert rhs_error(res["far"][1], res["full"][1], order, wl.lam0) <= 2e-6
    # sampled rows, per particle (conditioning-aware): far field vs full jet and vs the oracle
    picks = switch_rows(wl.x, wl.moments, order, wl.lam0, per_kind=3)
    rows = np.array(sorted({*np.random.default_rng(5).choice(wl.n, 8, replace=False),
                            *(j for v in picks.values() for j in v)}))
    ev, em = cond_errors(res["far"][0][rows], res["far"][1][rows], res["full"][0][rows],
                         res["full"][1][rows], wl.x, wl.moments, 0.0, order, wl.lam0, wl.nu, rows)
    assert ev <= 2e-6
    if order >= 2:
        assert em <= 2e-6
    ox, oM = oracle_rows_parallel(wl.x, wl.moments, 0.0, order, wl.lam0, wl.nu, rows)
    ev, em = cond_errors(res["far"][0][rows], res["far"][1][rows], ox, oM, wl.x, wl.moments, 0.0,
                         order, wl.lam0, wl.nu, rows)
    assert ev <= mixed_rhs_tol(order)
    if order >= 2:
        assert em <= mixed_rhs_tol(order)


@pytest.mark.parametrize("order,kind", [(2, "disk"), (4, "disk"), (6, "patches"), (8, "disk")])
def test_tree_far_field_matches_flat_and_full_jet(mm, order, kind, monkeypatch):
    """The list form's far field through the tree over the groups (node
    expansions built by exact shifts of the group expansions) against the
    flat far kernel (one expansion per far group) and against every pair
    through the full jet; the tree must evaluate fewer expansions for the
    same pairs, and every ordered pair is covered once."""
    if kind == "patches":
        wl = mmvm_inputs.two_patches(n=8192, order=order, sigma=0.1, seed=600 + order)
        rng = np.random.default_rng(order)
        wl.moments[:, 3:] = rng.normal(size=wl.moments[:, 3:].shape) * 1e-3 \
            * wl.moments[:, :1] * wl.lam0 ** 2
    else:
        wl = mmvm_inputs.random_disk(n=6000, order=order, radius=30.0, sigma=0.5,
                                     seed=610 + order)
    nv = mm.pair_variant_counts(order)[0]
    res, work = {}, {}
    for name, tree, flags in (("tree", "1", 0), ("flat", "0", 0),
                              ("full", "0", mm.MMVM_FLAG_NO_FAR_FIELD)):
        monkeypatch.setenv("MMVM_FAR_TREE", tree)
        if flags == 0:
            monkeypatch.setenv("MMVM_PAIR_VARIANT", str(nv))  # the first list variant
        else:
            monkeypatch.delenv("MMVM_PAIR_VARIANT", raising=False)
        with mm.Context(order, wl.lam0, wl.nu, mm.MMVM_MIXED_FP32, flags=flags) as ctx:
            ctx.set_state(wl.x, wl.moments, 0.0)
            cfg = mm.mmvm_pair_config(ctx.handle)
            if flags == 0:
                assert cfg["list_form"] == (2 if tree == "1" else 1)
            res[name] = ctx.rhs()
            work[name] = mm.mmvm_pair_work(ctx.handle)
    for name in ("tree", "flat"):
        near, far_pp, n_m2p, m2p_pairs = work[name]
        assert near + far_pp + m2p_pairs == wl.n * wl.n
    assert work["tree"][0] == work["flat"][0]  # the same near pairs
    assert work["tree"][2] < work["flat"][2]   # fewer expansions evaluated
    assert vel_error(res["tree"][0], res["full"][0]) <= 2e-6
    assert vel_error(res["tree"][0], res["flat"][0]) <= 1e-6
    if order >= 2:
        assert rhs_error(res["tree"][1], res["full"][1], order, wl.lam0) <= 2e-6
        assert rhs_error(res["tree"][1], res["flat"][1], order, wl.lam0) <= 1e-6
    picks = switch_rows(wl.x, wl.moments, order, wl.lam0, per_kind=3)
    rows = np.array(sorted({*np.random.default_rng(9).choice(wl.n, 8, replace=False),
                            *(j for v in picks.values() for j in v)}))
    ev, em = cond_errors(res["tree"][0][rows], res["tree"][1][rows], res["full"][0][rows],
                         res["full"][1][rows], wl.x, wl.moments, 0.0, order, wl.lam0, wl.nu, rows)
    assert ev <= 2e-6 and em <= 2e-6


@pytest.mark.parametrize("order", [0, 1, 2, 3, 4, 5, 6, 7, 8])
def test_every_kernel_variant(mm, order, monkeypatch):
    """Each compiled all-pairs variant (the direct form and the list form)
    reproduces the oracle (mixed precision, far field on)."""
    wl = mmvm_inputs.random_disk(n=300, order=order, radius=3.0, sigma=0.45, amp=0.02, moment_scale="absolute",
                                 seed=40 + order)
    ox, oM = rhs_regrouped(wl.x, wl.moments, 0.0, order, wl.lam0, wl.nu)
    from tests.parity_util import abs_scale_rows, rhs_error_cond, vel_error_cond

    sx, sM = abs_scale_rows(wl.x, wl.moments, 0.0, order, wl.lam0, wl.nu, np.arange(wl.n))
    seen = set()
    for v in range(32):
        monkeypatch.setenv("MMVM_PAIR_VARIANT", str(v))
        ctx = mm.Context(order, wl.lam0, wl.nu, mm.MMVM_MIXED_FP32)
        try:
            ctx.set_state(wl.x, wl.moments, 0.0)
        except mm.MMVMError as err:
            ctx.close()
            assert err.code == mm.MMVM_E_INVALID_ARG  # no such variant
            break
        cfg = mm.mmvm_pair_config(ctx.handle)
        gx, gM = ctx.rhs()
        ctx.close()
        assert cfg["variant"] == v
        seen.add(v)
        assert vel_error_cond(gx, ox, sx) <= mixed_rhs_tol(order), cfg
        if order >= 1:
            assert rhs_error_cond(gM, oM, sM, order, wl.lam0) <= mixed_rhs_tol(order), cfg
    assert len(seen) >= 2


@pytest.mark.parametrize("n", [262144])
def test_tree_far_field_at_large_n(mm, n, monkeypatch):
    """N = 262144 two patches with the core shrunk as sigma = 0.1 sqrt(65536 / N)
    (the near work per particle of the benchmark): the list form with the
    tree far field against every pair through the full jet on sampled rows
    (2e-6 per particle, conditioning-aware) and against the oracle (the mixed
    tolerance)."""
    sigma = 0.1 * math.sqrt(65536.0 / n)
    wl = mmvm_inputs.two_patches(n=n, order=6, sigma=sigma, seed=900)
    nv = mm.pair_variant_counts(6)[0]
    res = {}
    for name, flags in (("tree", 0), ("full", mm.MMVM_FLAG_NO_FAR_FIELD)):
        if flags == 0:
            monkeypatch.setenv("MMVM_PAIR_VARIANT", str(nv + 4))
            monkeypatch.setenv("MMVM_FAR_TREE", "1")
        else:
            monkeypatch.setenv("MMVM_PAIR_VARIANT", "0")
        with mm.Context(6, wl.lam0, wl.nu, mm.MMVM_MIXED_FP32, flags=flags) as ctx:
            ctx.set_state(wl.x, wl.moments, 0.0)
            if flags == 0:
                assert mm.mmvm_pair_config(ctx.handle)["list_form"] == 2
            res[name] = ctx.rhs()
            if flags == 0:
                near, far_pp, n_m2p, m2p_pairs = mm.mmvm_pair_work(ctx.handle)
    assert near + far_pp + m2p_pairs == wl.n * wl.n and n_m2p > 0 and far_pp > 0
    picks = switch_rows(wl.x, wl.moments, 6, wl.lam0, per_kind=3)
    rows = np.array(sorted({*np.random.default_rng(11).choice(wl.n, 9, replace=False),
                            *(j for v in picks.values() for j in v)}))
    ev, em = cond_errors(res["tree"][0][rows], res["tree"][1][rows], res["full"][0][rows],
                         res["full"][1][rows], wl.x, wl.moments, 0.0, 6, wl.lam0, wl.nu, rows)
    assert ev <= 2e-6 and em <= 2e-6
    ox, oM = oracle_rows_parallel(wl.x, wl.moments, 0.0, 6, wl.lam0, wl.nu, rows)
    ev, em = cond_errors(res["tree"][0][rows], res["tree"][1][rows], ox, oM, wl.x, wl.moments,
                         0.0, 6, wl.lam0, wl.nu, rows)
    assert ev <= MIXED_RHS_TOL and em <= MIXED_RHS_TOL
