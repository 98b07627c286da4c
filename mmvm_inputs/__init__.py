"""Seeded synthetic workloads for the multi-moment vortex method (MMVM).

This module only *draws* states: particle centres x^j, Hermite moments
M^j[k1,k2] laid out by total order, the core size lambda_0 and the viscosity.
It holds none of the method's arithmetic (no coefficients, no velocities, no
right-hand side), so both the FP64 oracle and the CUDA path may use it.

Moment layout (one row per particle): the moment of multi-index (k1, k2),
with n = k1 + k2 <= order, sits at column n(n+1)/2 + k2.  Column 0 is the
circulation M[0,0] (the particle's total vorticity).

Workload recipes (Section 3 of the paper for the physical set-ups; the sizes
are the benchmark configurations of this project):

* ``single_quadrupole``: one particle, a Lamb-Oseen core of circulation 1
  plus a quadrupole of amplitude eps on (2,0)/(0,2)/(1,1)
  (Section 3.1.1, eq:perturb2 / eq:IC_sd generalised to core sigma0):
  M[2,0] = eps*sigma0^2, M[0,2] = -eps*sigma0^2, M[1,1] = 2*eps*sigma0^2.
  With sigma0 = 2 and the (1,1) part off this is exactly eq:IC_sd with
  delta = eps.
* ``random_disk``: n particles uniform in a disk (r = R*sqrt(U)),
  circulations N(0,1), magnitudes floored at 0.1 (sign kept) and then the
  mean removed; first moments 0 (the centroid condition, eq:xjdef); moments
  of order >= 2 i.i.d. N(0, amp^2) in the weighted norm of the convergence
  theorem relative to the circulation (see random_disk).
* ``two_patches``: two co-rotating Gaussian patches of n/2 particles each,
  uniform in disks of radius 2 centred at (+-3, 0), circulations proportional
  to exp(-r^2) about the patch centre and normalised to 1 per patch, higher
  moments 0.
* ``tripole_coarse_grid``: the coarse-grid tripole of Section 3.2.2: a
  6 x 6 grid of centres on [-1, 1]^2, each particle's circulation the value
  of the perturbed Lamb-Oseen vorticity of eq:perturbM2 at its node times the
  node's area (eq:blurredIC), higher moments 0.
* ``vortex_pair``: two equal Gaussian vortices of circulation 1 at
  (+-b/2, 0) with core a (Section 3.2.1, vortex merger), higher moments 0.
* ``served_stream``: independent random_disk requests with log-uniform n,
  order drawn from {2,4,8}, Re uniform, step counts uniform, Poisson arrivals.

Every generator takes an explicit seed; the default seeds are 20101010 plus a
workload number.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

BASE_SEED = 20101010

__all__ = [
    "Workload",
    "n_moments",
    "single_quadrupole",
    "random_disk",
    "two_patches",
    "served_stream",
    "tripole_coarse_grid",
    "vortex_pair",
    "BASE_SEED",
]


def n_moments(order: int) -> int:
    """Number of moments with k1 + k2 <= order: (order+1)(order+2)/2."""
    return (order + 1) * (order + 2) // 2


def _col(k1: int, k2: int) -> int:
    n = k1 + k2
    return n * (n + 1) // 2 + k2


@dataclass
class Workload:
    """A synthetic MMVM initial-value problem.

    x: (n, 2) float64 particle centres; moments: (n, K) float64 Hermite
    moments (layout above); order: truncation order M; lam0: the shared core
    size lambda_0 (lambda^2 = lambda_0^2 + 4 nu t); nu: kinematic viscosity
    (Re = 1/nu with unit reference circulation); dt, steps: the RK4 schedule;
    t0: start time; name: what the workload is.
    """

    x: np.ndarray
    moments: np.ndarray
    order: int
    lam0: float
    nu: float
    dt: float
    steps: int
    t0: float = 0.0
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.x.shape[0])

    @property
    def K(self) -> int:
        return n_moments(self.order)

    def subset(self, n: int) -> "Workload":
        """The first n particles (a smaller case of the same recipe)."""
        return Workload(self.x[:n].copy(), self.moments[:n].copy(), self.order,
                        self.lam0, self.nu, self.dt, self.steps, self.t0,
                        f"{self.name}[:{n}]", dict(self.meta))


def single_quadrupole(order: int = 10, eps: float = 0.1, sigma0: float = 1.0,
                      Re: float = 1000.0, dt: float = 0.01, steps: int = 500,
                      with_11: bool = True) -> Workload:
    """One particle: Lamb-Oseen core (circulation 1) plus a quadrupole."""
    K = n_moments(order)
    m = np.zeros((1, K))
    m[0, 0] = 1.0
    if order >= 2:
        m[0, _col(2, 0)] = eps * sigma0 ** 2
        m[0, _col(0, 2)] = -eps * sigma0 ** 2
        if with_11:
            m[0, _col(1, 1)] = 2.0 * eps * sigma0 ** 2
    return Workload(np.zeros((1, 2)), m, order, sigma0, 1.0 / Re, dt, steps,
                    name=f"single particle M={order} eps={eps} Re={Re:g}",
                    meta={"eps": eps, "Re": Re, "sigma0": sigma0})


def random_disk(n: int = 4096, order: int = 4, radius: float = 10.0,
                sigma: float = 0.5, amp: float = 0.01, Re: float = 500.0,
                dt: float = 0.01, steps: int = 200, seed: int = BASE_SEED + 3,
                floor: float = 0.1, moment_scale: str = "weighted") -> Workload:
    """Particles uniform in a disk with N(0,1) circulations (mean removed).

    Moments of orders 2..M are amp * N(0,1) draws; first moments are zero.
    moment_scale = "weighted" (the recipe): each draw is measured in the
    weighted enstrophy norm of the convergence theorem relative to the
    particle's own circulation, M_k = amp |M_00| xi_k / sqrt(w_k) with
    w_k = 2^|k| k1! k2! / lambda0^(2|k|), so every particle is its Gaussian
    core plus a perturbation of relative size amp per moment.
    moment_scale = "absolute": M_k = amp xi_k (large high-order moments, for
    single right-hand-side stress tests; the ODE from such states is violent
    and leaves the finite range within tens of steps at M >= 4).
    """
    if moment_scale not in ("weighted", "absolute"):
        raise ValueError("moment_scale must be 'weighted' or 'absolute'")
    rng = np.random.default_rng(seed)
    r = radius * np.sqrt(rng.random(n))
    th = 2.0 * math.pi * rng.random(n)
    x = np.stack([r * np.cos(th), r * np.sin(th)], axis=1)
    g = rng.standard_normal(n)
    g = np.where(np.abs(g) < floor, np.where(g < 0, -floor, floor), g)
    if n > 1:
        g = g - g.mean()
    K = n_moments(order)
    m = np.zeros((n, K))
    m[:, 0] = g
    if order >= 2:
        hi = rng.standard_normal((n, K - 3)) * amp
        if moment_scale == "weighted":
            w = []
            for s in range(2, order + 1):
                for k2 in range(s + 1):
                    k1 = s - k2
                    w.append(2.0 ** s * math.factorial(k1) * math.factorial(k2) / sigma ** (2 * s))
            hi = hi * np.abs(g)[:, None] / np.sqrt(np.array(w))[None, :]
        m[:, 3:] = hi
    return Workload(x, m, order, sigma, 1.0 / Re, dt, steps,
                    name=f"random disk N={n} M={order} R={radius:g} sigma={sigma:g}",
                    meta={"seed": seed, "Re": Re, "moment_scale": moment_scale})


def two_patches(n: int = 65536, order: int = 6, sigma: float = 0.1,
                Re: float = 2000.0, dt: float = 0.05, steps: int = 100,
                seed: int = BASE_SEED + 4, radius: float = 2.0,
                separation: float = 6.0) -> Workload:
    """Two co-rotating Gaussian-weighted patches of n/2 particles each."""
    rng = np.random.default_rng(seed)
    half = n // 2
    parts_x, parts_g = [], []
    for c, cnt in ((-separation / 2, half), (separation / 2, n - half)):
        r = radius * np.sqrt(rng.random(cnt))
        th = 2.0 * math.pi * rng.random(cnt)
        xs = np.stack([c + r * np.cos(th), r * np.sin(th)], axis=1)
        w = np.exp(-r ** 2)
        parts_x.append(xs)
        parts_g.append(w / w.sum())
    x = np.concatenate(parts_x)
    K = n_moments(order)
    m = np.zeros((n, K))
    m[:, 0] = np.concatenate(parts_g)
    return Workload(x, m, order, sigma, 1.0 / Re, dt, steps,
                    name=f"two patches N={n} M={order} sigma={sigma:g}",
                    meta={"seed": seed, "Re": Re})


@dataclass
class Request:
    """One served solve: its workload and its arrival time (seconds)."""

    index: int
    arrival: float
    workload: Workload


def served_stream(count: int = 2000, rate: float = 1.0, seed: int = BASE_SEED + 5,
                  n_min: int = 64, n_max: int = 8192, orders=(2, 4, 8),
                  re_range=(100.0, 5000.0), step_range=(50, 500),
                  dt: float = 0.01) -> list[Request]:
    """Independent random-disk solves with Poisson arrivals (rate per second)."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for i in range(count):
        t += rng.exponential(1.0 / rate)
        n = int(round(math.exp(rng.uniform(math.log(n_min), math.log(n_max)))))
        order = int(rng.choice(orders))
        Re = float(rng.uniform(*re_range))
        steps = int(rng.integers(step_range[0], step_range[1] + 1))
        wl = random_disk(n=n, order=order, Re=Re, dt=dt, steps=steps,
                         seed=seed * 1000 + i)
        out.append(Request(i, t, wl))
    return out


def tripole_coarse_grid(order: int = 2, delta: float = 0.25, lam0: float = 1.0,
                        Re: float = 1000.0, nodes: int = 6, half_width: float = 1.0,
                        dt: float = 0.01, steps: int = 1600) -> Workload:
    """Coarse-grid approximation of a large quadrupole perturbation of the
    Lamb-Oseen vortex (Section 3.2.2).

    The initial vorticity is eq:perturbM2, phi_00 + 4 delta (phi_20 - phi_02)
    with phi_k = D^k phi_00 and phi_00 = exp(-|x|^2/lam0^2) / (pi lam0^2);
    written out, omega_0(x) = phi_00(x) (1 + 16 delta (x1^2 - x2^2) / lam0^4).
    The centres form a uniform nodes x nodes grid on [-half_width,
    half_width]^2, end points included; every node carries the area h^2
    (h the node spacing) and the circulation M^j[0,0] = omega_0(x_j) h^2
    (eq:blurredIC); all other moments are 0.  Every particle has the core
    lam0, the core of the expansion.  Deterministic (no random draws).
    """
    g = np.linspace(-half_width, half_width, nodes)
    h = g[1] - g[0]
    X1, X2 = np.meshgrid(g, g, indexing="ij")
    x = np.stack([X1.ravel(), X2.ravel()], axis=1)
    r2 = x[:, 0] ** 2 + x[:, 1] ** 2
    phi00 = np.exp(-r2 / lam0 ** 2) / (math.pi * lam0 ** 2)
    omega0 = phi00 * (1.0 + 16.0 * delta * (x[:, 0] ** 2 - x[:, 1] ** 2) / lam0 ** 4)
    m = np.zeros((x.shape[0], n_moments(order)))
    m[:, 0] = omega0 * h * h
    return Workload(x, m, order, lam0, 1.0 / Re, dt, steps,
                    name=f"coarse-grid tripole {nodes}x{nodes} M={order} delta={delta}",
                    meta={"delta": delta, "Re": Re, "node_area": h * h})


def vortex_pair(order: int = 6, a_over_b: float = 0.375, b: float = 2.0,
                Re: float = 1000.0, dt: float = 0.01, steps: int = 1200) -> Workload:
    """Two equal co-rotating Gaussian vortices (Section 3.2.1, vortex
    merger): centres (-b/2, 0) and (b/2, 0), circulation M[0,0] = 1 each,
    core lambda_0 = a = a_over_b * b (the radius in exp(-r^2/a^2)), higher
    moments 0, nu = 1/Re.  Deterministic."""
    x = np.array([[-0.5 * b, 0.0], [0.5 * b, 0.0]])
    m = np.zeros((2, n_moments(order)))
    m[:, 0] = 1.0
    return Workload(x, m, order, a_over_b * b, 1.0 / Re, dt, steps,
                    name=f"vortex pair a/b={a_over_b} M={order}",
                    meta={"a_over_b": a_over_b, "b": b, "Re": Re})
