"""Seeded synthetic workloads shaped like the paper's runs (Sec. 4 and 6:
32^3 elements, tau = 0.01) at the sizes of the benchmark configurations.

Input generation only: grid sizes, degrees, time steps, Gaussian centres and
directions drawn from a seeded NumPy generator.  No arithmetic of the method
lives here; both the CUDA path and the oracle consume these parameters.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

RICKER_FREQ = 8.0
RICKER_T0 = 1.0 / RICKER_FREQ


@dataclass
class WaveCase:
    name: str
    n_elem: tuple
    p: int
    tau: float
    steps: int
    u0: dict | None = None          # Gaussian initial displacement (amp, center, den)
    source: dict | None = None      # Ricker x Gaussian source (amp, center, den, freq, t0)
    c2: float = 1.0


@dataclass
class ElasticCase:
    name: str
    n_elem: tuple
    p: int
    tau: float
    steps: int
    lam: float = 1.0
    mu: float = 1.0
    rho: float = 1.0
    v0: dict | None = None          # vector Gaussian initial velocity (amp, dir, center, den)


def interior_point(seed: int, lo: float = 0.25, hi: float = 0.75):
    rng = np.random.default_rng(seed)
    return tuple(float(v) for v in rng.uniform(lo, hi, 3))


def unit_vector(seed: int):
    rng = np.random.default_rng(seed)
    a = rng.standard_normal(3)
    return tuple(float(v) for v in a / np.linalg.norm(a))


def pulse_case(ne=16, p=2, tau=1e-2, steps=20) -> WaveCase:
    """16^3 elements, quadratic C1 splines, Gaussian pulse exp(-|x-c|^2/0.01)
    at the cube centre, zero velocity, no source."""
    ne3 = (ne, ne, ne) if np.ndim(ne) == 0 else tuple(ne)
    return WaveCase("pulse", ne3, p, tau, steps, u0=dict(amp=1.0, center=(0.5, 0.5, 0.5), den=0.01))


def ricker_case(ne=128, p=2, tau=2e-3, steps=200, seed=0, sigma=0.02) -> WaveCase:
    """Zero initial state; source = Ricker(f=8, t0=1/8) in time times a
    Gaussian exp(-|x-s|^2/(2 sigma^2)) at a seeded point in [0.25, 0.75]^3."""
    ne3 = (ne, ne, ne) if np.ndim(ne) == 0 else tuple(ne)
    src = dict(amp=1.0, center=interior_point(seed), den=2.0 * sigma ** 2, freq=RICKER_FREQ, t0=RICKER_T0)
    return WaveCase("ricker", ne3, p, tau, steps, source=src)


def elastic_case(ne=96, p=2, tau=2e-3, steps=100, seed=0, sigma=0.05) -> ElasticCase:
    """lam = mu = rho = 1, zero displacement, initial velocity
    a exp(-|x-c|^2/(2 sigma^2)) with a seeded unit vector a and a seeded
    centre c in [0.3, 0.7]^3."""
    ne3 = (ne, ne, ne) if np.ndim(ne) == 0 else tuple(ne)
    v0 = dict(amp=1.0, dir=unit_vector(seed + 1000), center=interior_point(seed, 0.3, 0.7),
              den=2.0 * sigma ** 2)
    return ElasticCase("elastic", ne3, p, tau, steps, v0=v0)


def batch_cases(count=64, seed=0, steps=50, lo=32, hi=160, sigma=0.05):
    """Many independent P-wave simulations with uneven grids: elements per
    axis iid uniform in [lo, hi], p in {2, 3}, tau uniform in [1e-3, 5e-3],
    Gaussian pulse sigma = 0.05 at a random centre in [0.25, 0.75]^3."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        ne = tuple(int(v) for v in rng.integers(lo, hi + 1, 3))
        p = int(rng.choice([2, 3]))
        tau = float(rng.uniform(1e-3, 5e-3))
        c = tuple(float(v) for v in rng.uniform(0.25, 0.75, 3))
        out.append(WaveCase("batch%d" % i, ne, p, tau, steps,
                            u0=dict(amp=1.0, center=c, den=2.0 * sigma ** 2)))
    return out


@dataclass
class Request:
    rid: int
    arrival: float
    kind: str
    n_elem: tuple
    p: int
    tau: float
    steps: int
    source: dict = field(default_factory=dict)


def serving_requests(count=500, rate=20.0, seed=0, lo=24, hi=256, frac_wave=0.8, max_steps=500):
    """Poisson arrivals (mean `rate` per second); 80% P-wave / 20% elasticity;
    elements per axis iid log-uniform in [lo, hi]; p in {2, 3}; steps uniform
    in [10, max_steps]; tau in [1e-3, 5e-3]; Ricker (f in [4, 12]) times a
    Gaussian (sigma in [0.02, 0.05]) at a random point."""
    rng = np.random.default_rng(seed)
    t = 0.0
    reqs = []
    for i in range(count):
        t += float(rng.exponential(1.0 / rate))
        kind = "wave" if rng.uniform() < frac_wave else "elastic"
        ne = tuple(int(round(v)) for v in np.exp(rng.uniform(np.log(lo), np.log(hi), 3)))
        p = int(rng.choice([2, 3]))
        steps = int(rng.integers(10, max_steps + 1))
        tau = float(rng.uniform(1e-3, 5e-3))
        f = float(rng.uniform(4.0, 12.0))
        sig = float(rng.uniform(0.02, 0.05))
        c = tuple(float(v) for v in rng.uniform(0.25, 0.75, 3))
        d = unit_vector(seed * 100003 + i)
        src = dict(amp=1.0, center=c, den=2.0 * sig ** 2, freq=f, t0=1.0 / f, dir=d)
        reqs.append(Request(i, t, kind, ne, p, tau, steps, src))
    return reqs
