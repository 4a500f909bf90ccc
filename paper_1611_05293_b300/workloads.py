"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle runs.

This module holds no step arithmetic of the solver: it only draws starting
densities and parameter sets (NumPy PCG64, fixed seeds) with the shapes of
the paper's workloads, so that the CUDA path and the CPU oracle can be fed
identical inputs.  Densities are returned un-normalised; both solvers
normalise the charge to 1 themselves.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

__all__ = ["grid_axis", "gaussian", "noisy_gaussian", "random_field", "blobs",
           "scan_grid", "Request", "request_stream"]


def grid_axis(n: int, half_width: float = 6.0) -> np.ndarray:
    """Node coordinates -L + i*2L/(n-1), i = 0..n-1 (same for q and p)."""
    return -half_width + np.arange(n) * (2.0 * half_width / (n - 1))


def gaussian(n: int, half_width: float = 6.0, sigma_q: float = 1.0, sigma_p: float = 1.0,
             q0: float = 0.0, p0: float = 0.0) -> np.ndarray:
    """exp(-(q-q0)^2/2sq^2 - (p-p0)^2/2sp^2) sampled at the nodes, [q][p] layout."""
    x = grid_axis(n, half_width)
    gq = np.exp(-0.5 * ((x - q0) / sigma_q) ** 2)
    gp = np.exp(-0.5 * ((x - p0) / sigma_p) ** 2)
    return np.outer(gq, gp)


def noisy_gaussian(n: int, seed: int, eps: float = 1e-6, half_width: float = 6.0,
                   sigma: float = 1.0) -> np.ndarray:
    """Gaussian plus eps*max*U(-1,1) noise, clipped at zero (seeded)."""
    g = gaussian(n, half_width, sigma, sigma)
    rng = np.random.Generator(np.random.PCG64(seed))
    g = g + eps * g.max() * rng.uniform(-1.0, 1.0, size=g.shape)
    return np.clip(g, 0.0, None)


def random_field(n: int, seed: int) -> np.ndarray:
    """Uniform U(0,1) values on every node, including the boundary."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.uniform(0.0, 1.0, size=(n, n))


def blobs(n: int, seed: int, count: int = 6, half_width: float = 6.0) -> np.ndarray:
    """Sum of a few random Gaussian blobs: smooth but asymmetric structure."""
    rng = np.random.Generator(np.random.PCG64(seed))
    x = grid_axis(n, half_width)
    out = np.zeros((n, n))
    for _ in range(count):
        q0, p0 = rng.uniform(-2.5, 2.5, size=2)
        sq, sp = rng.uniform(0.4, 1.5, size=2)
        a = rng.uniform(0.2, 1.0)
        out += a * np.outer(np.exp(-0.5 * ((x - q0) / sq) ** 2), np.exp(-0.5 * ((x - p0) / sp) ** 2))
    return out


def scan_grid(n_s: int = 21, pis=(1.0, 2.0, 3.0), s_lo: float = 0.2, s_hi: float = 1.5,
              duplicate=(0.785, 2.0)):
    """(S_csr, Pi) pairs of a threshold scan: n_s x len(pis) points, plus one
    duplicate point used as an in-batch determinism probe."""
    pts = [(float(s), float(pi)) for pi in pis for s in np.linspace(s_lo, s_hi, n_s)]
    if duplicate is not None:
        pts.append((float(duplicate[0]), float(duplicate[1])))
    return pts


@dataclass
class Request:
    """One simulation request of a served parameter scan."""
    rid: int
    arrival_s: float
    n: int
    s_csr: float
    Pi: float
    steps_per_period: int
    periods: int

    @property
    def nsteps(self) -> int:
        return self.steps_per_period * self.periods

    @property
    def cell_updates(self) -> int:
        return self.n * self.n * self.nsteps


def request_stream(count: int, rate_per_s: float, seed: int,
                   sizes=(128, 256, 512, 1024), s_range=(0.2, 2.0), pi_range=(0.5, 4.0),
                   steps_range=(1000, 4000), periods_range=(5, 50)):
    """Poisson arrivals of requests with uneven grid sizes and run lengths."""
    rng = np.random.Generator(np.random.PCG64(seed))
    t = 0.0
    out = []
    for i in range(count):
        t += rng.exponential(1.0 / rate_per_s)
        out.append(Request(
            rid=i, arrival_s=t, n=int(rng.choice(sizes)),
            s_csr=float(rng.uniform(*s_range)), Pi=float(rng.uniform(*pi_range)),
            steps_per_period=int(rng.integers(steps_range[0], steps_range[1] + 1)),
            periods=int(rng.integers(periods_range[0], periods_range[1] + 1))))
    return out
