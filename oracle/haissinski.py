"""Haissinski equilibrium for the oracle (Appendix A of the paper names it;
the equation itself is the textbook one and is not printed there).

TEST INFRASTRUCTURE ONLY.

Below the instability threshold the damped, diffused system relaxes to
psi proportional to exp(-H) with H = (q^2 + p^2)/2 - S_csr Phi(q), where
Phi' = V (the wake potential of the profile itself, Eq. wakepotential) so
that dp/dtheta = -dH/dq = -q + S_csr V(q) is the kick of the time step.
The profile therefore solves the fixed-point equation

    rho(q) = A exp(-q^2/2 + S_csr int_{-L}^{q} V[rho](q') dq'),   int rho dq = 1,

which is solved here by damped iteration on the solver's own grid, with
the oracle's wake (direct DFT) and the trapezoid rule for the integral.
"""
from __future__ import annotations

import numpy as np

from . import oracle as _o


def profile(pr: "_o.Params", zre, zim, tol: float = 1e-13, damping: float = 0.5,
            max_iter: int = 20000) -> np.ndarray:
    """Haissinski profile rho_H on the grid nodes (rectangle-rule charge 1)."""
    n, d = pr.n, pr.delta
    q = -pr.half_width + d * np.arange(n)
    base = np.exp(-0.5 * q * q)
    rho = base / (d * base.sum())
    for _ in range(max_iter):
        V, _P = _o.wake(pr, zre, zim, rho)
        phi = np.concatenate(([0.0], np.cumsum(0.5 * d * (V[1:] + V[:-1]))))
        expo = -0.5 * q * q + pr.s_csr * phi
        new = np.exp(expo - expo.max())
        new /= d * new.sum()
        err = np.max(np.abs(new - rho)) / np.max(rho)
        rho = (1.0 - damping) * rho + damping * new
        if err < tol:
            return rho
    raise RuntimeError("Haissinski iteration did not converge")


def density(pr: "_o.Params", zre, zim, **kw) -> np.ndarray:
    """psi_H(q, p) = rho_H(q) exp(-p^2/2) on the grid, normalised to charge 1."""
    rho = profile(pr, zre, zim, **kw)
    d = pr.delta
    p = -pr.half_width + d * np.arange(pr.n)
    g = np.exp(-0.5 * p * p)
    psi = np.outer(rho, g / (d * g.sum()))
    return psi
