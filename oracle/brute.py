"""Dense-matrix restatement of one time step for tiny grids (n <= 16).

TEST INFRASTRUCTURE ONLY.  A second, deliberately different route to the
same definitions as vfps_oracle.c, used to pin it:

* interpolation weights come from solving the Vandermonde system of the
  nodes (the polynomial through the N_I nodes evaluated at t), not from the
  Lagrange product formula;
* each map is assembled as an explicit (n*n) x (n*n) matrix acting on the
  flattened index z = n*x + y (the paper's source-map picture, Sec. III.B)
  and applied by a matrix-vector product;
* the derivative stencils come from differentiating the interpolating
  polynomial (Eq. cubic diff: the cubic through y-1..y+2; the central
  difference: the quadratic through y-1..y+1);
* the Fourier sums are dense complex exponential matrices.
Clamping is not modelled here (it is non-linear); the C oracle's clamp has
its own tests.
"""
from __future__ import annotations

import math

import numpy as np


def nodes(ni: int) -> np.ndarray:
    first = -((ni - 1) // 2)
    return np.arange(first, first + ni, dtype=np.float64)


def weights(ni: int, t: float) -> np.ndarray:
    """w with sum_k w_k f(m_k) = P(t) for the polynomial P through the nodes."""
    m = nodes(ni)
    V = np.vander(m, ni, increasing=True)          # V[k, j] = m_k^j
    return np.linalg.solve(V.T, t ** np.arange(ni))


def derivative_stencil(kind: int) -> tuple[np.ndarray, np.ndarray]:
    """(offsets, coefficients) of P'(0) for the interpolating polynomial."""
    m = np.array([-1.0, 0.0, 1.0, 2.0]) if kind == 1 else np.array([-1.0, 0.0, 1.0])
    k = len(m)
    V = np.vander(m, k, increasing=True)
    e = np.zeros(k)
    e[1] = 1.0                                      # d/dt t^j at 0: only j = 1
    return m.astype(int), np.linalg.solve(V.T, e)


def _interp_rows(n, ni, r):
    """list of (node index, weight) for a 1-D source coordinate r (grid units)."""
    if r < -1.0 or r > n:
        return []
    m = math.floor(r)
    w = weights(ni, r - m)
    return [(m + int(o), wk) for o, wk in zip(nodes(ni), w) if 0 <= m + int(o) < n]


def rotation_matrix(n, L, steps, ni=4):
    d = 2 * L / (n - 1)
    phi = 2 * np.pi / steps
    R = np.array([[np.cos(phi), -np.sin(phi)], [np.sin(phi), np.cos(phi)]])
    A = np.zeros((n * n, n * n))
    for x in range(n):
        for y in range(n):
            src = R @ np.array([-L + x * d, -L + y * d])
            xr, yr = (src + L) / d
            for ix, wx in _interp_rows(n, ni, xr):
                for iy, wy in _interp_rows(n, ni, yr):
                    A[n * x + y, n * ix + iy] += wx * wy
    return A


def manhattan_matrices(n, L, steps, ni=4):
    """(drift, RF kick) matrices of the Manhattan rotation.  The step h is
    taken from the composite linear map [[1, h], [-h, 1 - h^2]] turning by
    2 pi/steps: trace 2 - h^2 = 2 cos(2 pi/steps)."""
    d = 2 * L / (n - 1)
    h = math.sqrt(2.0 - 2.0 * math.cos(2 * math.pi / steps))
    Dm = np.zeros((n * n, n * n))
    Km = np.zeros((n * n, n * n))
    for x in range(n):
        for y in range(n):
            q, p = -L + x * d, -L + y * d
            for ix, w in _interp_rows(n, ni, (q - h * p + L) / d):    # drift: q -> q + h p
                Dm[n * x + y, n * ix + y] += w
            for iy, w in _interp_rows(n, ni, (p + h * q + L) / d):    # RF kick: p -> p - h q
                Km[n * x + y, n * x + iy] += w
    return Dm, Km


def kick_matrix(n, L, steps, V, s_csr, ni=4):
    d = 2 * L / (n - 1)
    phi = 2 * np.pi / steps
    A = np.zeros((n * n, n * n))
    for x in range(n):
        shift = s_csr * V[x] * phi / d             # dp in grid cells
        for y in range(n):
            for iy, w in _interp_rows(n, ni, y - shift):
                A[n * x + y, n * x + iy] += w
    return A


def fokker_planck_matrix(n, L, steps, beta, kind=1):
    d = 2 * L / (n - 1)
    h = beta / steps
    off1, c1 = derivative_stencil(kind)
    off2, c2 = np.array([-1, 0, 1]), np.array([1.0, -2.0, 1.0])
    A = np.eye(n * n)
    for x in range(n):
        for y in range(n):
            p = -L + y * d
            row = n * x + y
            A[row, row] += h
            for o, c in zip(off1, c1):
                if 0 <= y + o < n:
                    A[row, n * x + y + o] += h * p * c / d
            for o, c in zip(off2, c2):
                if 0 <= y + o < n:
                    A[row, n * x + y + o] += h * c / (d * d)
    return A


def wake(n, L, pad, zre, zim, rho):
    """(V, P) with dense exponential matrices over k = -(M/2-1)..(M/2-1)."""
    d = 2 * L / (n - 1)
    M = 1 << int(np.ceil(np.log2(pad * n)))   # smallest power of two >= pad*n
    dk = 2 * np.pi / (M * d)
    K = M // 2
    z = np.asarray(zre) + 1j * np.asarray(zim)
    ks = np.arange(-(K - 1), K)                     # Nyquist dropped
    zfull = np.where(ks >= 0, z[np.abs(ks)], np.conj(z[np.abs(ks)]))
    i = np.arange(n)
    F = np.exp(-2j * np.pi * np.outer(ks, i) / M)   # forward
    rt = d * (F @ rho)
    Vc = dk * (np.exp(2j * np.pi * np.outer(i, ks) / M) @ (zfull * rt))
    P = dk * np.sum(zfull.real * np.abs(rt) ** 2)
    return Vc.real, P


def step(n, L, steps, beta, s_csr, pad, zre, zim, psi, ni=4, kind=1, renorm=True, rotation=0):
    """One step: returns (psi_next, V, P).  rotation 1 = Manhattan."""
    d = 2 * L / (n - 1)
    f = np.asarray(psi, dtype=np.float64).reshape(n * n)
    rho = d * f.reshape(n, n).sum(axis=1)
    V, P = wake(n, L, pad, zre, zim, rho)
    if rotation == 1:
        Dm, Km = manhattan_matrices(n, L, steps, ni)
        a = Km @ (Dm @ f)
    else:
        a = rotation_matrix(n, L, steps, ni) @ f
    b = kick_matrix(n, L, steps, V, s_csr, ni) @ a
    c = fokker_planck_matrix(n, L, steps, beta, kind) @ b
    if renorm:
        c = c / (d * d * c.sum())
    return c.reshape(n, n), V, P
