"""Pins of the oracle's Manhattan rotation (Sec. III.B, symplectic rotation:
an energy-dependent drift followed by a location-dependent RF kick, each a
1-D interpolation) against an exact node permutation, polynomial exactness,
charge conservation, the dense-matrix restatement and the full-turn
convergence order."""
import math

import numpy as np
import pytest

from oracle import brute as B
from oracle import oracle as O
from paper_1611_05293_b300 import workloads as W


def test_step_parameter_turns_one_period():
    """h = 2 sin(pi/steps): the drift-kick matrix [[1, h], [-h, 1 - h^2]] has
    unit determinant, and its steps-th power is the identity."""
    for steps in (6, 7, 50, 1000):
        pr = O.Params(steps_per_period=steps)
        h = O.manhattan_h(pr)
        assert abs(h - 2 * math.sin(math.pi / steps)) < 1e-15
        Mx = np.array([[1.0, h], [-h, 1.0 - h * h]])
        assert abs(np.linalg.det(Mx) - 1.0) < 1e-14
        assert np.max(np.abs(np.linalg.matrix_power(Mx, steps) - np.eye(2))) < 1e-9


@pytest.mark.parametrize("n", [9, 13])
def test_sixth_turn_is_a_permutation(n):
    """steps_per_period = 6 gives h = 1; with n odd the grid centre c is a node
    and every drift and RF-kick shift is a whole number of cells, so one
    Manhattan rotation maps nodes onto nodes:
    psi_b(x, y) = psi(2c - y, x + y - c), zero where that source is off the grid."""
    pr = O.Params(n=n, steps_per_period=6, rotation=1)
    f = W.random_field(n, 11)
    out = O.rfkick(pr, O.drift(pr, f))
    c = (n - 1) // 2
    ref = np.zeros_like(f)
    for x in range(n):
        for y in range(n):
            xs, ys = 2 * c - y, x + y - c
            if 0 <= xs < n and 0 <= ys < n:
                ref[x, y] = f[xs, ys]
    assert np.max(np.abs(out - ref)) < 1e-12


def test_drift_and_kick_exact_on_cubics():
    """Cubic interpolation is exact on cubics, so the drift of g(q) h(p) is
    g(q - h p) h(p) and the RF kick of g(q) k(p) is g(q) k(p + h q) wherever the
    stencil stays inside the grid."""
    n, L, steps = 40, 6.0, 37
    pr = O.Params(n=n, steps_per_period=steps, half_width=L, rotation=1)
    h = O.manhattan_h(pr)
    q = W.grid_axis(n, L)
    Q, P = np.meshgrid(q, q, indexing="ij")

    def g(a):
        return 0.3 - 0.2 * a + 0.05 * a * a + 0.01 * a ** 3

    def k(b):
        return np.cos(b)  # any function of the untouched coordinate

    d1 = O.drift(pr, g(Q) * k(P))
    inner = np.abs(Q - h * P) < L - 3 * pr.delta
    assert np.max(np.abs(d1 - g(Q - h * P) * k(P))[inner]) < 1e-12
    d2 = O.rfkick(pr, k(Q) * g(P))
    inner = np.abs(P + h * Q) < L - 3 * pr.delta
    assert np.max(np.abs(d2 - k(Q) * g(P + h * Q))[inner]) < 1e-12


def test_charge_conserved():
    """Each 1-D pass moves a row (or column) by one shift, and Lagrange weights
    sum to 1, so a distribution away from the edges keeps its charge."""
    n = 96
    pr = O.Params(n=n, steps_per_period=100, rotation=1)
    f = W.gaussian(n, 6.0, 0.6, 0.6)  # ~exp(-50) at the edges
    out = O.rfkick(pr, O.drift(pr, f))
    assert abs(out.sum() / f.sum() - 1.0) < 1e-13


@pytest.mark.parametrize("n,steps,ni", [(9, 7, 4), (12, 23, 4), (10, 9, 3), (11, 5, 2)])
def test_manhattan_step_matches_dense_matrices(n, steps, ni):
    """Full step (wake, Manhattan rotation, kick, Fokker-Planck, renormalisation)
    against the dense-matrix restatement."""
    L, beta, S, Pi = 6.0, 0.05, 0.7, 2.0
    pr = O.Params(n=n, steps_per_period=steps, interp_points=ni, beta=beta, s_csr=S, rotation=1)
    zr, zi = O.impedance(pr, 2, Pi)
    f = O.normalize(pr, W.random_field(n, 5) + 0.1)
    out, V, P = O.step(pr, zr, zi, f)[:3]
    ref, Vb, Pb = B.step(n, L, steps, beta, S, 2, zr, zi, f, ni=ni, rotation=1)
    assert np.max(np.abs(out - ref)) < 1e-12 * max(1.0, np.max(np.abs(ref)))


def test_full_turn_returns_with_fourth_order_error():
    """No wake, beta = 0: steps_per_period Manhattan steps are one full turn, so
    a Gaussian comes back to itself up to the interpolation error, which falls
    as Delta^4 (two 1-D cubic passes per step)."""
    errs = []
    for n in (48, 96, 192):
        pr = O.Params(n=n, steps_per_period=40, beta=0.0, renormalize=0, rotation=1)
        f = W.gaussian(n, 6.0, 1.0, 1.0)
        g = f.copy()
        for _ in range(40):
            g = O.rfkick(pr, O.drift(pr, g))
        errs.append(np.max(np.abs(g - f)) / f.max())
    order = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert errs[-1] < 1e-4  # measured 6.8e-5 at n = 192 (standard rotation: 6.4e-5)
    assert min(order) > 3.3, (errs, order)
