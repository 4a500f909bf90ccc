"""Pins of the oracle's interpolation (Sec. III.A: Eqs. interpolation,
lagrange-basis-polynomials, clamping) against closed forms and invariants."""
import math

import numpy as np
import pytest

from oracle import oracle as O


@pytest.mark.parametrize("ni", [2, 3, 4])
@pytest.mark.parametrize("t", [0.0, 0.1, 0.37, 0.5, 0.93])
def test_lagrange_reproduces_polynomials(ni, t):
    """Weights are exact on every polynomial of degree < N_I (defining property
    of the interpolating polynomial through N_I nodes)."""
    w = O.lagrange(ni, t)
    first = -((ni - 1) // 2)
    m = np.arange(first, first + ni, dtype=float)
    for deg in range(ni):
        assert abs(np.dot(w, m ** deg) - t ** deg) < 1e-14


def test_lagrange_textbook_values():
    """Cubic weights at the midpoint are (-1, 9, 9, -1)/16; at t=0 the node
    value is returned; quadratic at t=1/2 is (-1, 6, 3)/8 on nodes -1, 0, 1;
    linear is (1-t, t)."""
    assert np.allclose(O.lagrange(4, 0.5), np.array([-1, 9, 9, -1]) / 16.0, atol=1e-16)
    assert np.allclose(O.lagrange(4, 0.0), [0, 1, 0, 0], atol=0)
    assert np.allclose(O.lagrange(3, 0.5), np.array([-1, 6, 3]) / 8.0, atol=1e-16)
    assert np.allclose(O.lagrange(2, 0.3), [0.7, 0.3], atol=1e-16)


def test_lagrange_cubic_closed_form():
    """Cubic weights on nodes -1..2 equal the closed forms
    -t(t-1)(t-2)/6, (t+1)(t-1)(t-2)/2, -(t+1)t(t-2)/2, (t+1)t(t-1)/6."""
    for t in np.linspace(0, 1, 17):
        ref = [-t * (t - 1) * (t - 2) / 6, (t + 1) * (t - 1) * (t - 2) / 2,
               -(t + 1) * t * (t - 2) / 2, (t + 1) * t * (t - 1) / 6]
        assert np.allclose(O.lagrange(4, t), ref, atol=1e-15)


def _poly_grid(n, coef):
    x = np.arange(n, dtype=float)
    X, Y = np.meshgrid(x, x, indexing="ij")
    f = np.zeros((n, n))
    for (a, b), c in coef.items():
        f += c * X ** a * Y ** b
    return f


def test_interp2_exact_on_bicubics():
    """Tensor-product cubic interpolation is exact for x^a y^b with a, b <= 3
    whenever the 4x4 stencil lies inside the grid."""
    n = 12
    coef = {(0, 0): 0.3, (1, 0): -0.2, (0, 1): 0.7, (3, 0): 0.01, (0, 3): -0.02,
            (2, 1): 0.05, (1, 2): 0.03, (3, 3): 1e-4, (2, 2): -2e-3}
    f = _poly_grid(n, coef)
    pr = O.Params(n=n)
    rng = np.random.default_rng(0)
    for _ in range(50):
        xr, yr = rng.uniform(1.0, n - 3.0, size=2)
        ref = sum(c * xr ** a * yr ** b for (a, b), c in coef.items())
        assert abs(O.interp2(pr, f, xr, yr) - ref) < 1e-11 * max(1.0, abs(ref))


def test_interp2_zero_outside_and_cutoff():
    """Off-grid nodes are zero; a source more than one cell outside gives 0."""
    n = 8
    f = np.ones((n, n))
    pr = O.Params(n=n)
    assert O.interp2(pr, f, -1.01, 3.0) == 0.0
    assert O.interp2(pr, f, 3.0, n + 0.01) == 0.0
    # inside one cell of the edge: partial stencil, weights of the in-grid nodes
    v = O.interp2(pr, f, -0.5, 3.0)
    w = O.lagrange(4, 0.5)
    assert abs(v - (w[2] + w[3])) < 1e-15


def test_clamp_is_identity_between_nodes_and_cuts_overshoot():
    """Clamped interpolation (Eq. clamping, read as min{max[P, min(a,b)], max(a,b)})
    leaves values inside [min, max] of the nearest nodes unchanged and cuts
    overshoots to that range."""
    n = 10
    x = np.arange(n, dtype=float)
    smooth = np.outer(np.exp(-0.1 * (x - 4.5) ** 2), np.ones(n))
    p0 = O.Params(n=n, clamp=0)
    p1 = O.Params(n=n, clamp=1)
    # monotone region: interpolant lies between the nodes -> unchanged
    assert O.interp2(p1, smooth, 2.3, 4.0) == O.interp2(p0, smooth, 2.3, 4.0)
    # a step: cubic overshoots next to the jump; the clamp removes it
    step = np.zeros((n, n))
    step[5:, :] = 1.0
    raw = O.interp2(p0, step, 5.5, 4.0)
    assert raw > 1.0
    assert O.interp2(p1, step, 5.5, 4.0) == 1.0
    raw = O.interp2(p0, step, 3.5, 4.0)
    assert raw < 0.0
    assert O.interp2(p1, step, 3.5, 4.0) == 0.0
