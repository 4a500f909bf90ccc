"""Pins of the oracle's RotationMap (Sec. III.B, standard rotation) against
exact permutations, polynomial exactness, the dense-matrix restatement and
the interpolation-error convergence order."""
import numpy as np
import pytest

from oracle import brute as B
from oracle import oracle as O
from paper_1611_05293_b300 import workloads as W


@pytest.mark.parametrize("n", [8, 9, 16])
def test_quarter_turn_is_a_permutation(n):
    """steps_per_period = 4 rotates by 90 degrees: nodes map onto nodes,
    psi_new[x][y] = psi[n-1-y][x] (source of (q, p) is (-p, q))."""
    pr = O.Params(n=n, steps_per_period=4)
    f = W.random_field(n, 1)
    out = O.rotate(pr, f)
    ref = np.empty_like(f)
    for x in range(n):
        for y in range(n):
            ref[x, y] = f[n - 1 - y, x]
    assert np.max(np.abs(out - ref)) < 1e-13


@pytest.mark.parametrize("n", [8, 13])
def test_half_turn_is_a_point_reflection(n):
    pr = O.Params(n=n, steps_per_period=2)
    f = W.random_field(n, 2)
    out = O.rotate(pr, f)
    assert np.max(np.abs(out - f[::-1, ::-1])) < 1e-13


def test_rotation_exact_on_bicubic_polynomials():
    """Bicubic interpolation reproduces x^a y^b (a, b <= 3) exactly, so a
    rotated polynomial equals the polynomial at the rotated-back point for
    targets whose stencil lies inside the grid."""
    n, L, steps = 24, 6.0, 37
    pr = O.Params(n=n, steps_per_period=steps, half_width=L)
    q = W.grid_axis(n, L)
    Q, P = np.meshgrid(q, q, indexing="ij")

    def f(a, b):
        return 0.2 + 0.1 * a - 0.3 * b + 0.02 * a ** 3 - 0.01 * a * b * b + 1e-3 * a ** 3 * b ** 2

    out = O.rotate(pr, f(Q, P))
    phi = 2 * np.pi / steps
    Qs = Q * np.cos(phi) - P * np.sin(phi)
    Ps = Q * np.sin(phi) + P * np.cos(phi)
    ref = f(Qs, Ps)
    inner = (np.abs(Qs) < L - 3 * pr.delta) & (np.abs(Ps) < L - 3 * pr.delta)
    assert inner.sum() > 100
    assert np.max(np.abs(out - ref)[inner]) < 1e-11


@pytest.mark.parametrize("n,steps,ni", [(8, 7, 4), (11, 23, 4), (10, 9, 3), (9, 5, 2)])
def test_rotation_matches_dense_matrix(n, steps, ni):
    pr = O.Params(n=n, steps_per_period=steps, interp_points=ni)
    f = W.random_field(n, 3)
    A = B.rotation_matrix(n, 6.0, steps, ni)
    assert np.max(np.abs(O.rotate(pr, f) - (A @ f.ravel()).reshape(n, n))) < 1e-14


def test_full_turn_returns_gaussian_with_fourth_order_error():
    """No wake, beta = 0: steps_per_period steps make exactly one turn, which
    maps the round Gaussian onto itself.  The remaining error is the
    accumulated cubic-interpolation error, O(Delta^4) per step; halving Delta
    must cut it by about 2^4 once the grid resolves the Gaussian."""
    errs = []
    steps = 16
    for n in (65, 129, 257):
        pr = O.Params(n=n, steps_per_period=steps, beta=0.0)
        g = W.gaussian(n, 6.0)
        f = g.copy()
        for _ in range(steps):
            f = O.rotate(pr, f)
        errs.append(np.max(np.abs(f - g)) / g.max())
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    # stated interpolation error after one turn in 16 steps at N = 257: < 1e-5
    assert errs[-1] < 1e-5, errs
    assert np.all(orders > 3.7), (errs, orders)
