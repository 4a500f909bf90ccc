"""Pins of the oracle's FokkerPlanckMap (Eq. VFP right-hand side, Eq. cubic
diff) and WakeKickMap (Sec. III.B) against printed stencils, exactness on
polynomials, conservation and the dense-matrix restatement."""
import os

import numpy as np
import pytest

from oracle import brute as B
from oracle import oracle as O
from paper_1611_05293_b300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _impulse_response(pr, y0):
    """Column of the FP map: output increment when psi is a unit impulse."""
    n = pr.n
    f = np.zeros((n, n))
    f[n // 2, y0] = 1.0
    return O.fokker_planck(pr, f)[n // 2] - f[n // 2]


def test_cubic_derivative_matches_printed_stencil():
    """With the second difference and psi-term removed (p=0 row, h scaled out),
    the FP increment's derivative part equals Eq. cubic diff as printed."""
    rows = np.loadtxt(os.path.join(GOLDEN, "cubic_diff_stencil.txt"))
    printed = {int(o): c / 6.0 for o, c in rows}
    n = 21
    pr = O.Params(n=n, steps_per_period=1, beta=1.0, half_width=10.0)  # Delta = 1
    # p_y = -10 + y: use two rows with different p to isolate p*D1
    resp = {}
    for y in (5, 15):
        # the target row y receives sum_k c_k f(y+k): impulse at y+k gives coefficient
        resp[y] = {k: _impulse_response(pr, y + k)[y] for k in (-1, 0, 1, 2)}
    p5, p15 = -10 + 5, -10 + 15
    for k in (-1, 0, 1, 2):
        d1 = (resp[15][k] - resp[5][k]) / (p15 - p5)       # coefficient of p
        assert abs(d1 - printed[k]) < 1e-14
    assert np.allclose(B.derivative_stencil(1)[1], [printed[k] for k in (-1, 0, 1, 2)], atol=1e-14)


@pytest.mark.parametrize("fpd,deg", [(1, 3), (0, 2)])
def test_fp_exact_on_polynomials(fpd, deg):
    """psi polynomial in p of degree <= 3 (cubic derivative) or <= 2 (central):
    the step equals psi + h (psi + p psi' + psi'') exactly away from the edges."""
    n, L = 40, 6.0
    pr = O.Params(n=n, steps_per_period=10, beta=0.7, fp_derivative=fpd)
    p = W.grid_axis(n, L)
    c = [0.3, -0.2, 0.05, 0.01][: deg + 1]
    f = sum(ci * p ** i for i, ci in enumerate(c))
    d1 = sum(i * ci * p ** (i - 1) for i, ci in enumerate(c) if i >= 1)
    d2 = sum(i * (i - 1) * ci * p ** (i - 2) for i, ci in enumerate(c) if i >= 2)
    psi = np.tile(f, (n, 1))
    out = O.fokker_planck(pr, psi)
    h = pr.beta / pr.steps_per_period
    ref = f + h * (f + p * d1 + d2)
    inner = slice(2, n - 3)
    assert np.max(np.abs(out[:, inner] - ref[inner])) < 1e-12


def test_fp_conserves_charge():
    """Sum_y of (psi + p D1 psi + D2 psi) vanishes for both D1 rules when psi
    is zero near the edges (telescoping of the stencils)."""
    n = 64
    g = W.blobs(n, 7)
    g[:, :4] = 0
    g[:, -4:] = 0
    for fpd in (0, 1):
        pr = O.Params(n=n, steps_per_period=100, beta=3.0, fp_derivative=fpd)
        out = O.fokker_planck(pr, g)
        assert abs(out.sum() - g.sum()) < 1e-12 * g.sum()


def test_fp_gaussian_equilibrium_residual_is_second_order():
    """exp(-p^2/2) solves p psi + psi' = 0; the discrete residual is the
    O(Delta^2) error of the second difference (and O(Delta^3) of D1)."""
    res = []
    for n in (65, 129, 257):
        pr = O.Params(n=n, steps_per_period=1, beta=1.0)
        g = np.tile(np.exp(-0.5 * W.grid_axis(n) ** 2), (4, 1))
        pr.n = n
        psi = np.zeros((n, n))
        psi[:4] = g
        out = O.fokker_planck(pr, psi)
        res.append(np.max(np.abs(out[:4] - psi[:4])))
    orders = np.log2(np.array(res[:-1]) / np.array(res[1:]))
    assert np.all(orders > 1.9), (res, orders)


def test_fp_matches_dense_matrix():
    for n, fpd in ((9, 1), (12, 0)):
        pr = O.Params(n=n, steps_per_period=7, beta=0.4, fp_derivative=fpd)
        f = W.random_field(n, 11)
        A = B.fokker_planck_matrix(n, 6.0, 7, 0.4, fpd)
        assert np.max(np.abs(O.fokker_planck(pr, f) - (A @ f.ravel()).reshape(n, n))) < 1e-13


def test_kick_integer_shift_is_exact():
    """dp/Delta = S V phi/Delta an integer: the kick is an exact index shift
    (y_r = y - dp/Delta), zero-filled at the edge."""
    n = 32
    pr = O.Params(n=n, steps_per_period=50, s_csr=1.0)
    phi = 2 * np.pi / 50
    shifts = np.array([(x % 5) - 2 for x in range(n)], dtype=float)   # cells
    V = shifts * pr.delta / (pr.s_csr * phi)
    f = W.random_field(n, 4)
    out = O.kick(pr, V, f)
    for x in range(n):
        s = int(shifts[x])
        ref = np.zeros(n)
        for y in range(n):
            if 0 <= y - s < n:
                ref[y] = f[x, y - s]
        assert np.max(np.abs(out[x] - ref)) < 1e-13


def test_kick_exact_on_cubic_profiles():
    """A fractional shift of a cubic in p is exact away from the edges."""
    n = 48
    pr = O.Params(n=n, steps_per_period=40, s_csr=0.8)
    phi = 2 * np.pi / 40
    p = W.grid_axis(n)
    V = np.linspace(-1.0, 1.5, n)
    dp = pr.s_csr * V * phi
    f = np.tile(0.2 + 0.1 * p - 0.03 * p ** 2 + 0.002 * p ** 3, (n, 1))
    out = O.kick(pr, V, f)
    for x in range(n):
        ps = p - dp[x]
        ref = 0.2 + 0.1 * ps - 0.03 * ps ** 2 + 0.002 * ps ** 3
        inner = (ps > p[0] + 2 * pr.delta) & (ps < p[-1] - 3 * pr.delta)
        assert np.max(np.abs(out[x][inner] - ref[inner])) < 1e-12


def test_kick_matches_dense_matrix():
    n = 11
    pr = O.Params(n=n, steps_per_period=9, s_csr=2.5)
    V = np.random.default_rng(3).normal(size=n)
    f = W.random_field(n, 12)
    A = B.kick_matrix(n, 6.0, 9, V, 2.5)
    assert np.max(np.abs(O.kick(pr, V, f) - (A @ f.ravel()).reshape(n, n))) < 1e-14
