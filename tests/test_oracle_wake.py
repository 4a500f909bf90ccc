"""Pins of the oracle's wake potential, CSR power (Eq. wakepotential,
Sec. IV.C) and impedances (Sec. II.B) against closed forms, identities and
an independent arbitrary-precision evaluation."""
import math

import mpmath as mp
import numpy as np
import pytest

from oracle import brute as B
from oracle import impedance as I
from oracle import oracle as O
from paper_1611_05293_b300 import workloads as W


def _rho(n, seed):
    return np.random.default_rng(seed).uniform(0.0, 1.0, n)


@pytest.mark.parametrize("n,pad", [(16, 2), (37, 2), (64, 4)])
def test_constant_real_impedance_closed_form(n, pad):
    """Zhat_k = 1 for every k: with sum_{k=1}^{M/2-1} cos(k x) =
    (M delta_{m,0} - 1 - (-1)^m)/2 for x = 2 pi m/M, the wake is
    V_i = 2 pi rho_i - (2 pi/M) sum_j rho_j (1 + (-1)^(i-j))."""
    pr = O.Params(n=n, pad_factor=pad)
    M = pr.M
    zr, zi = np.ones(M // 2 + 1), np.zeros(M // 2 + 1)
    rho = _rho(n, 1)
    V, _ = O.wake(pr, zr, zi, rho)
    i = np.arange(n)
    sign = (-1.0) ** (i[:, None] - i[None, :])
    ref = 2 * np.pi * rho - (2 * np.pi / M) * ((1 + sign) @ rho)
    assert np.max(np.abs(V - ref)) < 1e-12 * np.max(np.abs(ref))


@pytest.mark.parametrize("n,pad", [(16, 2), (41, 2)])
def test_constant_imaginary_impedance_closed_form(n, pad):
    """Zhat_k = i: V_i = -2 dkappa Delta sum_j rho_j S(i-j) with Lagrange's
    identity S(m) = sum_{k=1}^{K-1} sin(k x) = sin((K-1)x/2) sin(Kx/2)/sin(x/2),
    x = 2 pi m/M, K = M/2.  Pins the sign of the phase exp(+i kappa q)."""
    pr = O.Params(n=n, pad_factor=pad)
    M, K, d = pr.M, pr.M // 2, pr.delta
    dk = 2 * np.pi / (M * d)
    zr, zi = np.zeros(K + 1), np.ones(K + 1)
    rho = _rho(n, 2)
    V, _ = O.wake(pr, zr, zi, rho)
    i = np.arange(n)
    m = i[:, None] - i[None, :]
    x = 2 * np.pi * m / M
    with np.errstate(invalid="ignore", divide="ignore"):
        S = np.where(m == 0, 0.0, np.sin((K - 1) * x / 2) * np.sin(K * x / 2) / np.sin(x / 2))
    ref = -2 * dk * d * (S @ rho)
    assert np.max(np.abs(V - ref)) < 1e-12 * np.max(np.abs(ref))


@pytest.mark.parametrize("model,Pi", [(1, 0.0), (2, 1.0), (2, 3.0)])
def test_csr_power_parseval_and_positivity(model, Pi):
    """P = dkappa sum 2 Re(Z)|rho~|^2 equals the real-space energy loss
    Delta sum_i rho_i V_i exactly (discrete Parseval), and is >= 0 for Re Z >= 0."""
    pr = O.Params(n=48)
    zr, zi = O.impedance(pr, model, Pi)
    rho, _ = O.project(pr, W.blobs(48, 4))
    V, P = O.wake(pr, zr, zi, rho)
    assert P > 0
    assert abs(P - pr.delta * np.dot(rho, V)) < 1e-12 * abs(P)
    assert np.all(zr >= 0)


@pytest.mark.parametrize("n", [8, 13])
def test_wake_matches_dense_matrix(n):
    pr = O.Params(n=n)
    zr, zi = O.impedance(pr, 2, 1.3)
    rho = _rho(n, 5)
    V, P = O.wake(pr, zr, zi, rho)
    Vb, Pb = B.wake(n, 6.0, 2, zr, zi, rho)
    assert np.max(np.abs(V - Vb)) < 1e-13 * np.max(np.abs(V))
    assert abs(P - Pb) < 1e-13 * abs(P)


def test_free_space_wake_acts_on_one_side():
    """With the printed Fourier convention V = int Z rho~ e^{ikq} dk and
    Zhat_FS ~ e^{i pi/6} kappa^{1/3}, the wake kernel vanishes for q < q'
    (one-sided): a narrow bunch at q = 0 produces a field on the +q side only
    (up to the periodic images of the zero-padded transform)."""
    pr = O.Params(n=256)
    zr, zi = O.impedance(pr, 1)
    x = W.grid_axis(256)
    rho = np.exp(-0.5 * (x / 0.2) ** 2)
    rho /= pr.delta * rho.sum()
    V, _ = O.wake(pr, zr, zi, rho)
    assert np.max(np.abs(V[x < -1.5])) < 0.15 * np.max(np.abs(V[x > 1.5]))


def test_free_space_impedance_matches_paper_formula():
    """Zhat_FS = 2 (sigma_z/R)^{1/3} Z(n)/Z0 with the paper's
    Z(n) = Z0 Gamma(2/3) 3^{-1/3} (sqrt3/2 + i/2) n^{1/3} at n = kappa R/sigma_z."""
    R, sz = 5.559, 1e-3
    for kap in (0.1, 1.0, 7.5):
        n = kap * R / sz
        Zn = math.gamma(2 / 3) * 3 ** (-1 / 3) * complex(math.sqrt(3) / 2, 0.5) * n ** (1 / 3)
        ref = 2 * (sz / R) ** (1 / 3) * Zn
        assert abs(I.zhat_free_space(kap) - ref) < 1e-14 * abs(ref)


def test_parallel_plates_limits():
    """Fig. impedance: at high frequency the shielded impedance converges to
    free space; towards f = 0 both go to 0 (Sec. II.B)."""
    Pi = 2.0
    hi = np.array([100.0, 300.0, 1000.0]) * Pi
    r = I.zhat_parallel_plates(hi, Pi) / I.zhat_free_space(hi)
    assert np.all(np.abs(r - 1) < 2e-4)
    lo = np.array([1e-3, 1e-2, 0.1]) * Pi
    zpp = np.abs(I.zhat_parallel_plates(lo, Pi))
    assert np.all(np.diff(zpp) > 0) and zpp[0] < 1e-6
    assert I.zhat_parallel_plates([0.0], Pi)[0] == 0


def test_parallel_plates_against_mpmath():
    """Independent evaluation with mpmath's Airy functions at 30 digits:
    term-by-term sum with its own remainder estimate from mpmath's Hurwitz
    zeta.  Agreement to 1e-10: in double precision Ai'Bi' + u Ai Bi cancels two
    O(sqrt u) terms down to O(u^-5/2), losing about 1e-16 u^3 relative."""
    mp.mp.dps = 30

    def zpp(kappa, Pi, P=400):
        kappa, Pi = mp.mpf(kappa), mp.mpf(Pi)
        a = mp.pi ** 2 * mp.mpf(2) ** (-mp.mpf(8) / 3) * (Pi / kappa) ** (mp.mpf(4) / 3)
        s = mp.mpc(0)
        for p in range(P):
            u = a * (2 * p + 1) ** 2
            ai, aip, bi, bip = mp.airyai(u), mp.airyai(u, 1), mp.airybi(u), mp.airybi(u, 1)
            s += aip * (aip - 1j * bip) + u * ai * (ai - 1j * bi)
        tail = 3 / (16 * mp.pi) * (a ** -2.5 * mp.zeta(5, P + 0.5) / 32
                                   + mp.mpf(105) / 32 * a ** -5.5 * mp.zeta(11, P + 0.5) / 2048)
        s -= 1j * tail
        return complex(4 * mp.pi ** 2 * mp.cbrt(2) * Pi ** (mp.mpf(2) / 3) * kappa ** (-mp.mpf(1) / 3) * s)

    for kap, Pi in [(1.0, 2.0), (5.0, 1.0), (40.0, 1.0), (12.0, 3.0), (0.2, 3.0)]:
        ref = zpp(kap, Pi)
        got = I.zhat_parallel_plates([kap], Pi)[0]
        assert abs(got - ref) < 1e-10 * abs(ref), (kap, Pi, got, ref)


def test_airy_large_argument_expansion():
    """The closed-form remainder uses Ai'Bi' + u Ai Bi = 3/(16 pi) u^{-5/2}
    (1 + 105/32 u^{-3} + 75075/2048 u^{-6} + 56581525/65536 u^{-9} + O(u^{-12}));
    check it against mpmath (relative error < 1e-12 from u = 25 on)."""
    mp.mp.dps = 60
    for u in (25, 30, 60, 100, 1000):
        u = mp.mpf(u)
        g = mp.airyai(u, 1) * mp.airybi(u, 1) + u * mp.airyai(u) * mp.airybi(u)
        approx = 3 / (16 * mp.pi) * u ** -2.5 * (1 + mp.mpf(105) / 32 / u ** 3
                                                  + mp.mpf(75075) / 2048 / u ** 6
                                                  + mp.mpf(56581525) / 65536 / u ** 9)
        assert abs(g / approx - 1) < 5e4 / u ** 12
