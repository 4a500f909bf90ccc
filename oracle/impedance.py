"""Normalised CSR impedances for the oracle (Sec. II.B of the paper).

TEST INFRASTRUCTURE ONLY: imported by tests, the smoke check and the
benchmark's CPU-baseline leg; never by the product library.

Normalisation (reading of the paper, which prints only Z(n) in Ohm):
with kappa = k sigma_z the dimensionless wave number and R the bending
radius, the dimensionless impedance is

    Zhat(kappa) = 2 (sigma_z/R)^(1/3) Z(n = kappa R/sigma_z) / Z_0 ,

so that the kick per radian of synchrotron phase is dp/dtheta = S_csr V(q)
with S_csr = I_n R^(1/3) / sigma_z^(4/3) and V(q) = int Zhat rho~ e^{i kappa q}
dkappa.  Then

* free space (Sec. II.B, first impedance):
      Zhat_FS = 2 Gamma(2/3) 3^(-1/3) (sqrt(3)/2 + i/2) kappa^(1/3);
* parallel plates at distance g = 2h (Sec. II.B, second impedance), with the
  shielding parameter Pi = R^(1/2) sigma_z / h^(3/2) of the half-distance h
  (the parameter of the threshold law S_th ~ 0.5 + 0.12 Pi):
      Zhat_PP = 4 pi^2 2^(1/3) Pi^(2/3) kappa^(-1/3) sum_p F(u_p),
      F(u) = Ai'(u) Ci'(u) + u Ai(u) Ci(u),  Ci = Ai - i Bi,
      u_p = pi^2 (2p+1)^2 2^(-8/3) (Pi/kappa)^(4/3),
  i.e. the printed formula with R/g = R/(2h).  The printed formula lacks the
  parentheses around the sum; the sum runs over both terms, and j is the
  same imaginary unit as in Z_FS.

The Airy functions are scipy's exponentially scaled ones (a library
primitive), so Bi does not overflow.  The sum is taken term by term while
u_p < 25 and the rest is added in closed form from the large-u behaviour
Ai'Bi' + u Ai Bi = 3/(16 pi) u^(-5/2) (1 + 105/32 u^(-3) + 75075/2048 u^(-6)
+ 56581525/65536 u^(-9) + O(u^-12)) (relative error below 1e-12 for u >= 25),
whose p-sums are Hurwitz zeta values; Ai'^2 + u Ai^2 < exp(-160) there.  The crossover is low because
in double precision Ai'Bi' + u Ai Bi cancels two O(sqrt u) terms down to
O(u^-5/2): scipy's terms lose about 1e-16 u^3 relative accuracy.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import airye, gamma, zeta

__all__ = ["zhat_free_space", "zhat_parallel_plates", "impedance_table", "kappa_grid", "fft_length"]

_FS_CONST = 2.0 * gamma(2.0 / 3.0) * 3.0 ** (-1.0 / 3.0) * complex(math.sqrt(3.0) / 2.0, 0.5)


def zhat_free_space(kappa):
    """Zhat_FS(kappa) for kappa >= 0 (complex array)."""
    kappa = np.asarray(kappa, dtype=np.float64)
    return _FS_CONST * np.cbrt(kappa)


def _pp_sum(a: float) -> complex:
    """sum_{p>=0} F(a (2p+1)^2) for one a = pi^2 2^(-8/3) (Pi/kappa)^(4/3)."""
    # exact terms while u_p < 25 (possibly none); the remainder in closed form
    pmax = max(0, int(math.ceil(0.5 * (math.sqrt(25.0 / a) - 1.0))))
    s = (2.0 * np.arange(pmax, dtype=np.float64) + 1.0)
    u = a * s * s
    eai, eaip, ebi, ebip = airye(u)
    zeta_u = (2.0 / 3.0) * u ** 1.5
    damp = np.exp(-2.0 * zeta_u)
    re = (eaip * eaip + u * eai * eai) * damp            # Ai'^2 + u Ai^2
    im = -(eaip * ebip + u * eai * ebi)                  # -(Ai'Bi' + u Ai Bi)
    # closed-form remainder p >= pmax: sum (2p+1)^-s = 2^-s zeta(s, pmax + 1/2)
    h5 = 2.0 ** -5 * zeta(5.0, pmax + 0.5)
    h11 = 2.0 ** -11 * zeta(11.0, pmax + 0.5)
    h17 = 2.0 ** -17 * zeta(17.0, pmax + 0.5)
    h23 = 2.0 ** -23 * zeta(23.0, pmax + 0.5)
    tail = 3.0 / (16.0 * math.pi) * (a ** -2.5 * h5 + 105.0 / 32.0 * a ** -5.5 * h11
                                     + 75075.0 / 2048.0 * a ** -8.5 * h17
                                     + 56581525.0 / 65536.0 * a ** -11.5 * h23)
    # add small terms first
    return complex(float(np.sum(re[::-1])), float(np.sum(im[::-1])) - tail)


def zhat_parallel_plates(kappa, Pi: float):
    """Zhat_PP(kappa; Pi) for kappa >= 0 (complex array); Zhat_PP(0) = 0."""
    kappa = np.atleast_1d(np.asarray(kappa, dtype=np.float64))
    out = np.zeros(kappa.shape, dtype=np.complex128)
    pref = 4.0 * math.pi ** 2 * 2.0 ** (1.0 / 3.0) * Pi ** (2.0 / 3.0)
    for idx, k in np.ndenumerate(kappa):
        if k <= 0.0:
            continue
        a = math.pi ** 2 * 2.0 ** (-8.0 / 3.0) * (Pi / k) ** (4.0 / 3.0)
        out[idx] = pref * k ** (-1.0 / 3.0) * _pp_sum(a)
    return out


def fft_length(n: int, pad_factor: int) -> int:
    """Zero-padded transform length: the smallest power of two >= pad_factor*n."""
    m = 1
    while m < pad_factor * n:
        m <<= 1
    return m


def kappa_grid(n: int, half_width: float, pad_factor: int):
    """kappa_k = 2 pi k / (M Delta) for k = 0..M/2, M = fft_length(n, pad),
    Delta = 2L/(n-1)."""
    M = fft_length(n, pad_factor)
    delta = 2.0 * half_width / (n - 1)
    return 2.0 * math.pi * np.arange(M // 2 + 1) / (M * delta)


def impedance_table(model: int, n: int, half_width: float, pad_factor: int, Pi: float = 0.0):
    """(re, im) arrays of length M/2+1 on the FFT grid.

    model 0: no wake; 1: free space; 2: parallel plates with shielding Pi.
    """
    kap = kappa_grid(n, half_width, pad_factor)
    if model == 0:
        z = np.zeros_like(kap, dtype=np.complex128)
    elif model == 1:
        z = zhat_free_space(kap)
    elif model == 2:
        z = zhat_parallel_plates(kap, Pi)
    else:
        raise ValueError(f"impedance model {model}")
    return np.ascontiguousarray(z.real), np.ascontiguousarray(z.imag)
