"""Physical-unit front end: machine parameters -> the normalised problem.

The solver works in the normalised variables of the paper (q = z/sigma_z,
p = delta/sigma_delta, time in synchrotron periods), with the damping
parameter beta = 1/(f_s tau_d), the shielding parameter Pi and the CSR
strength S_csr.  This module derives them from the parameters of an
isomagnetic ring such as the paper's ANKA-like set (Sec. IV.D, table of
iso-ANKA parameters), whose frequencies are already scaled by 2 pi R/C:

* bending radius R = c / (2 pi f_rev) of the isomagnetic ring;
* energy loss per turn U0 = C_gamma E0^4 / R (C_gamma = 8.846e-5 m/GeV^3)
  and the synchronous phase, cos(phi_s) = sqrt(1 - (U0 / e V_rf)^2);
* momentum compaction from the synchrotron frequency,
  f_s^2 = f_rev^2 h alpha_c e V_rf cos(phi_s) / (2 pi E0);
* natural bunch length sigma_z = c alpha_c sigma_delta / (2 pi f_s);
* Pi = R^(1/2) sigma_z / h_gap^(3/2) with h_gap the half gap (the reading of
  the shielding parameter used throughout: plates at +-h_gap);
* S_csr = I_n R^(1/3) / sigma_z^(4/3), I_n = r_e N / (2 pi nu_s gamma sigma_delta),
  N = I_bunch / (e f_rev,real) the bunch population, nu_s = f_s / f_rev;
* beta = 1 / (f_s tau_d).

Host-side arithmetic only (plain Python floats).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

C_LIGHT = 299792458.0          # m/s
E_CHARGE = 1.602176634e-19     # C
ME_EV = 0.51099895e6           # electron rest energy, eV
R_E = 2.8179403262e-15         # classical electron radius, m
C_GAMMA = 8.846e-5             # m / GeV^3


@dataclass
class Machine:
    """An isomagnetic electron ring (frequencies of the isomagnetic model)."""
    energy_eV: float           # E0
    sigma_delta: float         # natural relative energy spread
    damping_time_s: float      # longitudinal damping time tau_d
    harmonic: float            # RF harmonic number
    v_rf: float                # RF voltage, V
    f_rev: float               # revolution frequency, Hz
    f_s: float                 # synchrotron frequency, Hz
    gap_m: float               # full vacuum-chamber height (plates at +-gap/2)
    scale: float = 1.0         # 2 pi R / C: real f_rev = f_rev * scale


def iso_anka() -> Machine:
    """The paper's isomagnetic ANKA-like parameter set (scaled by 2 pi R/C = 0.316)."""
    return Machine(energy_eV=1.285e9, sigma_delta=0.47e-3, damping_time_s=3.353e-3, harmonic=58.21,
                   v_rf=1048e3, f_rev=8.582e6, f_s=28.13e3, gap_m=32e-3, scale=0.316)


def derived(m: Machine) -> dict:
    """R, U0, cos(phi_s), alpha_c, sigma_z, Pi, beta and the steps-free parts of S_csr."""
    R = C_LIGHT / (2.0 * math.pi * m.f_rev)
    U0 = C_GAMMA * (m.energy_eV / 1e9) ** 4 / R * 1e9
    if U0 >= m.v_rf:
        raise ValueError("RF voltage below the energy loss per turn")
    cphi = math.sqrt(1.0 - (U0 / m.v_rf) ** 2)
    alpha = 2.0 * math.pi * m.energy_eV * m.f_s ** 2 / (m.f_rev ** 2 * m.harmonic * m.v_rf * cphi)
    sigma_z = C_LIGHT * alpha * m.sigma_delta / (2.0 * math.pi * m.f_s)
    Pi = math.sqrt(R) * sigma_z / (0.5 * m.gap_m) ** 1.5
    beta = 1.0 / (m.f_s * m.damping_time_s)
    return dict(R=R, U0_eV=U0, cos_phi_s=cphi, alpha_c=alpha, sigma_z=sigma_z, Pi=Pi, beta=beta,
                gamma=m.energy_eV / ME_EV, nu_s=m.f_s / m.f_rev)


def s_csr(m: Machine, bunch_current_A: float) -> float:
    """CSR strength S_csr of a bunch current (A, as measured in the real ring)."""
    d = derived(m)
    N = bunch_current_A / (E_CHARGE * m.f_rev * m.scale)
    I_n = R_E * N / (2.0 * math.pi * d["nu_s"] * d["gamma"] * m.sigma_delta)
    return I_n * d["R"] ** (1.0 / 3.0) / d["sigma_z"] ** (4.0 / 3.0)


def bunch_current(m: Machine, S: float) -> float:
    """Bunch current (A) with CSR strength S (S_csr is linear in the current)."""
    return S / s_csr(m, 1.0)
