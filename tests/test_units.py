"""Physical-unit front end (paper_1611_05293_b300/units.py) on the paper's
isomagnetic ANKA-like parameter set (Sec. IV.D): the normalised damping
parameter is the printed damping time in synchrotron periods, the
circumference implied by 2 pi R/C = 0.316 is ANKA's 110 m, the bunch length
is the few-picosecond natural length, Pi sits between 1 and 2, and S_csr is
linear in the current."""
import math

import pytest

from paper_1611_05293_b300 import units as U


def test_iso_anka_normalised_parameters():
    m = U.iso_anka()
    d = U.derived(m)
    # tau_d = 3.353 ms at f_s = 28.13 kHz is 94.3 synchrotron periods
    assert abs(1.0 / d["beta"] - 3.353e-3 * 28.13e3) < 1e-9
    # real circumference C = 2 pi R / 0.316 = c / f_rev,real
    C = 2 * math.pi * d["R"] / m.scale
    assert abs(C - U.C_LIGHT / (m.f_rev * m.scale)) < 1e-9 and 109.0 < C < 112.0
    # synchrotron tune and the derived momentum compaction reproduce f_s
    fs = m.f_rev * math.sqrt(m.harmonic * d["alpha_c"] * m.v_rf * d["cos_phi_s"] / (2 * math.pi * m.energy_eV))
    assert abs(fs / m.f_s - 1.0) < 1e-12
    assert 2e-12 < d["sigma_z"] / U.C_LIGHT < 6e-12      # a few ps
    assert 1.0 < d["Pi"] < 2.0


def test_s_csr_linear_in_current_and_round_trip():
    m = U.iso_anka()
    s1, s2 = U.s_csr(m, 1e-4), U.s_csr(m, 3e-4)
    assert abs(s2 / s1 - 3.0) < 1e-12
    for S in (0.3, 0.84, 2.0):
        assert abs(U.s_csr(m, U.bunch_current(m, S)) / S - 1.0) < 1e-12


def test_rejects_rf_below_energy_loss():
    m = U.iso_anka()
    m.v_rf = 1e3
    with pytest.raises(ValueError):
        U.derived(m)
