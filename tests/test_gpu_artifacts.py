"""Interpolation artifacts at the paper's example parameters (Sec. IV.B,
Table "artifact parameters"): N = 256, 4000 steps per synchrotron period,
free-space impedance, scaled current xi = 0.516, damping time 200 T_s, start
a Gaussian quantised to 16 bits (as the paper's image starts are).

* Cubic interpolation stays physical: no density below -1e-3 of the
  profile's peak over 60 periods, and an energy spread above its natural
  value (free space above xi = 0.5 widens it; the paper reads 1.01) but
  within 8 % of it, averaged over periods 20-60.
* Quadratic interpolation does not: its profile reaches negative densities
  (the paper: its overshoots "create negative charge densities") below -2 %
  of the peak by period 50 (measured -3.7 %; -10 % by period 200, where its
  energy spread has fallen to 0.82 of the natural value against the cubic
  run's 1.02).  The paper's two-cell ripple itself does not appear in these
  runs.
* Clamping (Eq. clamping), with which the paper suppressed the artifacts it
  met, keeps the quadratic run's densities non-negative (measured: none
  below 0 over 60 periods).

Both run on the FP32 register-blocked kernel (the quadratic through its
N_I = 3 instance).
"""
import numpy as np
import pytest

from paper_1611_05293_b300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def V():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1611_05293_b300 import vfps
    vfps.lib()
    return vfps


def artifact_run(V, ni, periods=60, clamp=0):
    n, spp = 256, 4000
    g = W.gaussian(n)
    psi0 = np.round(g / g.max() * 65535) / 65535
    sim = V.Simulation(V.Params(n=n, steps_per_period=spp, beta=1.0 / 200, interp_points=ni, clamp=clamp), psi0)
    sim.set_impedance(V.IMPEDANCE_FREE_SPACE, 0.0, 0.516)
    sim.record_moments(spp // 10)
    min_rho = []
    for _ in range(periods // 2):
        sim.step(2 * spp)
        rho = sim.profile()
        min_rho.append(float(rho.min() / rho.max()))
    m = sim.moment_series()
    sim.close()
    sigma_p_per_period = m[9::10, 4]
    return np.asarray(min_rho), sigma_p_per_period


def test_cubic_stays_physical_quadratic_goes_negative(V):
    neg3, sp3 = artifact_run(V, 3)
    neg4, sp4 = artifact_run(V, 4)
    assert sp4.shape == (60,) and sp3.shape == (60,)
    # cubic: no negative densities to speak of, sigma_p a little above natural
    assert neg4.min() > -1e-3, neg4.min()
    assert 1.0 < sp4[19:60].mean() < 1.08, sp4[19:60].mean()
    # quadratic: negative densities of percent level, growing
    assert neg3[:25].min() < -0.02, neg3[:25].min()
    assert neg3[20:30].min() < neg3[:5].min(), (neg3[:5].min(), neg3[20:30].min())
    # quadratic with clamping: no negative densities
    neg3c, _ = artifact_run(V, 3, clamp=1)
    assert neg3c.min() > -1e-6, neg3c.min()
