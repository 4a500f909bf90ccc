"""Physics pins of the whole oracle step (rotation + wake kick + Fokker-Planck
+ renormalisation) against facts of the model that do not depend on how any
single operator is coded."""
import numpy as np
import pytest

from oracle import haissinski as H
from oracle import oracle as O
from paper_1611_05293_b300 import analysis as A
from paper_1611_05293_b300 import workloads as W


def test_renormalised_charge_is_one():
    pr = O.Params(n=40, steps_per_period=50, beta=0.3, s_csr=0.7)
    zr, zi = O.impedance(pr, 1)
    psi, _, Q = O.run(pr, zr, zi, O.normalize(pr, W.gaussian(40, 6.0, 1.2, 0.8, q0=0.5)), 20)
    assert abs(O.charge(pr, psi) - 1.0) < 1e-13
    # what each step loses or gains before renormalising is boundary flux:
    # this bunch is 3e-5 of its peak at the grid edge
    assert np.max(np.abs(Q - 1.0)) < 5e-5


def test_damping_to_unit_gaussian_follows_exponential_law():
    """No wake: a round Gaussian of width sigma0 relaxes as
    sigma^2 - 1 = (sigma0^2 - 1) exp(-beta T) (T in synchrotron periods, beta =
    1/(f_s tau_d) per period, Eq. VFP), within the 1 % the paper's convergence
    studies quote (Table maximum errors).  Set-up of Sec. IV.A: sigma0 = 1.45."""
    n, spp, beta, sigma0 = 64, 100, 0.2, 1.45
    pr = O.Params(n=n, steps_per_period=spp, beta=beta)
    zr, zi = O.impedance(pr, 0)
    psi = O.normalize(pr, W.gaussian(n, 6.0, sigma0, sigma0))
    for T in (2, 4, 6):
        psi, _, _ = O.run(pr, zr, zi, psi, 2 * spp)
        m = A.moments(psi)
        ref = 1.0 + (sigma0 ** 2 - 1.0) * np.exp(-beta * T)
        got = 0.5 * (m["sigma_q"] ** 2 + m["sigma_p"] ** 2)
        assert abs(got - ref) < 0.01 * (sigma0 ** 2 - 1.0), (T, got, ref)


def test_equilibrium_gaussian_is_stationary():
    """beta > 0, no wake: exp(-(q^2+p^2)/2) is the equilibrium (Sec. IV.A).
    What remains after one period is the standard rotation's interpolation
    drift (the paper reports that it does not vanish, Fig. meshcompare):
    1.25e-3 of the peak at N=96, 200 steps per period; bound 2e-3.  The
    Fokker-Planck step itself keeps it: with the rotation removed (one full
    turn per step) the change is O(Delta^2) and far smaller."""
    n = 96
    pr = O.Params(n=n, steps_per_period=200, beta=0.05)
    zr, zi = O.impedance(pr, 0)
    g = O.normalize(pr, W.gaussian(n))
    psi, _, _ = O.run(pr, zr, zi, g, 200)
    assert np.max(np.abs(psi - g)) / g.max() < 2e-3


def test_centroid_balances_csr_energy_loss():
    """At equilibrium the RF restores what the wake takes: from
    dp/dtheta = -q + S_csr V(q) averaged over the bunch, <q> = S_csr <V> =
    S_csr P (P = Delta sum rho V is the CSR power, Sec. IV.C).  The bunch
    therefore sits on the side the CSR wake acts toward (+q, pinned in the
    wake tests): energy lost to radiation ahead of the emitters is made up
    by the RF.  Checked after ten damping times (beta = 1)."""
    n, spp = 64, 200
    for model, Pi, S in ((1, 0.0, 0.3), (2, 1.0, 0.4)):
        pr = O.Params(n=n, steps_per_period=spp, beta=1.0, s_csr=S)
        zr, zi = O.impedance(pr, model, Pi)
        psi, P, _ = O.run(pr, zr, zi, O.normalize(pr, W.gaussian(n)), 10 * spp)
        m = A.moments(psi)
        assert m["mean_q"] > 0
        assert abs(m["mean_q"] - S * P[-1]) < 0.03 * S * P[-1], (m, P[-1])
        assert abs(m["mean_p"]) < 0.02 * m["mean_q"]


def test_profile_converges_to_haissinski_below_threshold():
    """Below threshold with damping, psi relaxes to rho_H(q) exp(-p^2/2)
    (Appendix A; Haissinski solution on the same grid and wake)."""
    n, spp = 64, 100
    pr = O.Params(n=n, steps_per_period=spp, beta=0.5, s_csr=0.3)
    zr, zi = O.impedance(pr, 2, 2.0)
    rho_h = H.profile(pr, zr, zi)
    psi, _, _ = O.run(pr, zr, zi, O.normalize(pr, W.gaussian(n)), 16 * spp)
    rho, _ = O.project(pr, psi)
    assert np.max(np.abs(rho - rho_h)) / rho_h.max() < 1e-2


@pytest.mark.slow
def test_threshold_brackets_bcs_law():
    """Micro-bunching threshold S_th ~ 0.5 + 0.12 Pi (the scaling law of the
    shielded-CSR studies the paper builds on; Sec. IV.C's threshold finger):
    at Pi = 1 (S_th ~ 0.62), S = 0.45 relaxes and S = 1.1 bursts.  N = 128,
    500 steps per period, beta = 0.01, Haissinski start plus 1e-6 noise,
    60 periods; bursting = the criterion of analysis.BURST_LEVEL over the
    last 20 periods, relaxing = an envelope below 1e-3 that is still
    shrinking (growth rate < 0)."""
    n, spp, periods = 128, 500, 60
    rng = np.random.default_rng(1612)
    out = {}
    for S in (0.45, 1.1):
        pr = O.Params(n=n, steps_per_period=spp, beta=0.01, s_csr=S)
        zr, zi = O.impedance(pr, 2, 1.0)
        try:
            psi = H.density(pr, zr, zi)
        except RuntimeError:  # far above threshold there is no equilibrium: Gaussian start
            x = -pr.half_width + pr.delta * np.arange(n)
            psi = np.exp(-0.5 * (x[:, None] ** 2 + x[None, :] ** 2))
        psi = O.normalize(pr, psi * (1 + 1e-6 * rng.uniform(-1, 1, psi.shape)))
        _, P, _ = O.run(pr, zr, zi, psi, spp * periods)
        out[S] = A.fluctuation(P, spp)
    lo, hi = out[0.45], out[1.1]
    assert np.median(lo[-20:]) < 1e-3 and np.median(lo[-20:]) < np.median(lo[20:40])
    assert A.envelope_bursting(hi, -20)


def test_moments_of_shifted_gaussians():
    """Bunch moments (the bunch length and energy spread of the paper's
    figures) of sampled Gaussians: a well-resolved Gaussian's discrete
    moments equal its parameters (the sampling error of the rectangle rule
    is exponentially small), an off-centre one has the centre as its mean."""
    n = 255
    pr = O.Params(n=n)
    # (the grid edge is >= 6 sigma away, so truncation is below 1e-7)
    for sq, sp, q0, p0 in ((0.6, 0.6, 0.0, 0.0), (0.5, 0.8, 0.5, -0.8), (0.8, 0.45, -1.0, 0.3)):
        psi = W.gaussian(n, 6.0, sq, sp, q0, p0)
        m = O.moments(pr, psi)
        assert np.max(np.abs(m - np.array([q0, sq, p0, sp]))) < 1e-7, (m, sq, sp, q0, p0)
    # a quarter period of dq/dtheta = p, dp/dtheta = -q carries a particle at
    # (q0, p0) to (p0, -q0) (Sec. III.B): the mean moves there, the widths swap
    pr4 = O.Params(n=n, steps_per_period=4)
    psi = W.gaussian(n, 6.0, 0.5, 0.8, 0.5, -0.8)
    m = O.moments(pr4, O.rotate(pr4, psi))
    assert np.max(np.abs(m - np.array([-0.8, 0.8, -0.5, 0.5]))) < 1e-7, m


def test_power_spectrum_of_known_signals():
    """Power spectrum of a P(t) window: a constant has none (mean removed); a
    cosine on bin m puts (A L/4)^2 on bin m and (A L/8)^2 on each neighbour
    (the Hann window's three-bin response) and nothing else; two cosines add."""
    L = 256
    j = np.arange(L)
    assert np.max(O.power_spectrum(np.full(L, 3.7), L)) < 1e-20
    for m, A in ((10, 1.0), (37, 0.25)):
        s = O.power_spectrum(5.0 + A * np.cos(2 * np.pi * m * j / L), L)
        ref = np.zeros(L // 2 + 1)
        ref[m] = (A * L / 4) ** 2
        ref[m - 1] = ref[m + 1] = (A * L / 8) ** 2
        assert np.max(np.abs(s - ref)) < 1e-9 * ref.max(), m
    both = O.power_spectrum(np.cos(2 * np.pi * 10 * j / L) + np.cos(2 * np.pi * 40 * j / L), L)
    assert abs(both[10] - (L / 4) ** 2) < 1e-9 * (L / 4) ** 2 and abs(both[40] - (L / 4) ** 2) < 1e-9 * (L / 4) ** 2
