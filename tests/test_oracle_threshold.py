"""Oracle brackets of the micro-bunching threshold that pin the two readings
the paper leaves open: the sign of the wake kick and the gap in the
shielding parameter.

The paper shows the threshold only as the "finger" of its measured and
simulated spectrograms (Sec. IV.C).  What the oracle must reproduce is the
scaling law of the shielded-CSR studies it builds on, S_th ~ 0.5 + 0.12 Pi,
and the paper's own free-space example: a run at scaled current xi = 0.516,
just above the free-space threshold of 0.5, oscillates weakly (Sec. IV.B,
Table "artifact parameters").

Each case brackets the law on the oracle: a point well below it relaxes
and a point above it bursts.  The same upper point is then run under the
other reading, where it must relax:
  * parallel plates, Pi = 2 and 3: Pi taken with the full plate distance g
    = 2h instead of the half distance h multiplies the physical shielding by
    2^(3/2) (the oracle's Pi_half = 2^(3/2) Pi_full); the threshold would
    then sit near 0.5 + 0.12 * 2^(3/2) Pi (1.18 and 1.52), above the
    bracket's upper point;
  * free space: the opposite kick sign (dp = -S V dtheta) keeps the bunch
    stable well past 0.5.
So a change of either reading makes one of these tests fail.

Bursting is the growth of the CSR-power fluctuation: the relative standard
deviation of P over each synchrotron period (the envelope of Sec. IV.C's
bursting), started from the Haissinski equilibrium plus 1e-6 noise.  A
point bursts by the one criterion of every scan here (analysis.BURST_LEVEL
over the last 20 periods), and relaxes when its envelope stays below 1e-3
and keeps shrinking.
"""
import numpy as np
import pytest

from oracle import haissinski as H
from oracle import oracle as O
from paper_1611_05293_b300 import analysis as A

N, SPP, BETA, PERIODS = 128, 500, 0.01, 60


def envelope(model, Pi, S, seed):
    op = O.Params(n=N, steps_per_period=SPP, beta=BETA, s_csr=S)
    zr, zi = O.impedance(op, model, Pi)
    rng = np.random.default_rng(seed)
    try:
        psi = H.density(op, zr, zi)
    except RuntimeError:
        x = -op.half_width + op.delta * np.arange(op.n)
        psi = np.exp(-0.5 * (x[:, None] ** 2 + x[None, :] ** 2))
    psi = O.normalize(op, psi * (1 + 1e-6 * rng.uniform(-1, 1, psi.shape)))
    _, P, _ = O.run(op, zr, zi, psi, SPP * PERIODS)
    return A.fluctuation(P, SPP)


def bursts(f):
    return A.envelope_bursting(f, -20)


# (model, Pi, S below the law, S above the law, Pi and S of the other reading)
CASES = {
    "pp_pi2": (2, 2.0, 0.45, 1.0, (2.0 * 2 ** 1.5, 1.0)),
    "pp_pi3": (2, 3.0, 0.55, 1.15, (3.0 * 2 ** 1.5, 1.15)),
    "free_space": (1, 0.0, 0.3, 0.7, (0.0, -0.7)),
}


@pytest.mark.slow
@pytest.mark.parametrize("case", list(CASES))
def test_threshold_bracket_pins_readings(case):
    model, Pi, s_lo, s_hi, (Pi_alt, s_alt) = CASES[case]
    lo = envelope(model, Pi, s_lo, 1700)
    hi = envelope(model, Pi, s_hi, 1701)
    alt = envelope(model, Pi_alt, s_alt, 1701)
    assert not bursts(lo), (case, "below the law", np.median(lo[-20:]))
    assert bursts(hi), (case, "above the law", np.median(hi[-20:]))
    assert not bursts(alt), (case, "other reading", np.median(alt[-20:]))
