"""Host statistics of solver output: bunch moments and CSR-power analysis.

These are post-processing utilities on arrays the library returns (psi
snapshots, the CSR-power series P(t)); none of them is part of a time step.

* moments(psi): centroids and RMS widths sigma_q (bunch length) and sigma_p
  (energy spread), the quantities plotted in the paper's convergence studies
  (Sec. IV.A, Figs. data-type, rotcompare, meshcompare).
* fluctuation(P, steps_per_period): relative standard deviation of P over
  each synchrotron period -- the "bursting" amplitude (Sec. IV.C: the
  spectrogram is the Fourier transform of P(t)).
* growth_rate(...): log-linear fit of that amplitude over a range of periods.
* is_bursting(...): the one bursting criterion of every threshold scan here
  (BURST_LEVEL, see below).
* bursting_period(P, steps_per_period): period (in synchrotron periods) of
  the dominant line of |FFT(P - mean)|^2 over the second half of the run.
* threshold(S_values, bursting): first S of a scan flagged as bursting.
"""
from __future__ import annotations

import numpy as np

__all__ = ["moments", "fluctuation", "growth_rate", "bursting_period", "threshold", "is_bursting",
           "BURST_LEVEL", "envelope_bursting"]

# Bursting criterion.  Started from the equilibrium plus 1e-6 noise, a point
# below the micro-bunching threshold has a CSR-power envelope (relative std of
# P per synchrotron period) that never exceeds its start transient, at most
# 2e-3 in every stable run of the N = 128 and N = 256 scans, and decays (growth
# rate < 0); above it the unstable mode grows out of the noise (growth rate >
# 0) until it saturates at 1e-2 .. 1 within about ten periods.  A median
# envelope above 1e-2 -- five times the largest stable level -- over a window
# of periods therefore means the envelope has grown, which is the growth-rate
# definition of bursting, without fitting a rate to a saturated signal (a fit
# over periods 5-20 gives slopes near zero or below for bursting points,
# whose growth is over by period 5).
BURST_LEVEL = 1e-2


def moments(psi: np.ndarray, half_width: float = 6.0) -> dict:
    n = psi.shape[0]
    x = -half_width + np.arange(n) * (2.0 * half_width / (n - 1))
    wq = psi.sum(axis=1)
    wp = psi.sum(axis=0)
    tot = wq.sum()
    mq = float((wq * x).sum() / tot)
    mp = float((wp * x).sum() / tot)
    sq = float(np.sqrt(max((wq * x * x).sum() / tot - mq * mq, 0.0)))
    sp = float(np.sqrt(max((wp * x * x).sum() / tot - mp * mp, 0.0)))
    return {"mean_q": mq, "mean_p": mp, "sigma_q": sq, "sigma_p": sp}


def fluctuation(P: np.ndarray, steps_per_period: int) -> np.ndarray:
    """Relative std of P within each complete synchrotron period."""
    k = len(P) // steps_per_period
    blocks = np.asarray(P[: k * steps_per_period]).reshape(k, steps_per_period)
    return blocks.std(axis=1) / np.abs(blocks.mean(axis=1))


def growth_rate(P: np.ndarray, steps_per_period: int, first: int = 5, last: int | None = None) -> float:
    """Slope (per synchrotron period) of log(fluctuation) over periods [first, last)."""
    f = fluctuation(P, steps_per_period)
    last = len(f) if last is None else min(last, len(f))
    if last - first < 3:
        raise ValueError("too few periods for a fit")
    t = np.arange(first, last)
    y = np.log(np.maximum(f[first:last], 1e-300))
    return float(np.polyfit(t, y, 1)[0])


def envelope_bursting(f, first: int | None = None, last: int | None = None, level: float = BURST_LEVEL) -> bool:
    """Bursting from a per-period envelope f (as fluctuation returns): its
    median over periods [first, last) exceeds `level`."""
    f = np.asarray(f, dtype=np.float64)
    return bool(np.median(f[first:last]) > level)


def is_bursting(P: np.ndarray, steps_per_period: int, first: int | None = None, last: int | None = None,
                level: float = BURST_LEVEL) -> bool:
    """The bursting criterion (BURST_LEVEL) on the CSR-power series P over
    periods [first, last) (default: the whole run)."""
    return envelope_bursting(fluctuation(P, steps_per_period), first, last, level)


def bursting_period(P: np.ndarray, steps_per_period: int) -> float:
    """Period (in synchrotron periods) of the strongest line of P(t) over the
    second half of the series, excluding the synchrotron harmonics' DC."""
    x = np.asarray(P[len(P) // 2:], dtype=np.float64)
    x = x - x.mean()
    spec = np.abs(np.fft.rfft(x * np.hanning(len(x)))) ** 2
    freq = np.fft.rfftfreq(len(x), d=1.0 / steps_per_period)  # cycles per synchrotron period
    spec[0] = 0.0
    k = int(np.argmax(spec))
    return float(1.0 / freq[k]) if freq[k] > 0 else float("inf")


def threshold(S_values, bursting) -> float | None:
    """First S (in increasing order) flagged as bursting, or None."""
    for s, b in sorted(zip(S_values, bursting)):
        if b:
            return float(s)
    return None
