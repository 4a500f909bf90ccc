"""Write the FP64 oracle's statistics of the above-threshold workloads.

TEST INFRASTRUCTURE.  Calls only the oracle (``oracle/``) and the seeded
input generators (``paper_1611_05293_b300.workloads``, which hold none of
the solver's arithmetic).  Every number in the JSON files it writes comes
from the FP64 CPU oracle; the GPU tests compare the CUDA path's statistics
of the same runs against them.

Above the micro-bunching threshold the dynamics are chaotic (Sec. IV.C:
bursting), so FP32 and FP64 runs from the same start agree on statistics,
not on trajectories.  Per complete synchrotron period k of each run the
files keep the mean and the standard deviation of the CSR power P(t)
(Sec. IV.C) over that period; the tests derive means, fluctuation levels
and growth rates from these.  For the long single runs they also keep the
strongest lines of the power spectrum of P(t) over a window (the column of
the paper's bursting spectrogram, Sec. IV.C).

    python tests/golden/make_oracle_statistics.py c2      # ~2 min on 8 cores
    python tests/golden/make_oracle_statistics.py c3      # ~40 min
    python tests/golden/make_oracle_statistics.py c5      # ~90 min
    python tests/golden/make_oracle_statistics.py c2 --dump DIR   # also P(t) as .npy

Workloads (seeds as in the input recipe):
  c2: N = 256, 1000 steps/period, 50 periods, beta = 1.25e-2, Pi = 2,
      S_csr = 0.9, unit Gaussian + 1e-6 max U(-1, 1) noise (seed 1611).
  c3: the threshold scan, N = 256, 1000 steps/period, 20 periods, beta =
      1e-2, S_csr in linspace(0.2, 1.5, 21) x Pi in {1, 2, 3}; starts: the
      oracle's Haissinski equilibrium of each point (the unit Gaussian where
      its iteration does not converge) times (1 + 1e-6 U(-1, 1)), seed 1612 + i.
  c5: N = 1024, 4000 steps/period, periods 0..40, beta = 1e-2, Pi = 1,
      S_csr = 3, unit Gaussian + 1e-6 noise (seed 1614).
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from oracle import haissinski as H  # noqa: E402
from oracle import oracle as O  # noqa: E402
from paper_1611_05293_b300 import workloads as W  # noqa: E402


def period_stats(P: np.ndarray, spp: int):
    """[[mean, std], ...] of P over each complete period."""
    k = len(P) // spp
    b = np.asarray(P[: k * spp]).reshape(k, spp)
    return [[float(m), float(s)] for m, s in zip(b.mean(axis=1), b.std(axis=1))]


def spectrum_lines(P: np.ndarray, spp: int, count: int = 5):
    """Strongest lines of |FFT(Hann (P - mean))|^2 of a window, as [cycles
    per synchrotron period, relative power], DC excluded, strongest first;
    the frequency is refined by the parabola through the peak bin and its
    two neighbours (in log power)."""
    x = np.asarray(P, dtype=np.float64)
    x = (x - x.mean()) * np.hanning(len(x))
    s = np.abs(np.fft.rfft(x)) ** 2
    s[0] = 0.0
    df = spp / len(x)
    peaks = [k for k in range(1, len(s) - 1) if s[k] >= s[k - 1] and s[k] >= s[k + 1]]
    peaks.sort(key=lambda k: -s[k])
    out = []
    for k in peaks[:count]:
        a, b, c = np.log(s[k - 1] + 1e-300), np.log(s[k]), np.log(s[k + 1] + 1e-300)
        den = a - 2 * b + c
        off = 0.5 * (a - c) / den if den < 0 else 0.0
        out.append([float((k + off) * df), float(s[k] / s.max())])
    return out


def haissinski_start(op, zr, zi, seed):
    rng = np.random.default_rng(seed)
    try:
        psi = H.density(op, zr, zi)
        start = "haissinski"
    except RuntimeError:
        x = -op.half_width + op.delta * np.arange(op.n)
        psi = np.exp(-0.5 * (x[:, None] ** 2 + x[None, :] ** 2))
        start = "gaussian"
    return O.normalize(op, psi * (1 + 1e-6 * rng.uniform(-1, 1, psi.shape))), start


def c2(dump):
    n, spp, periods, beta, Pi, S = 256, 1000, 50, 1.25e-2, 2.0, 0.9
    op = O.Params(n=n, steps_per_period=spp, beta=beta, s_csr=S)
    zr, zi = O.impedance(op, 2, Pi)
    psi0 = O.normalize(op, W.noisy_gaussian(n, 1611, 1e-6))
    t0 = time.time()
    _, P, _ = O.run(op, zr, zi, psi0, spp * periods)
    if dump:
        np.save(os.path.join(dump, "oracle_c2_P.npy"), P)
    half = P[spp * periods // 2:]
    return {"workload": "C2: N=256, 1000 steps/period, 50 periods, beta=1.25e-2, Pi=2, S=0.9, "
                        "noisy_gaussian(256, seed 1611, 1e-6)",
            "n": n, "steps_per_period": spp, "periods": periods, "beta": beta, "Pi": Pi, "S_csr": S,
            "seed": 1611, "period_stats": period_stats(P, spp),
            "second_half": {"mean": float(half.mean()), "lines": spectrum_lines(half, spp)},
            "oracle_seconds": time.time() - t0}


def c3(dump):
    n, spp, periods, beta = 256, 1000, 20, 1e-2
    pts = W.scan_grid(duplicate=None)
    out = []
    t0 = time.time()
    for i, (S, Pi) in enumerate(pts):
        op = O.Params(n=n, steps_per_period=spp, beta=beta, s_csr=S)
        zr, zi = O.impedance(op, 2, Pi)
        psi0, kind = haissinski_start(op, zr, zi, 1612 + i)
        _, P, _ = O.run(op, zr, zi, psi0, spp * periods)
        if dump:
            np.save(os.path.join(dump, f"oracle_c3_{i:02d}_P.npy"), P)
        out.append({"S_csr": S, "Pi": Pi, "seed": 1612 + i, "start": kind, "period_stats": period_stats(P, spp)})
        print(f"c3 point {i + 1}/{len(pts)} S={S:.3f} Pi={Pi:g} ({time.time() - t0:.0f} s)", flush=True)
    return {"workload": "C3: N=256, 1000 steps/period, 20 periods, beta=1e-2, S in linspace(0.2,1.5,21) x "
                        "Pi in {1,2,3}, Haissinski (or Gaussian) start x (1 + 1e-6 U(-1,1)), seed 1612+i",
            "n": n, "steps_per_period": spp, "periods": periods, "beta": beta, "points": out,
            "oracle_seconds": time.time() - t0}


def c5(dump):
    n, spp, periods, beta, Pi, S = 1024, 4000, 40, 1e-2, 1.0, 3.0
    op = O.Params(n=n, steps_per_period=spp, beta=beta, s_csr=S)
    zr, zi = O.impedance(op, 2, Pi)
    psi = O.normalize(op, W.noisy_gaussian(n, 1614, 1e-6))
    t0 = time.time()
    Ps = []
    for k in range(periods):  # one period per call: progress, and a bounded call
        psi, P, _ = O.run(op, zr, zi, psi, spp)
        Ps.append(P)
        print(f"c5 period {k + 1}/{periods} ({time.time() - t0:.0f} s)", flush=True)
    P = np.concatenate(Ps)
    if dump:
        np.save(os.path.join(dump, "oracle_c5_P.npy"), P)
    win = P[20 * spp:40 * spp]
    return {"workload": "C5: N=1024, 4000 steps/period, periods 0-40, beta=1e-2, Pi=1, S=3, "
                        "noisy_gaussian(1024, seed 1614, 1e-6)",
            "n": n, "steps_per_period": spp, "periods": periods, "beta": beta, "Pi": Pi, "S_csr": S,
            "seed": 1614, "period_stats": period_stats(P, spp),
            "periods_20_40": {"mean": float(win.mean()), "lines": spectrum_lines(win, spp)},
            "oracle_seconds": time.time() - t0}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("which", choices=["c2", "c3", "c5"])
    ap.add_argument("--dump", default="", help="directory for the full P(t) series (.npy)")
    a = ap.parse_args()
    O.build()
    res = {"c2": c2, "c3": c3, "c5": c5}[a.which](a.dump)
    res["generator"] = "tests/golden/make_oracle_statistics.py " + a.which
    with open(os.path.join(HERE, f"oracle_{a.which}.json"), "w") as f:
        json.dump(res, f, indent=0)
        f.write("\n")


if __name__ == "__main__":
    main()
