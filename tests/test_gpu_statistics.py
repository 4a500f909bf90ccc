"""Statistical parity with the FP64 oracle at the workloads' own sizes.

Above the micro-bunching threshold the dynamics are chaotic (Sec. IV.C:
bursting), so the FP32 GPU path and the FP64 oracle are compared on the
statistics the paper reads off its runs -- the mean CSR power, the lines of
its spectrum (the spectrogram column, Sec. IV.C) and the threshold of a
current scan -- not on trajectories.  The oracle's numbers were written by
tests/golden/make_oracle_statistics.py (FP64 CPU oracle only) from the same
seeded starts; these tests run the CUDA path through the C ABI and compare.

* C2: one N = 256 simulation, 1000 steps/period, 50 periods, Pi = 2,
  S_csr = 0.9 (above the ~0.74 threshold): mean CSR power over the second
  half and the frequency of its strongest line within 2 %.
* C5: N = 1024, 4000 steps/period, Pi = 1, S_csr = 3 (deep bursting),
  Gaussian start, against the oracle's same 40 periods.  The run is chaotic
  from period 2 on and still relaxing, with a slow bursting cycle of ~13 T_s
  (~0.075 cycles per period) that a 30-period window holds only twice: the
  mean CSR power of periods 10-40 depends on the phase of that cycle, which
  rounding alone decides.  So the GPU runs an ensemble -- the oracle's own
  start and 31 starts that differ from it by noise at the same 1e-6 level,
  in one batch -- and the oracle's run must look like a member: its window
  mean inside the ensemble's two-sigma prediction interval, the ensemble's
  median frequency of the slow bursting line (periods 20-40) within 2 % and
  its median fluctuation envelope within 10 %.  A fixed bound on one GPU
  run against one oracle run would test the draw, not the method.
* C3: the 63-point threshold scan (N = 256, S_csr in linspace(0.2, 1.5, 21)
  x Pi in {1, 2, 3}, 1000 steps/period, 20 periods) in one batch, plus a
  duplicate point as an in-batch determinism probe: the threshold per Pi
  (first bursting S by analysis.BURST_LEVEL over periods 10-20) within one
  scan point of the oracle's scan and within two of 0.5 + 0.12 Pi.
"""
import json
import os
import sys

import numpy as np
import pytest

from oracle import oracle as O
from paper_1611_05293_b300 import analysis as A
from paper_1611_05293_b300 import workloads as W

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
sys.path.insert(0, GOLDEN)
import make_oracle_statistics as G  # noqa: E402  (the generator's own start and statistics code)


@pytest.fixture(scope="module")
def V():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1611_05293_b300 import vfps
    vfps.lib()
    return vfps


def golden(name):
    with open(os.path.join(GOLDEN, f"oracle_{name}.json")) as f:
        return json.load(f)


def envelope(stats):
    s = np.asarray(stats, dtype=np.float64)
    return s[:, 1] / s[:, 0]


def test_c2_bursting_statistics_match_oracle(V):
    g = golden("c2")
    n, spp, periods = g["n"], g["steps_per_period"], g["periods"]
    sim = V.Simulation(V.Params(n=n, steps_per_period=spp, beta=g["beta"]), W.noisy_gaussian(n, g["seed"], 1e-6))
    sim.set_impedance(V.IMPEDANCE_PARALLEL_PLATES, g["Pi"], g["S_csr"])
    sim.step(spp * periods)
    P = sim.csr_power()
    sim.close()
    assert len(P) == spp * periods
    half = P[spp * periods // 2:]
    ref = g["second_half"]
    assert A.is_bursting(P, spp, first=periods // 2), "C2 must be above threshold"
    assert abs(half.mean() - ref["mean"]) <= 0.02 * ref["mean"], (half.mean(), ref["mean"])
    f_gpu, f_ref = G.spectrum_lines(half, spp)[0][0], ref["lines"][0][0]
    print(f"C2: mean P {half.mean():.6e} vs {ref['mean']:.6e} ({abs(half.mean() / ref['mean'] - 1):.2e}); "
          f"strongest line {f_gpu:.5f} vs {f_ref:.5f} ({abs(f_gpu / f_ref - 1):.1e})")
    assert abs(f_gpu - f_ref) <= 0.02 * f_ref, (f_gpu, f_ref)


def test_c3_threshold_scan_matches_oracle_scan(V):
    g = golden("c3")
    n, spp, periods, beta = g["n"], g["steps_per_period"], g["periods"], g["beta"]
    pts = g["points"]
    starts = []
    for p in pts:
        op = O.Params(n=n, steps_per_period=spp, beta=beta, s_csr=p["S_csr"])
        zr, zi = O.impedance(op, 2, p["Pi"])
        psi0, kind = G.haissinski_start(op, zr, zi, p["seed"])
        assert kind == p["start"]
        starts.append(psi0)
    twin = next(i for i, p in enumerate(pts) if abs(p["S_csr"] - 0.785) < 1e-9 and p["Pi"] == 2.0)
    b = V.Batch(len(pts) + 1)
    slots = [b.add(V.Params(n=n, steps_per_period=spp, beta=beta), starts[i], V.IMPEDANCE_PARALLEL_PLATES,
                   p["Pi"], p["S_csr"], nsteps=spp * periods) for i, p in enumerate(pts)]
    dup = b.add(V.Params(n=n, steps_per_period=spp, beta=beta), starts[twin], V.IMPEDANCE_PARALLEL_PLATES,
                pts[twin]["Pi"], pts[twin]["S_csr"], nsteps=spp * periods)
    b.run(spp * periods)
    P = [b.take(sl, psi=False, rho=False)["power"] for sl in slots]
    P_dup = b.take(dup, psi=False, rho=False)["power"]
    b.close()
    assert np.array_equal(P_dup, P[twin]), "the duplicate point must give the same bits as its twin"

    step = 0.065
    for Pi in (1.0, 2.0, 3.0):
        idx = [i for i, p in enumerate(pts) if p["Pi"] == Pi]
        S = [pts[i]["S_csr"] for i in idx]
        gpu = [A.is_bursting(P[i], spp, first=10, last=20) for i in idx]
        ora = [A.envelope_bursting(envelope(pts[i]["period_stats"]), 10, 20) for i in idx]
        th_g, th_o = A.threshold(S, gpu), A.threshold(S, ora)
        print(f"C3 Pi={Pi}: threshold {th_g} (oracle {th_o}), flags differing {sum(a != b_ for a, b_ in zip(gpu, ora))} of {len(S)}")
        assert th_g is not None and th_o is not None, (Pi, gpu, ora)
        assert abs(th_g - th_o) <= step + 1e-9, (Pi, th_g, th_o)
        assert abs(th_g - (0.5 + 0.12 * Pi)) <= 2 * step + 1e-9, (Pi, th_g)
        assert sum(a != b_ for a, b_ in zip(gpu, ora)) <= 1, (Pi, gpu, ora)
        # below the threshold the runs are not chaotic: their mean CSR power
        # per period follows the oracle's closely
        for i, burst in zip(idx, ora):
            if burst or pts[i]["S_csr"] >= th_o - 1e-9:
                continue
            m_gpu = P[i][: spp * periods].reshape(periods, spp).mean(axis=1)
            m_ref = np.asarray(pts[i]["period_stats"])[:, 0]
            assert np.max(np.abs(m_gpu - m_ref) / m_ref) < 1e-3, (Pi, pts[i]["S_csr"])


def test_c5_large_grid_statistics_match_oracle(V):
    g = golden("c5")
    n, spp, beta, periods = g["n"], g["steps_per_period"], g["beta"], g["periods"]
    members = 32
    b = V.Batch(members)
    slots = [b.add(V.Params(n=n, steps_per_period=spp, beta=beta),
                   W.noisy_gaussian(n, g["seed"] if k == 0 else 7000 + k, 1e-6), V.IMPEDANCE_PARALLEL_PLATES,
                   g["Pi"], g["S_csr"], nsteps=spp * periods) for k in range(members)]
    b.run(spp * periods)
    P = [b.take(sl, psi=False, rho=False)["power"] for sl in slots]
    b.close()
    assert all(len(p) == spp * periods for p in P)
    ref = np.asarray(g["period_stats"])
    mean_ref = ref[10:, 0].mean()
    env_ref = np.median(ref[20:40, 1] / ref[20:40, 0])
    slow_ref = next(f for f, _ in g["periods_20_40"]["lines"] if f < 0.5)
    means = np.array([p[10 * spp:].mean() for p in P])
    envs = np.array([np.median(A.fluctuation(p, spp)[20:40]) for p in P])
    # strongest line below 0.5 cycles per period (every peak of the window considered)
    slows = np.array([next((f for f, _ in G.spectrum_lines(p[20 * spp:40 * spp], spp, 1 << 20) if f < 0.5), np.nan)
                      for p in P])
    m, sd = means.mean(), means.std(ddof=1)
    half = 2.0 * sd * np.sqrt(1.0 + 1.0 / members)  # two-sigma prediction interval of one more draw
    print(f"C5: mean P (periods 10-40) oracle {mean_ref:.4e}, GPU ensemble {m:.4e} +- {sd:.2e} "
          f"(member 0 {means[0]:.4e}, range {means.min():.4e}..{means.max():.4e}); "
          f"slow line {np.nanmedian(slows):.5f} vs {slow_ref:.5f}; envelope {np.median(envs):.4f} vs {env_ref:.4f}")
    print("C5 members: means", np.round(means / mean_ref, 3).tolist(), "slow lines", np.round(slows, 4).tolist(),
          "envelopes", np.round(envs, 3).tolist())
    assert all(A.is_bursting(p, spp, first=20, last=40) for p in P)
    assert abs(mean_ref - m) <= half, (mean_ref, m, sd)
    assert sd / m < 0.4, sd / m  # one regime: no member left the bursting of the others
    assert np.isfinite(slows).sum() >= members // 2, slows
    assert abs(np.nanmedian(slows) - slow_ref) <= 0.02 * slow_ref, (np.nanmedian(slows), slow_ref)
    assert abs(np.median(envs) - env_ref) <= 0.1 * env_ref, (np.median(envs), env_ref)
