"""Moments recorded by the step itself, and the batched spectrogram, against
the oracle (through the C ABI).

* vfps_record_moments: the bunch length and energy spread the paper plots in
  its convergence studies (Sec. IV.A) -- {<q>, sigma_q, <p>, sigma_p} of every
  k-th state, formed by the step's epilogue -- against the oracle's moments
  of the oracle's state at the same steps: FP64 within 1e-11, FP32 within
  1e-5 (both rotations, the general and the FP32 streaming kernels).
  Recording changes no bit of the run, and a batch slot records the same
  bits as its solo run.
* vfps_spectrogram / vfps_batch_spectrogram: the paper's bursting
  spectrogram (Sec. IV.C), windows of the CSR-power series transformed on
  the device, against the oracle's power spectrum of the same windows
  (pinned on constants and cosines): within 1e-5 of the window's peak, the
  same strongest line; many slots in one launch equal their solo spectra.
"""
import numpy as np
import pytest

from oracle import oracle as O
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


@pytest.mark.parametrize("n,precision,rotation,tol", [
    (64, 1, 0, 1e-11), (64, 0, 0, 1e-5), (64, 0, 1, 1e-5), (100, 0, 0, 1e-5), (256, 0, 0, 1e-5),
    (48, 1, 1, 1e-11)])
def test_recorded_moments_match_oracle(V, n, precision, rotation, tol):
    spp, beta, S, Pi, every, chunks = 200, 0.05, 0.5, 2.0, 5, 12
    psi0 = W.blobs(n, 31)
    sim = V.Simulation(V.Params(n=n, steps_per_period=spp, beta=beta, precision=precision, rotation=rotation), psi0)
    sim.set_impedance(V.IMPEDANCE_PARALLEL_PLATES, Pi, S)
    sim.record_moments(every)
    sim.step(every * chunks)
    rec = sim.moment_series()
    sim.close()
    assert rec.shape == (chunks, 5)
    assert np.array_equal(rec[:, 0], every * np.arange(1, chunks + 1))
    op = O.Params(n=n, steps_per_period=spp, beta=beta, s_csr=S, rotation=rotation)
    zr, zi = O.impedance(op, 2, Pi)
    psi = O.normalize(op, psi0)
    for k in range(chunks):
        psi, _, _ = O.run(op, zr, zi, psi, every)
        ref = O.moments(op, psi)
        assert np.max(np.abs(rec[k, 1:] - ref)) < tol, (k, rec[k, 1:], ref)


def test_recording_changes_no_bit_and_batch_equals_solo(V):
    n, spp = 256, 1000
    psi0 = W.noisy_gaussian(n, 1611, 1e-6)
    pts = ((0.9, 2.0), (1.2, 1.0))
    states, series = {}, {}
    for rec_on in (False, True):
        for S, Pi in pts:
            sim = V.Simulation(V.Params(n=n, steps_per_period=spp, beta=1e-2), psi0)
            sim.set_impedance(V.IMPEDANCE_PARALLEL_PLATES, Pi, S)
            if rec_on:
                sim.record_moments(7)
            sim.step(100)
            states[(rec_on, S)] = (sim.get_state(), sim.csr_power())
            if rec_on:
                series[S] = sim.moment_series()
            sim.close()
    for S, _ in pts:
        assert np.array_equal(states[(False, S)][0], states[(True, S)][0])
        assert np.array_equal(states[(False, S)][1], states[(True, S)][1])
    b = V.Batch(4)
    slots = [b.add(V.Params(n=n, steps_per_period=spp, beta=1e-2), psi0, V.IMPEDANCE_PARALLEL_PLATES, Pi, S,
                   nsteps=100) for S, Pi in pts]
    for sl in slots:
        b.record_moments(sl, 7)
    b.run(100)
    for sl, (S, _) in zip(slots, pts):
        got = b.moment_series(sl)
        assert np.array_equal(got, series[S]), S
        assert np.array_equal(b.take(sl)["psi"], states[(True, S)][0])
    b.close()


def test_spectrogram_matches_oracle_and_batch_equals_solo(V):
    n, spp, S, Pi = 64, 500, 1.3, 2.0
    L, hop, count = 512, 256, 12
    sim = V.Simulation(V.Params(n=n, steps_per_period=spp, beta=1e-2), None)
    sim.set_impedance(V.IMPEDANCE_PARALLEL_PLATES, Pi, S)
    sim.step(6000)
    spec = sim.spectrogram(L, hop, count)
    last = sim.power_spectrum(L)
    P = sim.csr_power()
    sim.close()
    assert spec.shape == (count, L // 2 + 1)
    assert np.array_equal(spec[-1], last)
    T = len(P)
    span = L + (count - 1) * hop
    for w in range(count):
        a = T - span + w * hop
        ref = O.power_spectrum(P[a:a + L], L)
        assert np.max(np.abs(spec[w] - ref)) <= 1e-5 * ref.max(), w
        assert int(np.argmax(spec[w][1:])) == int(np.argmax(ref[1:])), w
    b = V.Batch(3)
    sl = [b.add(V.Params(n=n, steps_per_period=spp, beta=1e-2), None, V.IMPEDANCE_PARALLEL_PLATES, Pi, s_, nsteps=6000)
          for s_ in (S, 0.4, 2.0)]
    b.run(6000)
    many = b.spectrogram(sl, L, hop, count)
    b.close()
    assert many.shape == (3, count, L // 2 + 1)
    assert np.array_equal(many[0], spec)
    with pytest.raises(V.VfpsError):
        V.Simulation(V.Params(n=n, steps_per_period=spp), None).spectrogram(L, hop, count)  # no steps yet
