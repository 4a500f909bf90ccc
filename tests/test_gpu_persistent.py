"""Persistent launches of lone simulations (several steps per cooperative
launch, a dedicated finaliser CTA, bounded device waits).

* The persistent path gives the same bits as one ticketed launch per step
  (VFPS_PERSISTENT=0): state, CSR-power and charge series, recorded moments,
  for the compiled grid sizes (N = 256, 512 and 1024), a run-time size with 8- and
  4-row kick blocks, the Manhattan rotation, and step counts that cross
  launch boundaries.
* A wait that nothing ends runs out: with the finaliser CTA withholding its
  tagged kick records (test hook VFPS_FAULT_NO_SIGNAL) the launch returns
  within the spin limit, the next synchronising call reports ETIMEOUT, and
  the context stays usable for the next simulation.  The failure is made by a flag that
  nothing sets; no device fault is involved.
"""
import contextlib
import os
import time

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


@contextlib.contextmanager
def env(**kv):
    old = {k: os.environ.get(k) for k in kv}
    os.environ.update({k: str(v) for k, v in kv.items()})
    try:
        yield
    finally:
        for k, v in old.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v


def run(V, params, Pi, S, chunks, persistent, every=0, seed=1612):
    """Run one simulation in step() calls of the given sizes; return state,
    power and charge series, moment series (or None) and the step mode."""
    with env(VFPS_PERSISTENT="1" if persistent else "0"):
        sim = V.Simulation(params, W.noisy_gaussian(params.n, seed, 1e-6))
    try:
        sim.set_impedance(V.IMPEDANCE_PARALLEL_PLATES, Pi, S)
        if every:
            sim.record_moments(every)
        for c in chunks:
            sim.step(c)
        out = (sim.get_state(), sim.csr_power(), sim.charge_series(),
               sim.moment_series() if every else None, sim.persistent)
    finally:
        sim.close()
    return out


CASES = [
    # (name, n, steps/period, Pi, S_csr, rotation, step() calls)
    ("n256_bursting", 256, 1000, 2.0, 0.9, 0, [300]),
    ("n1024_c5", 1024, 4000, 1.0, 3.0, 0, [100]),
    ("n512_two_warps_per_column", 512, 2000, 2.0, 1.2, 0, [150]),
    ("n512_manhattan", 512, 2000, 2.0, 1.2, 1, [100]),
    ("n128_runtime_size", 128, 500, 2.0, 0.9, 0, [120]),
    ("n60_four_row_blocks", 60, 500, 1.0, 0.8, 0, [90]),
    ("n256_manhattan", 256, 1000, 2.0, 0.9, 1, [200]),
    ("n256_launch_boundaries", 256, 1000, 2.0, 0.9, 0, [3, 300, 1, 257]),
]


@pytest.mark.parametrize("name,n,spp,Pi,S,rot,chunks", CASES, ids=[c[0] for c in CASES])
def test_persistent_steps_give_the_ticketed_bits(V, name, n, spp, Pi, S, rot, chunks):
    p = V.Params(n=n, steps_per_period=spp, beta=1e-2, rotation=rot)
    psi_a, P_a, Q_a, _, mode_a = run(V, p, Pi, S, chunks, True)
    psi_b, P_b, Q_b, _, mode_b = run(V, p, Pi, S, chunks, False)
    assert mode_a and not mode_b, "the two runs must take the two launch modes"
    assert len(P_a) == sum(chunks)
    assert np.array_equal(P_a, P_b)
    assert np.array_equal(Q_a, Q_b)
    assert np.array_equal(psi_a, psi_b)
    assert np.all(np.isfinite(psi_a)) and P_a[-1] > 0


def test_persistent_moment_recording_gives_the_ticketed_bits(V):
    p = V.Params(n=256, steps_per_period=1000, beta=1e-2)
    a = run(V, p, 2.0, 0.9, [150], True, every=7)
    b = run(V, p, 2.0, 0.9, [150], False, every=7)
    assert a[4] and not b[4]
    assert len(a[3]) == 150 // 7
    assert np.array_equal(a[3], b[3])
    assert np.array_equal(a[0], b[0])


def test_bounded_wait_runs_out_with_etimeout(V):
    p = V.Params(n=256, steps_per_period=1000, beta=1e-2)
    with env(VFPS_FAULT_NO_SIGNAL="1", VFPS_SPIN_LIMIT="20000"):
        sim = V.Simulation(p)
    try:
        assert sim.persistent
        t0 = time.time()
        sim.step(4)  # step 0 completes; the workers then wait for kick records that never come
        with pytest.raises(V.VfpsError) as ei:
            sim.csr_power()
        assert ei.value.code == V.ETIMEOUT
        assert time.time() - t0 < 20.0
    finally:
        sim.close()
    # the context is still usable, and the next simulation is unaffected
    psi_a, P_a, _, _, mode_a = run(V, p, 2.0, 0.9, [40], True)
    psi_b, P_b, _, _, _ = run(V, p, 2.0, 0.9, [40], False)
    assert mode_a
    assert np.array_equal(P_a, P_b) and np.array_equal(psi_a, psi_b)


@pytest.mark.parametrize("n,spp,S,Pi", [(256, 1000, 0.9, 2.0), (1024, 4000, 3.0, 1.0)])
def test_concurrent_persistent_simulations_keep_their_bits(V, n, spp, S, Pi):
    """Two lone simulations stepping at once on their own streams (at N=1024
    their two grids of one-per-SM CTAs cannot be resident together, so the
    cooperative launches take turns): no wait runs out, and each ends with
    the bits of its solo run."""
    import torch

    def make(stream, seed):
        sim = V.Simulation(V.Params(n=n, steps_per_period=spp, beta=1e-2), W.noisy_gaussian(n, seed, 1e-6), stream)
        sim.set_impedance(V.IMPEDANCE_PARALLEL_PLATES, Pi, S)
        return sim

    a, b = make(torch.cuda.Stream(), 1), make(torch.cuda.Stream(), 2)
    try:
        assert a.persistent and b.persistent
        for _ in range(4):
            a.step(300)
            b.step(300)
        got = [(a.get_state(), a.csr_power()), (b.get_state(), b.csr_power())]
    finally:
        a.close()
        b.close()
    for seed, (psi, P) in zip((1, 2), got):
        sim = make(None, seed)
        sim.step(1200)
        assert np.array_equal(psi, sim.get_state()) and np.array_equal(P, sim.csr_power()), seed
        sim.close()
