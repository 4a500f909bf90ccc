"""Haissinski start on the device (vfps_haissinski) against the oracle's
solver of the same fixed-point equation (oracle/haissinski.py): the profile
and the state rho_H(q) g(p), FP64 and FP32 simulations, a batch slot against
the same simulation alone, the equilibrium it starts (below threshold the
CSR power stays put), and the failure path (too few iterations: ECONVERGE,
state unchanged)."""
import numpy as np
import pytest

from oracle import haissinski as H
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


def oracle_start(n, spp, S, Pi, pad=2):
    op = O.Params(n=n, steps_per_period=spp, beta=1e-2, s_csr=S, pad_factor=pad)
    zr, zi = O.impedance(op, 2, Pi)
    return H.profile(op, zr, zi), H.density(op, zr, zi)


@pytest.mark.parametrize("n,precision,S,Pi,tol,pad", [(64, 1, 0.3, 2.0, 1e-10, 2), (100, 1, 0.6, 1.0, 1e-10, 2),
                                                      (256, 0, 0.6, 1.0, 2e-6, 2), (128, 0, 0.4, 3.0, 2e-6, 2),
                                                      (64, 1, 0.5, 2.0, 1e-10, 8), (1024, 0, 0.5, 2.0, 2e-6, 2)])
def test_device_haissinski_matches_oracle(V, n, precision, S, Pi, tol, pad):
    spp = 500
    sim = V.Simulation(V.Params(n=n, steps_per_period=spp, beta=1e-2, precision=precision, pad_factor=pad))
    sim.set_impedance(V.IMPEDANCE_PARALLEL_PLATES, Pi, S)
    iters = sim.haissinski(tol=1e-13)
    assert 1 < iters < 20000
    rho_ref, psi_ref = oracle_start(n, spp, S, Pi, pad)
    rho = sim.profile()
    psi = sim.get_state()
    sim.close()
    assert np.max(np.abs(rho - rho_ref)) / rho_ref.max() < tol
    assert np.max(np.abs(psi - psi_ref)) / psi_ref.max() < tol


def test_batch_slot_haissinski_equals_solo(V):
    n, spp, S, Pi = 96, 500, 0.5, 2.0
    p = V.Params(n=n, steps_per_period=spp, beta=1e-2)
    sim = V.Simulation(p)
    sim.set_impedance(V.IMPEDANCE_PARALLEL_PLATES, Pi, S)
    it_solo = sim.haissinski()
    sim.step(20)
    solo = sim.get_state(), sim.csr_power()
    sim.close()
    b = V.Batch(2)
    other = b.add(p, W.blobs(n, 5), V.IMPEDANCE_PARALLEL_PLATES, 1.0, 0.9, nsteps=20)
    sl = b.add(p, None, V.IMPEDANCE_PARALLEL_PLATES, Pi, S, nsteps=20)
    assert b.haissinski(sl) == it_solo
    b.run(20)
    r = b.take(sl)
    b.take(other)
    b.close()
    assert np.array_equal(r["psi"], solo[0])
    assert np.array_equal(r["power"], solo[1])


def test_equilibrium_start_keeps_csr_power_below_threshold(V):
    """Started at its Haissinski equilibrium (S = 0.4 < threshold), the run
    stays there: the CSR power over one synchrotron period moves by much less
    than from a Gaussian start."""
    n, spp, S, Pi = 128, 500, 0.4, 2.0
    p = V.Params(n=n, steps_per_period=spp, beta=1e-2)
    drift = {}
    for start in ("gaussian", "haissinski"):
        sim = V.Simulation(p)
        sim.set_impedance(V.IMPEDANCE_PARALLEL_PLATES, Pi, S)
        if start == "haissinski":
            sim.haissinski()
        sim.step(spp)
        P = sim.csr_power()
        sim.close()
        drift[start] = (P.max() - P.min()) / P.mean()
    assert drift["haissinski"] < 0.05
    assert drift["haissinski"] < 0.2 * drift["gaussian"]


def test_not_converged_leaves_state_unchanged(V):
    n = 64
    sim = V.Simulation(V.Params(n=n, steps_per_period=500, beta=1e-2), W.blobs(n, 3))
    sim.set_impedance(V.IMPEDANCE_PARALLEL_PLATES, 2.0, 0.8)
    before, rho_before = sim.get_state(), sim.profile()
    with pytest.raises(V.VfpsError) as e:
        sim.haissinski(tol=1e-13, max_iter=2)
    assert e.value.code == V.ECONVERGE
    assert np.array_equal(sim.get_state(), before)
    assert np.array_equal(sim.profile(), rho_before)
    with pytest.raises(V.VfpsError):
        sim.haissinski(tol=0.0)
    sim.close()


def test_adiabatic_chaining_of_scan_points(V):
    """A current scan chained adiabatically (Sec. IV.C: each point starts from
    the previous point's final state, through vfps_set_state), from a
    Haissinski start at the first point; FP64 against the oracle doing the
    same chain."""
    n, spp, Pi, steps = 48, 400, 2.0, 60
    Ss = (0.3, 0.5, 0.7)
    p = V.Params(n=n, steps_per_period=spp, beta=1e-2, precision=1)
    sim = V.Simulation(p)
    sim.set_impedance(V.IMPEDANCE_PARALLEL_PLATES, Pi, Ss[0])
    sim.haissinski()
    got = []
    for i, S in enumerate(Ss):
        if i:
            state = sim.get_state()
            sim.set_impedance(V.IMPEDANCE_PARALLEL_PLATES, Pi, S)
            sim.set_state(state)
        sim.step(steps)
        got.append((sim.get_state(), sim.csr_power()[-steps:]))
    sim.close()
    op = O.Params(n=n, steps_per_period=spp, beta=1e-2, s_csr=Ss[0])
    zr, zi = O.impedance(op, 2, Pi)
    psi = H.density(op, zr, zi)
    for (g_psi, g_pow), S in zip(got, Ss):
        op = O.Params(n=n, steps_per_period=spp, beta=1e-2, s_csr=S)
        psi, P, _ = O.run(op, zr, zi, O.normalize(op, psi), steps)
        assert np.max(np.abs(g_psi - psi)) / psi.max() < 1e-9, S
        assert np.max(np.abs(g_pow - P) / P) < 1e-9, S
