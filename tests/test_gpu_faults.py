"""Failure paths, with the faults made on the host (no device fault):

* an allocation that fails (VFPS_FAULT_ALLOC=k makes the library's k-th
  device allocation return ENOMEM): the failing admission is refused
  cleanly, and the batch goes on with the slots it has, each equal to its
  solo run;
* a NaN in the initial state is refused (EINVAL) before any device work;
* a state with negative charge is refused (EINVAL); a run whose charge is
  lost on the device reports ENAN from the next synchronising call.
"""
import os
import subprocess
import sys
import textwrap

import numpy as np
import pytest

from paper_1611_05293_b300 import workloads as W

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def V():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1611_05293_b300 import vfps
    vfps.lib()
    return vfps


def test_failed_allocation_is_refused_and_batch_continues(V):
    code = textwrap.dedent("""
        import sys, numpy as np
        sys.path.insert(0, %r)
        from paper_1611_05293_b300 import vfps as V, workloads as W
        b = V.Batch(3)
        p = V.Params(n=64, steps_per_period=500, beta=1e-2)
        s0 = b.add(p, W.blobs(64, 1), V.IMPEDANCE_PARALLEL_PLATES, 2.0, 0.8, nsteps=20)   # allocation 1
        s1 = b.add(p, W.blobs(64, 2), V.IMPEDANCE_PARALLEL_PLATES, 2.0, 0.9, nsteps=20)   # allocation 2
        try:
            b.add(p, W.blobs(64, 3), V.IMPEDANCE_PARALLEL_PLATES, 2.0, 1.0, nsteps=20)    # allocation 3 fails
            print("NOERROR")
        except V.VfpsError as e:
            print("CODE", e.code)
        b.run(20)
        for s, seed, S in ((s0, 1, 0.8), (s1, 2, 0.9)):
            r = b.take(s)
            sim = V.Simulation(p, W.blobs(64, seed)); sim.set_impedance(V.IMPEDANCE_PARALLEL_PLATES, 2.0, S); sim.step(20)
            print("EQUAL", bool(np.array_equal(r["psi"], sim.get_state())))
            sim.close()
        print("USAGE", b.usage()[0])
        b.close()
    """) % ROOT
    env = dict(os.environ, VFPS_FAULT_ALLOC="3")
    out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = out.stdout.split()
    assert "CODE" in lines and lines[lines.index("CODE") + 1] == str(V.ENOMEM), out.stdout
    assert out.stdout.count("EQUAL True") == 2, out.stdout
    assert "USAGE" in lines and lines[lines.index("USAGE") + 1] == "2", out.stdout


def test_nan_input_is_refused(V):
    psi = W.blobs(32, 4)
    psi[3, 5] = np.nan
    with pytest.raises(V.VfpsError) as e:
        V.Simulation(V.Params(n=32, steps_per_period=100), psi)
    assert e.value.code == V.EINVAL


def test_negative_charge_is_refused(V):
    sim = V.Simulation(V.Params(n=32, steps_per_period=100, beta=1e-2), W.blobs(32, 5))
    with pytest.raises(V.VfpsError) as e:
        sim.set_state(-W.blobs(32, 6))   # finite, but its total charge is negative
    assert e.value.code == V.EINVAL
    sim.close()


@pytest.mark.parametrize("precision,n", [(0, 64), (0, 33), (1, 32)])
def test_charge_lost_on_device_reports_enan(V, precision, n):
    """S_csr = 1e6 kicks every cell ~1e5 cells off the grid in the first step
    (sources outside the grid give 0), so the charge after the step is zero:
    the finaliser flags it and the next synchronising call returns ENAN."""
    sim = V.Simulation(V.Params(n=n, steps_per_period=100, beta=1e-2, precision=precision), W.blobs(n, 7))
    sim.set_impedance(V.IMPEDANCE_PARALLEL_PLATES, 2.0, 1e6)
    sim.step(2)
    with pytest.raises(V.VfpsError) as e:
        sim.profile()
    assert e.value.code == V.ENAN
    sim.close()
