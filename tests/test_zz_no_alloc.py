"""The allocation-free step (vfps_step_static) against the handle API.

vfps_step_static serves callers that may not allocate device memory (an
application pool owns the device, or a latency-critical loop cannot afford
cudaMalloc).  It must give the same next state and CSR power as
vfps_create + vfps_step on the same input, within the FP32 per-step
tolerance (1e-5 relative L-inf), on two calls in a row -- the second call
reuses the scratch that the first one left behind.  This file runs last
(pytest collects it after the other test files).
"""
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_1611_05293_b300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1611_05293_b300 import vfps
    vfps.lib()
    return torch, vfps


def rel_linf(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


@pytest.mark.parametrize("n", [64, 66])   # 64: register-blocked kernel, 66: general kernel
def test_static_step_matches_handle_on_two_calls(env, n):
    torch, V = env
    params = V.Params(n=n, steps_per_period=500, beta=1e-2)
    sim = V.Simulation(params, W.blobs(n, 21))
    sim.set_impedance(V.IMPEDANCE_PARALLEL_PLATES, 2.0, 0.9)
    s0 = sim.get_state()
    sim.step(1)
    s1 = sim.get_state()
    sim.step(1)
    s2 = sim.get_state()
    P = sim.csr_power()
    sim.close()

    stream = torch.cuda.current_stream()
    x0 = torch.tensor(s0, dtype=torch.float32, device="cuda")
    y1 = torch.empty_like(x0)
    y2 = torch.empty_like(x0)
    p0 = V.step_static(params, V.IMPEDANCE_PARALLEL_PLATES, 2.0, 0.9, x0.data_ptr(), y1.data_ptr(), stream)
    p1 = V.step_static(params, V.IMPEDANCE_PARALLEL_PLATES, 2.0, 0.9, y1.data_ptr(), y2.data_ptr(), stream)
    torch.cuda.synchronize()
    assert rel_linf(y1.double().cpu().numpy(), s1) < 1e-5
    assert rel_linf(y2.double().cpu().numpy(), s2) < 1e-5
    assert abs(p0 - P[0]) < 1e-5 * P[0]
    assert abs(p1 - P[1]) < 1e-5 * P[1]


def test_static_step_rejects_sizes_beyond_its_scratch(env):
    torch, V = env
    x = torch.zeros((2048, 2048), dtype=torch.float32, device="cuda")
    y = torch.zeros_like(x)
    with pytest.raises(V.VfpsError) as e:
        V.step_static(V.Params(n=2048, steps_per_period=4000), 1, 0.0, 0.5, x.data_ptr(), y.data_ptr())
    assert e.value.code == V.EINVAL
    assert "exceeds the static scratch limit" in str(e.value)


def test_static_step_normalises_any_input_charge(env):
    """psi_in may carry any positive charge and psi_out comes back with charge
    1, whatever the params' renormalize flag says: a state scaled by 3 gives
    the same next state and power as the unit-charge one."""
    torch, V = env
    n = 64
    for renorm in (1, 0):
        params = V.Params(n=n, steps_per_period=500, beta=1e-2, renormalize=renorm)
        sim = V.Simulation(V.Params(n=n, steps_per_period=500, beta=1e-2), W.blobs(n, 22))
        s0 = sim.get_state()
        sim.close()
        x1 = torch.tensor(s0, dtype=torch.float32, device="cuda")
        x3 = 3.0 * x1
        y1, y3 = torch.empty_like(x1), torch.empty_like(x1)
        p1 = V.step_static(params, V.IMPEDANCE_PARALLEL_PLATES, 2.0, 0.9, x1.data_ptr(), y1.data_ptr())
        p3 = V.step_static(params, V.IMPEDANCE_PARALLEL_PLATES, 2.0, 0.9, x3.data_ptr(), y3.data_ptr())
        torch.cuda.synchronize()
        a, b = y1.double().cpu().numpy(), y3.double().cpu().numpy()
        assert rel_linf(b, a) < 1e-6, renorm
        assert abs(p3 - p1) < 1e-6 * p1, (renorm, p1, p3)
        delta = 12.0 / (n - 1)
        assert abs(delta * delta * a.sum() - 1.0) < 1e-5, renorm


_NO_ALLOC_SCRIPT = r"""
import sys, torch
sys.path.insert(0, sys.argv[1])
from paper_1611_05293_b300 import vfps as V, workloads as W
n = 64
params = V.Params(n=n, steps_per_period=500, beta=1e-2)
x = torch.tensor(W.blobs(n, 23), dtype=torch.float32, device="cuda")
y = torch.empty_like(x)
V.step_static(params, V.IMPEDANCE_PARALLEL_PLATES, 2.0, 0.9, x.data_ptr(), y.data_ptr())
torch.cuda.synchronize()
free0 = torch.cuda.mem_get_info()[0]
for _ in range(3):
    V.step_static(params, V.IMPEDANCE_PARALLEL_PLATES, 2.0, 0.9, y.data_ptr(), x.data_ptr())
    V.step_static(params, V.IMPEDANCE_PARALLEL_PLATES, 2.0, 0.9, x.data_ptr(), y.data_ptr())
torch.cuda.synchronize()
assert torch.cuda.mem_get_info()[0] == free0, "device memory changed"
assert bool(torch.isfinite(y).all())
print("NO_ALLOC_OK")
"""


def test_static_step_allocates_nothing(env):
    """In a fresh process whose first library device allocation is made to
    fail (VFPS_FAULT_ALLOC=1, the library's host-side fault injector), seven
    calls in a row still succeed, and after the first one (which loads the
    module and looks up the scratch address) the free device memory does not
    change."""
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env_vars = dict(os.environ, VFPS_FAULT_ALLOC="1")
    out = subprocess.run([sys.executable, "-c", _NO_ALLOC_SCRIPT, root], env=env_vars, capture_output=True,
                         text=True, timeout=300)
    assert out.returncode == 0 and "NO_ALLOC_OK" in out.stdout, (out.stdout[-2000:], out.stderr[-2000:])
