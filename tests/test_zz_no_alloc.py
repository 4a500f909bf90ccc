"""The allocation-free step (vfps_step_static) against the handle API.

vfps_step_static serves callers that may not allocate device memory (an
application pool owns the device, or a latency-critical loop cannot afford
cudaMalloc).  It must give the same next state and CSR power as
vfps_create + vfps_step on the same input, within the FP32 per-step
tolerance (1e-5 relative L-inf), on two calls in a row -- the second call
reuses the scratch that the first one left behind.  This file runs last
(pytest collects it after the other test files).
"""
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
