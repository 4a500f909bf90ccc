"""FP32 against FP64 at the step rates of the workloads (Sec. IV.A).

The paper compares data types on a damped bunch (Table "datatype offset":
binary32 and binary64 agree on the converged bunch length to better than
1e-6) and lists the typical error of the data type as below 0.1 % (table of
typical errors).  It does not say at how many steps per period.  Here the
rounding of FP32 psi adds a fixed relative error per step while the
physical change per step shrinks as 1/steps, so the FP32 - FP64 difference
grows with the step rate.  These tests state and hold it at the rates the
workloads use -- 1000 steps/period (single runs and scans) and 4000 (the
large-grid run) -- for the two quantities the paper reports: the bunch
length sigma_q of a damped bunch, and the mean CSR power of a run with the
shielded wake below threshold.  The FP64 path itself matches the FP64 oracle
to 1e-10 (test_gpu_parity), so it serves as the reference here.
"""
import numpy as np
import pytest

from paper_1611_05293_b300 import workloads as W

pytestmark = pytest.mark.gpu

# stated bounds (relative), each above the measured value quoted beside it
SIGMA_BOUND = {1000: 5e-5, 4000: 5e-4}   # measured 1.5e-5 and 1.6e-4 (N = 256, 120 periods)
POWER_BOUND = {1000: 1e-4, 4000: 1e-3}


@pytest.fixture(scope="module")
def V():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1611_05293_b300 import vfps
    vfps.lib()
    return vfps


@pytest.mark.parametrize("spp", [1000, 4000])
def test_damped_bunch_length_fp32_vs_fp64(V, spp):
    """Set-up of the data-type study: sigma_q = sigma_p = 2.8 start, tau_d =
    5 T_s (beta = 0.2), no wake, N = 256, 120 periods; the relative FP32 -
    FP64 difference of sigma_q and sigma_p stays under the stated bound,
    which is below the paper's 0.1 %."""
    n, periods = 256, 120
    psi0 = W.gaussian(n, 6.0, 2.8, 2.8)
    sig = {}
    for precision in (1, 0):
        sim = V.Simulation(V.Params(n=n, steps_per_period=spp, beta=0.2, precision=precision), psi0)
        sim.step(spp * periods)
        sig[precision] = sim.moments()
        sim.close()
    err = np.abs(sig[0][[1, 3]] - sig[1][[1, 3]]) / sig[1][[1, 3]]
    print(f"spp={spp}: FP32-FP64 relative error of sigma_q, sigma_p = {err}")
    assert np.all(err < SIGMA_BOUND[spp]) and np.all(err < 1e-3), (spp, err)


@pytest.mark.parametrize("spp,n,Pi,periods", [(1000, 256, 2.0, 20), (4000, 1024, 1.0, 5)])
def test_mean_csr_power_fp32_vs_fp64(V, spp, n, Pi, periods):
    """Shielded CSR wake below threshold (S_csr = 0.5), Gaussian start with
    1e-6 noise, at the grid and step rate of the scans (N = 256, 1000
    steps/period) and of the large-grid run (N = 1024, 4000): the mean CSR
    power of the last half of the run, FP32 against FP64."""
    psi0 = W.noisy_gaussian(n, 1611, 1e-6)
    mean = {}
    for precision in (1, 0):
        sim = V.Simulation(V.Params(n=n, steps_per_period=spp, beta=1e-2, precision=precision), psi0)
        sim.set_impedance(V.IMPEDANCE_PARALLEL_PLATES, Pi, 0.5)
        sim.step(spp * periods)
        P = sim.csr_power()
        sim.close()
        mean[precision] = P[len(P) // 2:].mean()
    err = abs(mean[0] - mean[1]) / mean[1]
    print(f"spp={spp}, N={n}: FP32-FP64 relative error of <P> = {err:.3e}")
    assert err < POWER_BOUND[spp] and err < 1e-3, (spp, err)
