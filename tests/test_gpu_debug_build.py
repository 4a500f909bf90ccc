"""The debug build (VFPS_DEBUG: shared-memory index checks that record the
failing site and skip the access, reported as EBOUNDS; no device fault)
against the release build: over grid sizes (ragged, fast and general
kernels, the compiled-in sizes 256 and 1024), both rotations, pinned
launch shapes and the pair kernel, no check fires and both builds give the
same bits."""
import os
import subprocess
import sys
import textwrap

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = textwrap.dedent("""
    import sys, numpy as np
    sys.path.insert(0, %(root)r)
    from paper_1611_05293_b300 import vfps as V, workloads as W, build as B
    V.LIB_PATH = B.build(debug=%(debug)s)
    out = {}
    for n in (8, 12, 36, 64, 100, 256, 1024):
        for rot in (0, 1):
            p = V.Params(n=n, steps_per_period=500, beta=1e-2, rotation=rot)
            sim = V.Simulation(p, W.blobs(n, n + rot)); sim.set_impedance(2, 2.0, 0.9); sim.step(3)
            out[f"solo_{n}_{rot}"] = sim.get_state(); sim.close()
            for Wd, tps in ((2, 1), (4, 4), (8, 1), (8, 4), (4, -1), (8, -1)):
                for pair in (False, True):
                    b = V.Batch(2); b.autotune(False); b.pin_shape(Wd, tps); b.pairing(pair)
                    s = [b.add(p, W.blobs(n, 7 * i + n), 2, 2.0, 0.7 + 0.2 * i, nsteps=3) for i in range(2)]
                    b.run(3)
                    for i, sl in enumerate(s):
                        out[f"b_{n}_{rot}_{Wd}_{tps}_{int(pair)}_{i}"] = b.take(sl)["psi"]
                    b.close()
    np.savez(%(path)r, **out)
    print("OK")
""")


def test_debug_build_has_no_index_failures_and_same_bits(tmp_path):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    res = {}
    for debug in (False, True):
        path = str(tmp_path / f"out_{int(debug)}.npz")
        code = SCRIPT % {"root": ROOT, "debug": debug, "path": path}
        run = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=1200)
        assert run.returncode == 0 and "OK" in run.stdout, run.stderr[-3000:]
        res[debug] = np.load(path)
    assert sorted(res[False].files) == sorted(res[True].files)
    for k in res[False].files:
        assert np.array_equal(res[False][k], res[True][k]), k
