"""CPU-side checks of the C-ABI library: it loads, exports every symbol that
include/vfps.h declares, and its host-only impedance tables agree with the
oracle's independent ones.  No compute call needs a GPU here."""
import os
import re

import numpy as np
import pytest

from oracle import oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def V():
    from paper_1611_05293_b300 import build
    build.build()
    from paper_1611_05293_b300 import vfps
    vfps.lib()
    return vfps


def header_symbols():
    src = open(os.path.join(ROOT, "include", "vfps.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(vfps_\w+)\s*\(", src)))


def test_library_exports_every_declared_symbol(V):
    syms = header_symbols()
    assert len(syms) >= 20
    L = V.lib()
    for s in syms:
        assert hasattr(L, s), s
    assert sorted(V.EXPORTS) == syms


def test_strerror_and_defaults(V):
    assert V.lib().vfps_strerror(0) == b"ok"
    assert V.lib().vfps_strerror(-5).startswith(b"non-finite")
    p = V.CParams()
    V.lib().vfps_params_default(p)
    assert (p.n, p.steps_per_period, p.interp_points, p.pad_factor, p.renormalize) == (256, 1000, 4, 2, 1)
    assert p.half_width == 6.0


@pytest.mark.parametrize("model,Pi,n,pad", [(1, 0.0, 64, 2), (2, 2.0, 64, 2), (2, 0.5, 256, 2),
                                            (2, 3.0, 100, 2), (2, 1.0, 128, 8)])
def test_library_impedance_matches_oracle(V, model, Pi, n, pad):
    """Two independent Airy evaluations (scipy's scaled Airy functions with a
    Hurwitz-zeta remainder in the oracle; series, K-Bessel integral and the
    large-x expansion in the library) agree to 1e-10 relative."""
    z = V.impedance_table(model, n, 6.0, pad, Pi)
    pr = O.Params(n=n, pad_factor=pad)
    zr, zi = O.impedance(pr, model, Pi)
    zo = zr + 1j * zi
    assert z.shape == zo.shape
    assert z[0] == 0
    rel = np.abs(z[1:] - zo[1:]) / np.abs(zo[1:])
    assert rel.max() < 1e-10


def test_impedance_table_rejects_bad_arguments(V):
    out = np.zeros(1024)
    L = V.lib()
    assert L.vfps_impedance_table(2, 64, 6.0, 2, 0.0, V._dptr(out)) == V.EINVAL
    assert L.vfps_impedance_table(5, 64, 6.0, 2, 1.0, V._dptr(out)) == V.EINVAL
    assert L.vfps_impedance_table(1, 4, 6.0, 2, 1.0, V._dptr(out)) == V.EINVAL
