"""Python face of the FP64 CPU oracle (oracle/vfps_oracle.c).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
benchmark's ``cpu_baseline`` / ``--impl reference`` legs are the only
callers.  The product library never imports this module, and this module
imports nothing from the product.

``build()`` compiles the C file with gcc (-O2, OpenMP, no fast-math) into
``oracle/liboracle.so``; every other function loads that library.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

from . import impedance as _imp

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "vfps_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile liboracle.so next to its source (skipped when up to date)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared",
           "-o", _LIB + ".tmp", _SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(_LIB + ".tmp", _LIB)
    return _LIB


class _CParams(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("steps_per_period", ctypes.c_int),
                ("interp_points", ctypes.c_int), ("clamp", ctypes.c_int),
                ("fp_derivative", ctypes.c_int), ("pad_factor", ctypes.c_int),
                ("renormalize", ctypes.c_int), ("rotation", ctypes.c_int),
                ("half_width", ctypes.c_double),
                ("beta", ctypes.c_double), ("s_csr", ctypes.c_double)]


@dataclass
class Params:
    """Normalised problem: grid, time step, damping, interpolation, kick."""
    n: int = 64
    steps_per_period: int = 500
    beta: float = 1e-2
    s_csr: float = 0.0
    half_width: float = 6.0
    interp_points: int = 4
    clamp: int = 0
    fp_derivative: int = 1
    pad_factor: int = 2
    renormalize: int = 1
    rotation: int = 0      # 0: standard rotation, 1: Manhattan (drift, then RF kick)

    @property
    def delta(self) -> float:
        return 2.0 * self.half_width / (self.n - 1)

    @property
    def M(self) -> int:
        """FFT length: smallest power of two >= pad_factor * n."""
        return _imp.fft_length(self.n, self.pad_factor)

    def c(self) -> _CParams:
        return _CParams(self.n, self.steps_per_period, self.interp_points, self.clamp,
                        self.fp_derivative, self.pad_factor, self.renormalize, self.rotation,
                        self.half_width, self.beta, self.s_csr)


_D = ctypes.POINTER(ctypes.c_double)


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(_LIB):
            build()
        L = ctypes.CDLL(_LIB)
        P = ctypes.POINTER(_CParams)
        L.or_lagrange.argtypes = [ctypes.c_int, ctypes.c_double, _D]
        L.or_interp2.argtypes = [P, _D, ctypes.c_double, ctypes.c_double]
        L.or_interp2.restype = ctypes.c_double
        L.or_interp_p.argtypes = [P, _D, ctypes.c_int, ctypes.c_double]
        L.or_interp_p.restype = ctypes.c_double
        L.or_rotate.argtypes = [P, _D, _D]
        L.or_drift.argtypes = [P, _D, _D]
        L.or_rfkick.argtypes = [P, _D, _D]
        L.or_manhattan_h.argtypes = [P]
        L.or_manhattan_h.restype = ctypes.c_double
        L.or_project.argtypes = [P, _D, _D]
        L.or_project.restype = ctypes.c_double
        L.or_wake.argtypes = [P, _D, _D, _D, _D, _D]
        L.or_kick.argtypes = [P, _D, _D, _D]
        L.or_fokker_planck.argtypes = [P, _D, _D]
        L.or_moments.argtypes = [P, _D, _D]
        L.or_charge.argtypes = [P, _D]
        L.or_charge.restype = ctypes.c_double
        L.or_normalize.argtypes = [P, _D]
        L.or_normalize.restype = ctypes.c_double
        L.or_step.argtypes = [P, _D, _D, _D, _D, _D, _D, _D, _D]
        L.or_run.argtypes = [P, _D, _D, _D, ctypes.c_longlong, _D, _D]
        L.or_power_spectrum.argtypes = [_D, ctypes.c_int, _D]
        _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(_D)


def _grid(a, n):
    a = np.ascontiguousarray(a, dtype=np.float64)
    assert a.shape == (n, n), a.shape
    return a


def lagrange(ni: int, t: float) -> np.ndarray:
    w = np.zeros(4)
    lib().or_lagrange(ni, float(t), _p(w))
    return w[:ni].copy()


def interp2(pr: Params, psi, xr: float, yr: float) -> float:
    psi = _grid(psi, pr.n)
    return lib().or_interp2(ctypes.byref(pr.c()), _p(psi), float(xr), float(yr))


def rotate(pr: Params, psi) -> np.ndarray:
    psi = _grid(psi, pr.n)
    out = np.empty_like(psi)
    lib().or_rotate(ctypes.byref(pr.c()), _p(psi), _p(out))
    return out


def manhattan_h(pr: Params) -> float:
    return lib().or_manhattan_h(ctypes.byref(pr.c()))


def drift(pr: Params, psi) -> np.ndarray:
    psi = _grid(psi, pr.n)
    out = np.empty_like(psi)
    lib().or_drift(ctypes.byref(pr.c()), _p(psi), _p(out))
    return out


def rfkick(pr: Params, psi) -> np.ndarray:
    psi = _grid(psi, pr.n)
    out = np.empty_like(psi)
    lib().or_rfkick(ctypes.byref(pr.c()), _p(psi), _p(out))
    return out


def project(pr: Params, psi):
    """(rho, Q) of psi."""
    psi = _grid(psi, pr.n)
    rho = np.empty(pr.n)
    q = lib().or_project(ctypes.byref(pr.c()), _p(psi), _p(rho))
    return rho, q


def wake(pr: Params, zre, zim, rho):
    """(V, P) from the profile rho and the impedance table (M/2+1 values)."""
    zre = np.ascontiguousarray(zre, dtype=np.float64)
    zim = np.ascontiguousarray(zim, dtype=np.float64)
    assert zre.shape == (pr.M // 2 + 1,) and zim.shape == zre.shape
    rho = np.ascontiguousarray(rho, dtype=np.float64)
    V = np.empty(pr.n)
    P = np.zeros(1)
    lib().or_wake(ctypes.byref(pr.c()), _p(zre), _p(zim), _p(rho), _p(V), _p(P))
    return V, float(P[0])


def kick(pr: Params, V, psi) -> np.ndarray:
    psi = _grid(psi, pr.n)
    V = np.ascontiguousarray(V, dtype=np.float64)
    out = np.empty_like(psi)
    lib().or_kick(ctypes.byref(pr.c()), _p(V), _p(psi), _p(out))
    return out


def fokker_planck(pr: Params, psi) -> np.ndarray:
    psi = _grid(psi, pr.n)
    out = np.empty_like(psi)
    lib().or_fokker_planck(ctypes.byref(pr.c()), _p(psi), _p(out))
    return out


def moments(pr: Params, psi) -> np.ndarray:
    """(<q>, sigma_q, <p>, sigma_p) of psi."""
    psi = _grid(psi, pr.n)
    out = np.zeros(4)
    lib().or_moments(ctypes.byref(pr.c()), _p(psi), _p(out))
    return out


def charge(pr: Params, psi) -> float:
    return lib().or_charge(ctypes.byref(pr.c()), _p(_grid(psi, pr.n)))


def normalize(pr: Params, psi) -> np.ndarray:
    psi = _grid(psi, pr.n).copy()
    lib().or_normalize(ctypes.byref(pr.c()), _p(psi))
    return psi


def step(pr: Params, zre, zim, psi):
    """One time step.  Returns (psi_next, rho_t, V_t, P_t, Q_before_renorm)."""
    psi = _grid(psi, pr.n).copy()
    work = np.empty(2 * pr.n * pr.n)
    rho = np.empty(pr.n)
    V = np.empty(pr.n)
    P = np.zeros(1)
    Q = np.zeros(1)
    zre = np.ascontiguousarray(zre, dtype=np.float64)
    zim = np.ascontiguousarray(zim, dtype=np.float64)
    lib().or_step(ctypes.byref(pr.c()), _p(zre), _p(zim), _p(psi), _p(work),
                  _p(rho), _p(V), _p(P), _p(Q))
    return psi, rho, V, float(P[0]), float(Q[0])


def run(pr: Params, zre, zim, psi, nsteps: int):
    """nsteps steps.  Returns (psi_final, P_series, Q_series); P_series[t] is
    the CSR power of psi_t, Q_series[t] the charge before renormalising."""
    psi = _grid(psi, pr.n).copy()
    P = np.empty(nsteps)
    Q = np.empty(nsteps)
    zre = np.ascontiguousarray(zre, dtype=np.float64)
    zim = np.ascontiguousarray(zim, dtype=np.float64)
    lib().or_run(ctypes.byref(pr.c()), _p(zre), _p(zim), _p(psi), int(nsteps), _p(P), _p(Q))
    return psi, P, Q


def impedance(pr: Params, model: int, Pi: float = 0.0):
    """The oracle's impedance table on pr's FFT grid (see oracle.impedance)."""
    return _imp.impedance_table(model, pr.n, pr.half_width, pr.pad_factor, Pi)


def power_spectrum(x, L: int) -> np.ndarray:
    """|DFT|^2 (k = 0..L/2) of the last L values of x, mean removed, Hann window."""
    x = np.ascontiguousarray(np.asarray(x, dtype=np.float64)[-L:])
    assert x.size == L
    out = np.zeros(L // 2 + 1)
    lib().or_power_spectrum(_p(x), int(L), _p(out))
    return out
