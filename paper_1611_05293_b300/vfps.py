"""Python binding of libvfps.so (include/vfps.h): argument marshalling only.

Every step of the solver runs in the library's CUDA kernels; this module
converts NumPy arrays to pointers, checks return codes and raises
``VfpsError``.  There is no fallback: if the in-tree library is missing the
import of the binding fails.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libvfps.so")

OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, ENAN, EBUSY, EBOUNDS, ECONVERGE = 0, -1, -2, -3, -4, -5, -6, -7, -8
IMPEDANCE_NONE, IMPEDANCE_FREE_SPACE, IMPEDANCE_PARALLEL_PLATES, IMPEDANCE_TABLE = 0, 1, 2, 3

# every symbol include/vfps.h declares
EXPORTS = [
    "vfps_params_default", "vfps_create", "vfps_set_impedance", "vfps_step", "vfps_profile",
    "vfps_csr_power", "vfps_charge_series", "vfps_get_state", "vfps_set_state",
    "vfps_steps_done", "vfps_step_mode", "vfps_destroy", "vfps_strerror", "vfps_last_cuda_error", "vfps_impedance_table",
    "vfps_batch_create", "vfps_batch_add", "vfps_batch_slot_bytes", "vfps_batch_run",
    "vfps_batch_poll", "vfps_batch_take", "vfps_batch_remove", "vfps_batch_usage",
    "vfps_batch_destroy", "vfps_step_static", "vfps_batch_launches_per_step",
    "vfps_moments", "vfps_batch_moments", "vfps_batch_autotune", "vfps_batch_shapes",
    "vfps_batch_pin_shape", "vfps_power_spectrum", "vfps_batch_power_spectrum", "vfps_batch_pairing",
    "vfps_haissinski", "vfps_batch_haissinski",
    "vfps_record_moments", "vfps_moment_series", "vfps_spectrogram",
    "vfps_batch_record_moments", "vfps_batch_moment_series", "vfps_batch_spectrogram", "vfps_batch_idle",
    "vfps_checkpoint_bytes", "vfps_save_checkpoint", "vfps_load_checkpoint",
    "vfps_batch_add_many", "vfps_batch_take_many",
]


class VfpsError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        msg = f"{what}: {_lib_strerror(code)} ({code})"
        if code == ECUDA:
            try:
                msg += f" [{lib().vfps_last_cuda_error().decode()}]"
            except Exception:
                pass
        super().__init__(msg)


class CParams(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("steps_per_period", ctypes.c_int32),
                ("interp_points", ctypes.c_int32), ("clamp", ctypes.c_int32),
                ("fp_derivative", ctypes.c_int32), ("pad_factor", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("renormalize", ctypes.c_int32),
                ("rotation", ctypes.c_int32),
                ("half_width", ctypes.c_double), ("beta", ctypes.c_double)]


@dataclass
class Params:
    """Mirror of vfps_params (defaults as in vfps_params_default)."""
    n: int = 256
    steps_per_period: int = 1000
    beta: float = 0.0
    half_width: float = 6.0
    interp_points: int = 4
    clamp: int = 0
    fp_derivative: int = 1
    pad_factor: int = 2
    precision: int = 0
    renormalize: int = 1
    rotation: int = 0   # 0 standard rotation, 1 Manhattan rotation (drift, then RF kick)

    def c(self) -> CParams:
        return CParams(self.n, self.steps_per_period, self.interp_points, self.clamp,
                       self.fp_derivative, self.pad_factor, self.precision, self.renormalize,
                       self.rotation, self.half_width, self.beta)


_lib = None
_D = ctypes.POINTER(ctypes.c_double)
_VP = ctypes.c_void_p
_I64 = ctypes.c_int64
_I32 = ctypes.c_int32


def lib() -> ctypes.CDLL:
    """Load the in-tree library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libvfps.so not built at {LIB_PATH}; run paper_1611_05293_b300/build.py")
    L = ctypes.CDLL(LIB_PATH)
    P = ctypes.POINTER(CParams)
    sig = {
        "vfps_params_default": (None, [P]),
        "vfps_create": (ctypes.c_int, [P, _D, _VP, ctypes.POINTER(_VP)]),
        "vfps_set_impedance": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_double, ctypes.c_double, _D]),
        "vfps_step": (ctypes.c_int, [_VP, _I64]),
        "vfps_profile": (ctypes.c_int, [_VP, _D]),
        "vfps_moments": (ctypes.c_int, [_VP, _D]),
        "vfps_power_spectrum": (ctypes.c_int, [_VP, _I32, _D]),
        "vfps_batch_power_spectrum": (ctypes.c_int, [_VP, _I32, _I32, _D]),
        "vfps_batch_moments": (ctypes.c_int, [_VP, _I32, _D]),
        "vfps_batch_autotune": (ctypes.c_int, [_VP, _I32]),
        "vfps_batch_pin_shape": (ctypes.c_int, [_VP, _I32, _I32]),
        "vfps_batch_pairing": (ctypes.c_int, [_VP, _I32]),
        "vfps_haissinski": (ctypes.c_int, [_VP, ctypes.c_double, _I32, ctypes.POINTER(_I32)]),
        "vfps_batch_haissinski": (ctypes.c_int, [_VP, _I32, ctypes.c_double, _I32, ctypes.POINTER(_I32)]),
        "vfps_batch_shapes": (ctypes.c_int, [_VP, ctypes.POINTER(_I32), _I32, ctypes.POINTER(_I32)]),
        "vfps_csr_power": (ctypes.c_int, [_VP, _D, _I64, ctypes.POINTER(_I64)]),
        "vfps_charge_series": (ctypes.c_int, [_VP, _D, _I64, ctypes.POINTER(_I64)]),
        "vfps_get_state": (ctypes.c_int, [_VP, _D]),
        "vfps_set_state": (ctypes.c_int, [_VP, _D]),
        "vfps_steps_done": (ctypes.c_int, [_VP, ctypes.POINTER(_I64)]),
        "vfps_step_mode": (ctypes.c_int, [_VP, ctypes.POINTER(_I32)]),
        "vfps_destroy": (ctypes.c_int, [_VP]),
        "vfps_strerror": (ctypes.c_char_p, [ctypes.c_int]),
        "vfps_last_cuda_error": (ctypes.c_char_p, []),
        "vfps_impedance_table": (ctypes.c_int, [ctypes.c_int, _I32, ctypes.c_double, _I32,
                                                ctypes.c_double, _D]),
        "vfps_batch_create": (ctypes.c_int, [_I32, _I64, _VP, ctypes.POINTER(_VP)]),
        "vfps_batch_add": (ctypes.c_int, [_VP, P, _D, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                          _D, _I64, ctypes.POINTER(_I32)]),
        "vfps_batch_slot_bytes": (_I64, [P]),
        "vfps_batch_run": (ctypes.c_int, [_VP, _I64]),
        "vfps_batch_poll": (ctypes.c_int, [_VP, ctypes.POINTER(_I32), _I32, ctypes.POINTER(_I32)]),
        "vfps_batch_take": (ctypes.c_int, [_VP, _I32, _D, _D, _D, _I64, ctypes.POINTER(_I64),
                                           ctypes.POINTER(_I64)]),
        "vfps_batch_remove": (ctypes.c_int, [_VP, _I32]),
        "vfps_batch_usage": (ctypes.c_int, [_VP, ctypes.POINTER(_I32), ctypes.POINTER(_I64)]),
        "vfps_batch_launches_per_step": (ctypes.c_int, [_VP, ctypes.POINTER(_I32)]),
        "vfps_batch_destroy": (ctypes.c_int, [_VP]),
        "vfps_step_static": (ctypes.c_int, [P, ctypes.c_int, ctypes.c_double, ctypes.c_double, _VP, _VP,
                                            _D, _VP]),
        "vfps_record_moments": (ctypes.c_int, [_VP, _I32]),
        "vfps_moment_series": (ctypes.c_int, [_VP, _D, _I64, ctypes.POINTER(_I64)]),
        "vfps_spectrogram": (ctypes.c_int, [_VP, _I32, _I32, _I32, _D]),
        "vfps_batch_record_moments": (ctypes.c_int, [_VP, _I32, _I32]),
        "vfps_batch_idle": (ctypes.c_int, [_VP, ctypes.POINTER(_I32)]),
        "vfps_checkpoint_bytes": (ctypes.c_int, [_VP, ctypes.POINTER(_I64)]),
        "vfps_batch_add_many": (ctypes.c_int, [_VP, _I32, P, _D, ctypes.c_int, _D, _D, _I64,
                                               ctypes.POINTER(_I32)]),
        "vfps_batch_take_many": (ctypes.c_int, [_VP, _I32, ctypes.POINTER(_I32), _D, _D, _I64,
                                                ctypes.POINTER(_I64)]),
        "vfps_save_checkpoint": (ctypes.c_int, [_VP, ctypes.c_void_p, _I64]),
        "vfps_load_checkpoint": (ctypes.c_int, [_VP, ctypes.c_void_p, _I64]),
        "vfps_batch_moment_series": (ctypes.c_int, [_VP, _I32, _D, _I64, ctypes.POINTER(_I64)]),
        "vfps_batch_spectrogram": (ctypes.c_int, [_VP, ctypes.POINTER(_I32), _I32, _I32, _I32, _I32, _D]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def _lib_strerror(code: int) -> str:
    try:
        return lib().vfps_strerror(code).decode()
    except Exception:  # library not loadable while formatting an error
        return "error"


def _check(rc: int, what: str) -> None:
    if rc != OK:
        raise VfpsError(rc, what)


def _dptr(a):
    return None if a is None else a.ctypes.data_as(_D)


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None and a.shape != shape:
        raise ValueError(f"expected shape {shape}, got {a.shape}")
    return a


def _stream_ptr(stream):
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


def impedance_table(model: int, n: int, half_width: float = 6.0, pad_factor: int = 2,
                    Pi: float = 0.0) -> np.ndarray:
    """Host-side library impedance table (complex, M/2+1 values)."""
    M = 1
    while M < pad_factor * n:
        M <<= 1
    out = np.zeros(M + 2)
    _check(lib().vfps_impedance_table(model, n, half_width, pad_factor, Pi, _dptr(out)),
           "vfps_impedance_table")
    return out[0::2] + 1j * out[1::2]


class Simulation:
    """One simulation handle (vfps_create ... vfps_destroy)."""

    def __init__(self, params: Params, psi0=None, stream=None):
        self.params = params
        n = params.n
        psi = None if psi0 is None else _f64(psi0, (n, n))
        h = _VP()
        _check(lib().vfps_create(ctypes.byref(params.c()), _dptr(psi), _stream_ptr(stream),
                                 ctypes.byref(h)), "vfps_create")
        self._h = h
        self._taken = {}  # series name -> values drained so far

    def set_impedance(self, model: int, Pi: float = 0.0, S_csr: float = 0.0, table=None):
        tab = None
        if table is not None:
            t = np.asarray(table, dtype=np.complex128)
            tab = np.empty(2 * t.size)
            tab[0::2], tab[1::2] = t.real, t.imag
        _check(lib().vfps_set_impedance(self._h, model, Pi, S_csr, _dptr(tab)), "vfps_set_impedance")

    def step(self, nsteps: int):
        _check(lib().vfps_step(self._h, int(nsteps)), "vfps_step")

    def profile(self) -> np.ndarray:
        out = np.empty(self.params.n)
        _check(lib().vfps_profile(self._h, _dptr(out)), "vfps_profile")
        return out

    def power_spectrum(self, length: int) -> np.ndarray:
        """|DFT|^2 of the last `length` CSR-power values (mean removed, Hann), on the device."""
        out = np.empty(length // 2 + 1)
        _check(lib().vfps_power_spectrum(self._h, int(length), _dptr(out)), "vfps_power_spectrum")
        return out

    def moments(self) -> np.ndarray:
        """(<q>, sigma_q, <p>, sigma_p) of the current state, computed on the device."""
        out = np.empty(4)
        _check(lib().vfps_moments(self._h, _dptr(out)), "vfps_moments")
        return out

    def record_moments(self, every: int):
        """Record (<q>, sigma_q, <p>, sigma_p) of every `every`-th state as part
        of the step (0 stops)."""
        _check(lib().vfps_record_moments(self._h, int(every)), "vfps_record_moments")

    def moment_series(self, cap: int = 1 << 20) -> np.ndarray:
        """Drain the recorded moments: rows (t, <q>, sigma_q, <p>, sigma_p)."""
        out = np.empty((max(1, cap), 5))
        k = _I64()
        _check(lib().vfps_moment_series(self._h, _dptr(out), int(cap), ctypes.byref(k)), "vfps_moment_series")
        return out[:k.value].copy()

    def spectrogram(self, length: int, hop: int, count: int) -> np.ndarray:
        """(count, length/2 + 1) power spectra of CSR-power windows, on the device."""
        out = np.empty((count, length // 2 + 1))
        _check(lib().vfps_spectrogram(self._h, int(length), int(hop), int(count), _dptr(out)), "vfps_spectrogram")
        return out

    def _series(self, fn, cap):
        # one value per step since the series was last drained: a buffer of
        # that size (a huge one costs more in first-touch faults than the copy)
        taken = self._taken.get(fn.__name__, 0)
        cap = min(cap, max(1, self.steps_done() - taken))
        out = np.empty(max(cap, 1))
        k = _I64()
        _check(fn(self._h, _dptr(out), cap, ctypes.byref(k)), fn.__name__)
        self._taken[fn.__name__] = taken + k.value
        return out[:k.value].copy()

    def csr_power(self, cap: int = 1 << 22) -> np.ndarray:
        return self._series(lib().vfps_csr_power, cap)

    def charge_series(self, cap: int = 1 << 22) -> np.ndarray:
        return self._series(lib().vfps_charge_series, cap)

    def get_state(self) -> np.ndarray:
        n = self.params.n
        out = np.empty((n, n))
        _check(lib().vfps_get_state(self._h, _dptr(out)), "vfps_get_state")
        return out

    def set_state(self, psi):
        n = self.params.n
        _check(lib().vfps_set_state(self._h, _dptr(_f64(psi, (n, n)))), "vfps_set_state")

    def save_checkpoint(self) -> bytes:
        """The device state between steps, as raw bytes (bitwise resume)."""
        k = _I64()
        _check(lib().vfps_checkpoint_bytes(self._h, ctypes.byref(k)), "vfps_checkpoint_bytes")
        buf = ctypes.create_string_buffer(k.value)
        _check(lib().vfps_save_checkpoint(self._h, buf, k.value), "vfps_save_checkpoint")
        return buf.raw

    def load_checkpoint(self, data: bytes):
        """Resume from save_checkpoint's bytes (same parameters and impedance)."""
        buf = ctypes.create_string_buffer(bytes(data), len(data))
        _check(lib().vfps_load_checkpoint(self._h, buf, len(data)), "vfps_load_checkpoint")
        self._taken = {}

    def haissinski(self, tol: float = 1e-13, max_iter: int = 20000) -> int:
        """Replace the state by the Haissinski equilibrium rho_H(q) g(p) of the
        current impedance and S_csr, solved on the device; returns iterations."""
        it = _I32()
        _check(lib().vfps_haissinski(self._h, float(tol), int(max_iter), ctypes.byref(it)), "vfps_haissinski")
        return it.value

    def steps_done(self) -> int:
        k = _I64()
        _check(lib().vfps_steps_done(self._h, ctypes.byref(k)), "vfps_steps_done")
        return k.value

    @property
    def persistent(self) -> bool:
        """True when step() runs this simulation in persistent launches."""
        on = _I32()
        _check(lib().vfps_step_mode(self._h, ctypes.byref(on)), "vfps_step_mode")
        return bool(on.value)

    def close(self):
        if getattr(self, "_h", None):
            lib().vfps_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Slots that advance together (vfps_batch_*)."""

    def __init__(self, max_slots: int, budget_bytes: int = 0, stream=None):
        b = _VP()
        _check(lib().vfps_batch_create(max_slots, budget_bytes, _stream_ptr(stream), ctypes.byref(b)),
               "vfps_batch_create")
        self._b = b
        self.params = {}
        self.nsteps = {}   # slot -> upper bound on the steps it has taken (its P(t) length)

    @staticmethod
    def slot_bytes(params: Params) -> int:
        return int(lib().vfps_batch_slot_bytes(ctypes.byref(params.c())))

    def add(self, params: Params, psi0=None, model: int = 0, Pi: float = 0.0, S_csr: float = 0.0,
            nsteps: int = 0, table=None) -> int:
        n = params.n
        psi = None if psi0 is None else _f64(psi0, (n, n))
        tab = None
        if table is not None:
            t = np.asarray(table, dtype=np.complex128)
            tab = np.empty(2 * t.size)
            tab[0::2], tab[1::2] = t.real, t.imag
        s = _I32()
        _check(lib().vfps_batch_add(self._b, ctypes.byref(params.c()), _dptr(psi), model, Pi, S_csr,
                                    _dptr(tab), int(nsteps), ctypes.byref(s)), "vfps_batch_add")
        self.params[s.value] = params
        self.nsteps[s.value] = (int(nsteps), 0)
        return s.value

    def add_many(self, params: Params, psi0, model: int, Pi, S_csr, nsteps: int = 0) -> list[int]:
        """vfps_batch_add_many: len(Pi) simulations of one parameter set; psi0 is
        None or a (count, n, n) float64 array (pinned memory copies fastest)."""
        Pi = _f64(Pi)
        S = _f64(S_csr)
        count = int(Pi.size)
        n = params.n
        ps = None if psi0 is None else _f64(psi0, (count, n, n))
        out = (_I32 * count)()
        _check(lib().vfps_batch_add_many(self._b, count, ctypes.byref(params.c()), _dptr(ps), int(model),
                                         _dptr(Pi), _dptr(S), int(nsteps), out), "vfps_batch_add_many")
        slots = [out[i] for i in range(count)]
        for sl in slots:
            self.params[sl] = params
            self.nsteps[sl] = (int(nsteps), 0)
        return slots

    def take_many(self, slots, psi_out=None, power_cap: int = 0):
        """vfps_batch_take_many: states of `slots` into psi_out (a C-contiguous
        (len(slots), n, n) float64 array, e.g. pinned) and, with power_cap > 0,
        their CSR-power series (list of arrays)."""
        count = len(slots)
        sl = (_I32 * count)(*[int(x) for x in slots])
        if psi_out is not None:
            n = self.params[slots[0]].n
            if psi_out.shape != (count, n, n) or psi_out.dtype != np.float64 or not psi_out.flags.c_contiguous:
                raise ValueError(f"psi_out must be a C-contiguous float64 array of shape {(count, n, n)}")
        pw = np.empty((count, max(1, power_cap))) if power_cap > 0 else None
        npw = (_I64 * count)()
        _check(lib().vfps_batch_take_many(self._b, count, sl, _dptr(psi_out), _dptr(pw), int(power_cap), npw),
               "vfps_batch_take_many")
        return [pw[i, :npw[i]].copy() for i in range(count)] if pw is not None else None

    def try_add(self, *a, **kw):
        """add(), but returns None instead of raising when the batch is full (EBUSY)."""
        try:
            return self.add(*a, **kw)
        except VfpsError as e:
            if e.code == EBUSY:
                return None
            raise

    def run(self, chunk_steps: int):
        # every unfinished slot advances by up to chunk_steps, and never past
        # its target: the bound holds whether or not the call succeeds
        for k, (target, done) in self.nsteps.items():
            self.nsteps[k] = (target, min(target, done + int(chunk_steps)))
        _check(lib().vfps_batch_run(self._b, int(chunk_steps)), "vfps_batch_run")

    def idle(self) -> bool:
        """True once every queued step and set-up has finished (never blocks)."""
        k = _I32()
        _check(lib().vfps_batch_idle(self._b, ctypes.byref(k)), "vfps_batch_idle")
        return bool(k.value)

    def poll(self) -> list[int]:
        cap = max(1, len(self.params))
        out = (_I32 * cap)()
        k = _I32()
        _check(lib().vfps_batch_poll(self._b, out, cap, ctypes.byref(k)), "vfps_batch_poll")
        return [out[i] for i in range(k.value)]

    def shapes(self) -> list:
        """Launch groups: dicts with n, instances, W, tiles per strip, final, paired."""
        cap = 64
        out = (_I32 * (6 * cap))()
        k = _I32()
        _check(lib().vfps_batch_shapes(self._b, out, cap, ctypes.byref(k)), "vfps_batch_shapes")
        return [dict(n=out[6 * i], instances=out[6 * i + 1], W=out[6 * i + 2], tps=out[6 * i + 3],
                     final=bool(out[6 * i + 4]), paired=bool(out[6 * i + 5])) for i in range(k.value)]

    def pairing(self, on: bool = True):
        """Run FP32 simulations of equal geometry two at a time (off by default)."""
        _check(lib().vfps_batch_pairing(self._b, 1 if on else 0), "vfps_batch_pairing")

    def pin_shape(self, W: int = 0, tps: int = 0):
        """Fix the CTA width and strip length of the FP32 groups (tps=-1: balanced grid; 0, 0 releases)."""
        _check(lib().vfps_batch_pin_shape(self._b, int(W), int(tps)), "vfps_batch_pin_shape")

    def autotune(self, on: bool = True):
        """Enable or disable the per-configuration autotuner (on by default)."""
        _check(lib().vfps_batch_autotune(self._b, 1 if on else 0), "vfps_batch_autotune")

    def power_spectrum(self, slot: int, length: int) -> np.ndarray:
        """|DFT|^2 of the slot's last `length` CSR-power values, on the device."""
        out = np.empty(length // 2 + 1)
        _check(lib().vfps_batch_power_spectrum(self._b, int(slot), int(length), _dptr(out)),
               "vfps_batch_power_spectrum")
        return out

    def moments(self, slot: int) -> np.ndarray:
        """(<q>, sigma_q, <p>, sigma_p) of a slot's current state, on the device."""
        out = np.empty(4)
        _check(lib().vfps_batch_moments(self._b, int(slot), _dptr(out)), "vfps_batch_moments")
        return out

    def record_moments(self, slot: int, every: int):
        """vfps_batch_record_moments."""
        _check(lib().vfps_batch_record_moments(self._b, int(slot), int(every)), "vfps_batch_record_moments")

    def moment_series(self, slot: int, cap: int = 1 << 20) -> np.ndarray:
        """The slot's moment records so far: rows (t, <q>, sigma_q, <p>, sigma_p)."""
        out = np.empty((max(1, cap), 5))
        k = _I64()
        _check(lib().vfps_batch_moment_series(self._b, int(slot), _dptr(out), int(cap), ctypes.byref(k)),
               "vfps_batch_moment_series")
        return out[:k.value].copy()

    def spectrogram(self, slots, length: int, hop: int, count: int) -> np.ndarray:
        """(len(slots), count, length/2 + 1) windowed CSR-power spectra, one launch."""
        sl = (_I32 * len(slots))(*[int(x) for x in slots])
        out = np.empty((len(slots), count, length // 2 + 1))
        _check(lib().vfps_batch_spectrogram(self._b, sl, len(slots), int(length), int(hop), int(count), _dptr(out)),
               "vfps_batch_spectrogram")
        return out

    def take(self, slot: int, psi=True, rho=True, power_cap: int = 1 << 22, psi_out=None):
        """vfps_batch_take.  psi_out: an (n, n) C-contiguous float64 array to
        write the state into (e.g. a row of one preallocated array for all
        slots) instead of a new one."""
        n = self.params[slot].n
        if psi_out is not None:
            if psi_out.shape != (n, n) or psi_out.dtype != np.float64 or not psi_out.flags.c_contiguous:
                raise ValueError(f"psi_out must be a C-contiguous float64 array of shape {(n, n)}")
            ps = psi_out
        else:
            ps = np.empty((n, n)) if psi else None
        rh = np.empty(n) if rho else None
        # a slot's series holds one value per step taken: a buffer of that
        # bound (a huge one costs more in first-touch faults than the copy)
        power_cap = min(power_cap, max(1, self.nsteps.get(slot, (0, power_cap))[1]))
        pw = np.empty(max(1, power_cap))
        npow, steps = _I64(), _I64()
        _check(lib().vfps_batch_take(self._b, slot, _dptr(ps), _dptr(rh), _dptr(pw), power_cap,
                                     ctypes.byref(npow), ctypes.byref(steps)), "vfps_batch_take")
        return {"psi": ps, "rho": rh, "power": pw[:npow.value].copy(), "steps": steps.value}

    def haissinski(self, slot: int, tol: float = 1e-13, max_iter: int = 20000) -> int:
        """vfps_haissinski for one slot; returns iterations."""
        it = _I32()
        _check(lib().vfps_batch_haissinski(self._b, int(slot), float(tol), int(max_iter), ctypes.byref(it)),
               "vfps_batch_haissinski")
        return it.value

    def remove(self, slot: int):
        _check(lib().vfps_batch_remove(self._b, slot), "vfps_batch_remove")
        self.params.pop(slot, None)
        self.nsteps.pop(slot, None)

    def usage(self):
        a, b = _I32(), _I64()
        _check(lib().vfps_batch_usage(self._b, ctypes.byref(a), ctypes.byref(b)), "vfps_batch_usage")
        return a.value, b.value

    def launches_per_step(self) -> int:
        k = _I32()
        _check(lib().vfps_batch_launches_per_step(self._b, ctypes.byref(k)), "vfps_batch_launches_per_step")
        return k.value

    def close(self):
        if getattr(self, "_b", None):
            lib().vfps_batch_destroy(self._b)
            self._b = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def step_static(params: Params, model: int, Pi: float, S_csr: float, psi_in_ptr: int, psi_out_ptr: int,
                stream=None, want_power: bool = True):
    """vfps_step_static on caller-owned device buffers (raw device pointers).
    Returns P(psi_in) when want_power (the call then synchronises)."""
    p = ctypes.c_double()
    rc = lib().vfps_step_static(ctypes.byref(params.c()), model, Pi, S_csr, ctypes.c_void_p(psi_in_ptr),
                                ctypes.c_void_p(psi_out_ptr), ctypes.byref(p) if want_power else None,
                                _stream_ptr(stream))
    if rc != OK:
        msg = lib().vfps_last_cuda_error().decode()
        raise VfpsError(rc, f"vfps_step_static [{msg}]")
    return p.value if want_power else None
