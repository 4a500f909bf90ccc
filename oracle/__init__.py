"""FP64 CPU oracle for the per-step VFP phase-space update (test infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
legs may import, call, link or execute anything in this package.  The
product library (``paper_1611_05293_b300``) never does, and this package
imports nothing from the product.  It shares no code with the CUDA path.

Modules:
  vfps_oracle.c  plain FP64 C solver: interpolation, rotation, projection,
                 wake (direct DFT), kick, Fokker-Planck step, renormalisation
  oracle.py      ctypes face of the C solver and its gcc build
  impedance.py   normalised free-space and parallel-plates CSR impedances
  brute.py       dense-matrix NumPy restatement for tiny grids
  haissinski.py  Haissinski equilibrium profile (fixed-point iteration)

Parity status: every function has a pin in tests/test_oracle_*.py.
"""
