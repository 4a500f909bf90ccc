"""B300-native (sm_103a) per-step phase-space update of a Vlasov-Fokker-Planck solver.

Layout:
  csrc/vfps_kernels.cuh  fused step kernel (rotation, kick, Fokker-Planck,
                         projection epilogue) and the last-CTA FFT finaliser
  csrc/vfps.cu           runtime and C ABI (include/vfps.h)
  csrc/impedance_host.cpp  FP64 host tables of the CSR impedances
  build.py               nvcc build of libvfps.so (in-tree)
  vfps.py                ctypes binding (marshalling only)
  workloads.py           seeded synthetic inputs
  serve.py               continuous-batching request loop over vfps_batch_*
  analysis.py            host statistics of the CSR-power series

Importing the package loads nothing; ``from paper_1611_05293_b300 import vfps``
loads the CUDA library and raises if it is missing.
"""
__all__ = ["vfps", "workloads", "build"]
