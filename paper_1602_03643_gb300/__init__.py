"""GB300-native P1-P1 IPCS (fractional-step) Navier-Stokes step.

The compute path is liboasis.so (hand-written sm_103a CUDA kernels behind the
C ABI of include/oasis.h); ``capi`` is its ctypes binding and ``driver`` a
small convenience wrapper.  Build with ``python -m paper_1602_03643_gb300.build``.
"""
from . import capi  # noqa: F401
