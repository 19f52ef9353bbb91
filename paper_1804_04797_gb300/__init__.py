"""GB300 (sm_103a) state-vector simulator of random lattice circuits (arXiv:1804.04797).

The simulation runs in the CUDA library built from csrc/ (C interface: include/sv.h);
``sv`` is its ctypes binding and ``inputs`` names the seeded synthetic workloads.
"""
from . import inputs  # noqa: F401
