"""GB300-native (sm_103a) phase-field lattice Boltzmann step.

Implements the coupled per-time-step lattice update of Zhang, Liang & Guo,
"On the formulations of interfacial force in the phase-field-based lattice
Boltzmann method" (arXiv 2012.14729): moments of h_i and f_i, central-scheme
derivatives of phi, the interfacial force in any of the eight formulations,
and the collision and streaming of both D2Q9 populations, fused in one CUDA
kernel behind the C ABI of include/pflbm.h.

``pflbm`` is the ctypes binding (C names) plus a ``Domain`` convenience
class; ``workloads`` builds seeded initial conditions; ``build`` compiles the
library with nvcc.
"""
from . import build  # noqa: F401
