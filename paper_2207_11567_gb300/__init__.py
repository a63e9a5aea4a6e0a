"""GB300 (sm_103a) library for one full time step of the hybrid low-Mach lattice Boltzmann /
finite-difference combustion solver (Hosseini, Darabiha, Thevenin, Section 2).

The compute path is the CUDA library ``libhlbm.so`` behind the C ABI of ``include/hlbm.h``;
this package holds its sources (``csrc/``), the build script and a thin ctypes binding. Import
fails when the library has not been built: there is no CPU fallback.
"""
from . import _lib  # noqa: F401  (loads libhlbm.so or raises)
from .solver import Solver, from_workload  # noqa: F401
from .adjoint import AdjointProblem, HybridStepFn  # noqa: F401
from .flame1d import FlameSolution, free_flame  # noqa: F401
