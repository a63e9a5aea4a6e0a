"""Seeded synthetic inputs shared by the GPU library's tests/benchmark and the CPU oracle.

This module holds configurations (SI parameters, chemistry constants) and seeded generators of
masks, inlet profiles and initial fields. It contains none of the time step's arithmetic: the
library and the oracle each convert units, build equilibria and advance the state themselves.
"""
from .configs import SPECIES, chemistry_2step, chemistry_1step, mixture_phi  # noqa: F401
from .generate import Workload, make, names  # noqa: F401
