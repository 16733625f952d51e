"""Seeded synthetic 4D-STEM electron-event data.

This package only makes inputs: workload recipes (``workloads``) and a
forward-model event generator (``generate``).  It holds none of the
reconstruction arithmetic (no COM, no binning, no scan transform, no SSB), so
both the FP64 oracle and the CUDA path can consume its output without sharing
any of the method's code.
"""

from .workloads import Workload, workload, geometry, batching_datasets, candidate_aberrations  # noqa: F401
from .generate import generate, EventData  # noqa: F401
