"""Seeded synthetic inputs (geometry + workload recipes) shared by the oracle tests, the GPU tests and the bench.

Holds no arithmetic of the refinement method itself.
"""
from .configs import NAMES, Workload, batched_workloads, small_workload, workload  # noqa: F401
