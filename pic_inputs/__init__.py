"""Seeded synthetic inputs shared by the tests, the oracle runs and the benchmark.

This package holds no arithmetic of the PIC method: it only draws particle positions
and velocities for the cold two-stream problem (and states the per-workload
constants).  Both the CUDA path and the oracle receive the same arrays from here.
"""

from .twostream import (  # noqa: F401
    WORKLOADS,
    EnsembleRun,
    Workload,
    ensemble_particles,
    ensemble_runs,
    lattice_twostream,
    random_twostream,
    splitmix64_uniform,
    workload_particles,
)
