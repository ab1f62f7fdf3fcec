"""Seeded synthetic inputs for the ADDFE/FDM forward/adjoint/gradient path.

This package only *draws and lays out* inputs: grid geometry constants, the
layered-skin-with-inclusion coefficient models, detector positions and
incidence directions.  It holds none of the method's arithmetic (no operator,
no time stepping, no source pulse, no functional), so that the CPU oracle and
the CUDA path can both be fed from it without sharing any of the method.
"""
from .models import (  # noqa: F401
    SplitMix64,
    Workload,
    box_bounds,
    detector_grid,
    free_box,
    hemisphere_directions,
    layered_inclusion_model,
    shard_directions,
    workload,
    WORKLOADS,
    batched_problems,
)
