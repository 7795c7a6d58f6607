"""Seeded synthetic inputs for the nonrigid SENSE operator.

This package produces inputs only: phantoms, displacement fields, coil
sensitivity maps and non-Cartesian trajectories.  It holds none of the
operator's arithmetic (no kernel, no FFT, no gridding), so that both the FP64
oracle and the CUDA path can be fed the same data without sharing any code of
the method itself.

The paper's in-vivo data (1.5T scanner, 8-channel cardiac coil, 3D cones
phyllotaxis trajectory, four respiratory phases; "Nonrigid Respiratory Motion
Correction" section) are not available, so every array here is synthetic with
the shapes and structure of that workload.
"""

from .workloads import (  # noqa: F401
    phantom,
    bump_displacement,
    rigid_translation,
    coil_maps,
    cones_trajectory,
    phase_sample_counts,
    workload,
    make,
    small_case,
    WORKLOADS,
    Spec,
    INTERLEAVES_PER_HEARTBEAT,
)
