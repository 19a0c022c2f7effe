"""Seeded synthetic inputs for the SCAO real-time pipeline.

This package makes the *inputs* that both the CUDA path and the CPU oracle
consume: telescope/DM geometry, frozen-flow von Karman phase screens, rendered
Shack-Hartmann frames with photon and read noise, dark/flat calibration maps
and random control matrices.  It holds none of the pipeline's arithmetic
(calibration, centroiding, reconstruction, integration); those live in the
oracle and in the CUDA kernels, independently.

The paper runs its pipeline on "fake image data" (Sec. 2.1); these generators
stand in for that data and for the real camera of Sec. 3.3.
"""
from .configs import WorkloadConfig, CONFIGS, tiny_scao, elt_scao, elt_scao_6wfs
from .geometry import valid_subaps, valid_actuators
from .turbulence import PhaseScreenLayer, FrozenFlow
from .wfs import ShackHartmann, calibration_maps, control_matrix, make_frames

__all__ = [
    "WorkloadConfig", "CONFIGS", "tiny_scao", "elt_scao", "elt_scao_6wfs",
    "valid_subaps", "valid_actuators",
    "PhaseScreenLayer", "FrozenFlow",
    "ShackHartmann", "calibration_maps", "control_matrix", "make_frames",
]
