"""Workload descriptions for the synthetic SCAO inputs.

Two sizes matter: a tiny 8x8-subaperture system that the FP64 oracle runs in
milliseconds, and the ELT-scale single-conjugate system (74x74 subapertures of
10x10 pixels, 39 m pupil, 28 % central obscuration, 75x75 DM) whose shape
follows the paper's ELT SCAO experiment (Sec. 3.1: 80x80 subapertures,
0.25 D obscuration, 10x10 pixels, 81x81 DM).
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace
from typing import Tuple

from .geometry import valid_subaps, valid_actuators


@dataclass(frozen=True)
class WorkloadConfig:
    name: str
    nsub: int                 # subapertures across the pupil (square grid)
    npx: int                  # pixels per subaperture side
    obs: float                # central obscuration, fraction of the diameter
    dm_side: int              # actuators across the DM (square grid)
    diameter_m: float         # telescope diameter
    r0_m: float               # Fried parameter at 500 nm
    L0_m: float               # outer scale
    wind_mps: Tuple[float, ...]        # one entry per frozen-flow layer
    wind_dir_deg: Tuple[float, ...]
    screen_seeds: Tuple[int, ...]
    noise_seed: int
    matrix_seed: int
    calib_seed: int
    n_frames: int
    frame_rate_hz: float = 1000.0
    spot_sigma_px: float = 1.2
    flux_e: float = 1000.0    # photo-electrons per subaperture
    read_noise_e: float = 1.0
    dark_lo: float = 90.0
    dark_hi: float = 110.0
    flat_sigma: float = 0.02
    slope_rms_px: float = 0.3  # plate scale chosen so slopes have this RMS
    gain: float = 0.4
    leak: float = 0.99
    n_wfs: int = 1            # WFS stacked into one control matrix (stress sizing)

    @property
    def frame_side(self) -> int:
        return self.nsub * self.npx

    @property
    def subaps(self):
        return valid_subaps(self.nsub, self.obs)

    @property
    def n_valid(self) -> int:
        return int(self.subaps.shape[0])

    @property
    def nslopes(self) -> int:
        return 2 * self.n_valid * self.n_wfs

    @property
    def nact(self) -> int:
        return int(valid_actuators(self.dm_side).shape[0])

    def with_(self, **kw) -> "WorkloadConfig":
        return replace(self, **kw)


def tiny_scao() -> WorkloadConfig:
    """8x8 subaps of 8x8 px, unobstructed circular pupil (52 valid), 9x9 DM (69 valid)."""
    return WorkloadConfig(
        name="tiny_scao_8x8", nsub=8, npx=8, obs=0.0, dm_side=9, diameter_m=4.0,
        r0_m=0.15, L0_m=25.0, wind_mps=(10.0,), wind_dir_deg=(0.0,),
        screen_seeds=(0,), noise_seed=0, matrix_seed=0, calib_seed=0, n_frames=1000)


def elt_scao() -> WorkloadConfig:
    """74x74 subaps of 10x10 px on a 39 m pupil, 28 % obscuration (3972 valid), 75x75 DM (4421 valid)."""
    return WorkloadConfig(
        name="elt_scao_74x74", nsub=74, npx=10, obs=0.28, dm_side=75, diameter_m=39.0,
        r0_m=0.157, L0_m=25.0, wind_mps=(10.0, 15.0, 20.0), wind_dir_deg=(0.0, 120.0, 240.0),
        screen_seeds=(1, 2, 3), noise_seed=100, matrix_seed=7, calib_seed=11, n_frames=10000)


def elt_scao_6wfs() -> WorkloadConfig:
    """Stress sizing: six ELT WFS stacked into one 4421 x 47664 control matrix."""
    return replace(elt_scao(), name="elt_scao_6wfs", n_wfs=6)


CONFIGS = {
    "tiny": tiny_scao,
    "elt": elt_scao,
    "elt6": elt_scao_6wfs,
}
