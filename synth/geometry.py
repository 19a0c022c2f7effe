"""Pupil and deformable-mirror geometry.

The paper prints only counts (Sec. 3.1: an 80x80 grid with a 0.25 D central
obscuration has 4708 active subapertures; an 81x81 circular DM has 5170
actuators).  The rules here are the simplest ones that reproduce them:

* a subaperture is valid when its centre lies inside the annulus
  ``obs * n/2 <= r <= n/2`` (radii in subaperture pitches from the grid
  centre) -- this gives exactly 4708 for the paper's case;
* an actuator on an m x m grid is valid when its distance from the grid
  centre is at most ``(m-1)/2 + 0.5`` pitches (a circle, no obscuration) --
  this gives 5169 for m = 81, one short of the paper's 5170, whose exact rule
  is not given.
"""
from __future__ import annotations

import numpy as np


def valid_subaps(nsub: int, obs: float) -> np.ndarray:
    """Valid subapertures as an int32 array of (row, col), in row-major grid order."""
    c = (np.arange(nsub) + 0.5) - nsub / 2.0
    yy, xx = np.meshgrid(c, c, indexing="ij")
    r = np.hypot(xx, yy)
    ok = (r <= nsub / 2.0) & (r >= obs * nsub / 2.0)
    rows, cols = np.nonzero(ok)          # row-major order
    return np.stack([rows, cols], axis=1).astype(np.int32)


def valid_actuators(side: int) -> np.ndarray:
    """Valid DM actuators as an int32 array of (row, col), in row-major grid order."""
    c = np.arange(side) - (side - 1) / 2.0
    yy, xx = np.meshgrid(c, c, indexing="ij")
    ok = np.hypot(xx, yy) <= (side - 1) / 2.0 + 0.5
    rows, cols = np.nonzero(ok)
    return np.stack([rows, cols], axis=1).astype(np.int32)


def subap_index_grid(nsub: int, subaps: np.ndarray) -> np.ndarray:
    """nsub x nsub int32 grid holding each valid subap's index, -1 elsewhere."""
    g = np.full((nsub, nsub), -1, dtype=np.int32)
    g[subaps[:, 0], subaps[:, 1]] = np.arange(subaps.shape[0], dtype=np.int32)
    return g
