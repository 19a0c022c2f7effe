"""Deformable mirror in Fried geometry, its interaction with the Shack-Hartmann WFS,
and a regularised least-squares reconstructor.

These make the inputs of a physical closed loop (the control matrix, and the
mirror's effect on the wavefront the WFS sees); the pipeline's own arithmetic
(calibration, centroiding, reconstruction, integration) stays in the oracle and
in the CUDA kernels.

Geometry: the actuators sit on the corners of the subaperture grid, a
``(nsub+1) x (nsub+1)`` lattice (75 x 75 for 74 x 74 subapertures); the valid
ones are those of :func:`synth.valid_actuators`.  The mirror surface is the
bilinear interpolation of the commands (zero at invalid actuators) on that
lattice, in the phase units of the turbulence screens: a command ``a`` at an
actuator raises the phase there by ``a``.

The WFS slope of a subaperture is the plate scale times the difference of the
mean phase along its right and left edges (x) and its bottom and top edges (y)
(:class:`synth.ShackHartmann`).  On a bilinear surface the mean along an edge
is the mean of the edge's two corner values, so a subaperture with corner
commands ``a00`` (top left), ``a01`` (top right), ``a10`` (bottom left) and
``a11`` (bottom right) sees

    sx = plate * ((a01 + a11) - (a00 + a10)) / 2
    sy = plate * ((a10 + a11) - (a00 + a01)) / 2

which is the interaction matrix ``D`` (slopes x block then y block, one row per
slope, one column per valid actuator).  Piston and the checkerboard ("waffle")
pattern give no slopes in this geometry; the reconstructor
``R = (D^T D + alpha I)^-1 D^T`` (``alpha`` a small fraction of the mean
diagonal of ``D^T D``) keeps them at zero.
"""
from __future__ import annotations

import numpy as np
import torch
import torch.nn.functional as F

from .configs import WorkloadConfig
from .geometry import valid_actuators


class FriedDM:
    """Commands -> mirror phase on the WFS sampling grid, and -> WFS slopes."""

    def __init__(self, cfg: WorkloadConfig, plate_scale: float, samples_per_subap: int):
        if cfg.dm_side != cfg.nsub + 1:
            raise ValueError("Fried geometry needs dm_side == nsub + 1")
        self.cfg = cfg
        self.side = cfg.dm_side
        self.plate = float(plate_scale)
        self.S = int(samples_per_subap)
        self.act = valid_actuators(cfg.dm_side).astype(np.int64)     # nact x (row, col)
        self.nact = int(self.act.shape[0])
        self.index = -np.ones((self.side, self.side), np.int64)
        self.index[self.act[:, 0], self.act[:, 1]] = np.arange(self.nact)

    # -- commands -> mirror phase -----------------------------------------------
    def command_map(self, a: torch.Tensor) -> torch.Tensor:
        """Commands (B x nact) -> lattice values (B x side x side), zero off the DM."""
        a = torch.as_tensor(a)
        a2 = a.reshape(-1, self.nact)
        m = torch.zeros((a2.shape[0], self.side, self.side), dtype=a2.dtype, device=a2.device)
        r = torch.as_tensor(self.act[:, 0], device=a2.device)
        c = torch.as_tensor(self.act[:, 1], device=a2.device)
        m[:, r, c] = a2
        return m

    def phase(self, a: torch.Tensor) -> torch.Tensor:
        """Mirror phase on the WFS grid (B x npts x npts, npts = S nsub + 1): bilinear
        interpolation of the lattice, the lattice points landing on every S-th sample."""
        m = self.command_map(a)
        npts = self.S * self.cfg.nsub + 1
        return F.interpolate(m[:, None], size=(npts, npts), mode="bilinear",
                             align_corners=True)[:, 0]

    # -- interaction matrix ---------------------------------------------------------
    def interaction(self, subaps: np.ndarray | None = None, n_wfs: int | None = None) -> np.ndarray:
        """D (nslopes x nact, float64) in the pipeline's slope order: for each WFS the
        x slopes of all valid subapertures, then their y slopes."""
        sa = self.cfg.subaps if subaps is None else np.asarray(subaps)
        nw = self.cfg.n_wfs if n_wfs is None else n_wfs
        nv = sa.shape[0]
        D = np.zeros((2 * nv * nw, self.nact))
        h = 0.5 * self.plate
        for i, (r, c) in enumerate(sa):
            a00, a01 = self.index[r, c], self.index[r, c + 1]
            a10, a11 = self.index[r + 1, c], self.index[r + 1, c + 1]
            for w in range(nw):
                bx = 2 * nv * w + i
                by = bx + nv
                for k, sx, sy in ((a00, -h, -h), (a01, h, -h), (a10, -h, h), (a11, h, h)):
                    if k >= 0:
                        D[bx, k] += sx
                        D[by, k] += sy
        return D


def reconstructor(D: np.ndarray, alpha_rel: float = 1e-3) -> np.ndarray:
    """Regularised least-squares reconstructor R = (D^T D + alpha I)^-1 D^T (nact x
    nslopes, float64), alpha = alpha_rel times the mean diagonal of D^T D."""
    DtD = D.T @ D
    alpha = alpha_rel * float(np.trace(DtD)) / DtD.shape[0]
    return np.linalg.solve(DtD + alpha * np.eye(DtD.shape[0]), D.T)
