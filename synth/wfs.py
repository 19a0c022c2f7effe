"""Shack-Hartmann frame rendering, calibration maps and control matrices.

Frames follow the generator recipe used throughout this repository:

* the true slope of a subaperture is the mean phase gradient across it
  (right-minus-left and bottom-minus-top edge means of the sampled phase),
  multiplied by a plate scale fixed so that the slopes of frame 0 have the
  configured RMS (0.3 px by default);
* the spot is a pixel-integrated Gaussian (differences of ``erf``) of width
  ``spot_sigma_px`` and total flux ``flux_e`` photo-electrons, centred at
  ``(npx-1)/2 + slope`` in both axes -- flux falling outside the box is lost;
* each pixel gets Poisson photon noise on its expected electrons, then
  Gaussian read noise, then the detector response
  ``raw = clamp(round(flat * e + dark), 0, 65535)`` with gain 1 e-/ADU.

Everything is seeded; frames produced by one call depend on (seed, start
index, count) and on the device the noise is drawn on.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from .configs import WorkloadConfig
from .turbulence import FrozenFlow

SAMPLES_PER_SUBAP = 8


class ShackHartmann:
    """Frozen-flow turbulence seen through the configured Shack-Hartmann WFS."""

    def __init__(self, cfg: WorkloadConfig, device="cpu", screen_seeds=None):
        self.cfg = cfg
        self.device = torch.device(device)
        sa = torch.from_numpy(cfg.subaps.astype(np.int64))
        self.sub_r = sa[:, 0].to(self.device)
        self.sub_c = sa[:, 1].to(self.device)
        S = SAMPLES_PER_SUBAP
        npts = S * cfg.nsub + 1
        pitch = cfg.diameter_m / (cfg.nsub * S)
        self.flow = FrozenFlow(npts, pitch, cfg.r0_m, cfg.L0_m, cfg.wind_mps, cfg.wind_dir_deg,
                               screen_seeds if screen_seeds is not None else cfg.screen_seeds,
                               device=self.device)
        g0 = self._gradients(self.flow.phase(torch.zeros(1)))
        self.plate_scale = float(cfg.slope_rms_px / torch.sqrt(torch.mean(g0.double() ** 2)))

    # -- turbulence -> slopes -------------------------------------------------
    def _gradients(self, phase: torch.Tensor) -> torch.Tensor:
        S = SAMPLES_PER_SUBAP
        ar = torch.arange(S + 1, device=self.device)
        rows = S * self.sub_r[:, None] + ar[None, :]          # nv x (S+1)
        cols = S * self.sub_c[:, None] + ar[None, :]
        left = phase[:, rows, (S * self.sub_c)[:, None]]
        right = phase[:, rows, (S * (self.sub_c + 1))[:, None]]
        top = phase[:, (S * self.sub_r)[:, None], cols]
        bottom = phase[:, (S * (self.sub_r + 1))[:, None], cols]
        gx = right.mean(-1) - left.mean(-1)
        gy = bottom.mean(-1) - top.mean(-1)
        return torch.stack([gx, gy], dim=-1)                   # B x nv x 2

    def true_slopes(self, frame_indices, wfs: int = 0) -> torch.Tensor:
        """Noise-free slopes in pixels (B x nv x 2, (x, y)) at the given frame indices."""
        idx = torch.as_tensor(frame_indices, dtype=torch.float64).reshape(-1)
        t = idx / self.cfg.frame_rate_hz + 1000.0 * wfs
        return self._gradients(self.flow.phase(t)) * self.plate_scale

    # -- slopes -> detector counts --------------------------------------------
    def render(self, slopes_px: torch.Tensor, dark: torch.Tensor, flat: torch.Tensor,
               gen: torch.Generator) -> torch.Tensor:
        """Render uint16 frames (B x H x W) for true slopes ``slopes_px`` (B x nv x 2)."""
        cfg = self.cfg
        n = cfg.npx
        B = slopes_px.shape[0]
        dev = self.device
        x = torch.arange(n, device=dev, dtype=torch.float32)
        mu = (n - 1) / 2.0 + slopes_px.to(device=dev, dtype=torch.float32)
        k = 1.0 / (cfg.spot_sigma_px * math.sqrt(2.0))

        def box_integral(m):     # B x nv -> B x nv x n
            hi = (x + 0.5 - m[..., None]) * k
            lo = (x - 0.5 - m[..., None]) * k
            return 0.5 * (torch.erf(hi) - torch.erf(lo))

        ix = box_integral(mu[..., 0])
        iy = box_integral(mu[..., 1])
        expect = cfg.flux_e * iy[..., :, None] * ix[..., None, :]    # B x nv x n(y) x n(x)
        photons = torch.poisson(expect, generator=gen)
        grid = torch.zeros((B, cfg.nsub, cfg.nsub, n, n), device=dev, dtype=torch.float32)
        grid[:, self.sub_r, self.sub_c] = photons
        img = grid.permute(0, 1, 3, 2, 4).reshape(B, cfg.frame_side, cfg.frame_side)
        img = img + cfg.read_noise_e * torch.randn(img.shape, generator=gen, device=dev)
        raw = torch.clamp(torch.round(flat * img + dark), 0, 65535)
        return raw.to(torch.int32).to(torch.uint16)


def calibration_maps(cfg: WorkloadConfig, device="cpu", seed: int | None = None):
    """Dark ~ U(dark_lo, dark_hi) ADU and flat ~ N(1, flat_sigma) per pixel, float32,
    shaped (n_wfs, H, W)."""
    gen = torch.Generator().manual_seed(cfg.calib_seed if seed is None else seed)
    shape = (cfg.n_wfs, cfg.frame_side, cfg.frame_side)
    dark = cfg.dark_lo + (cfg.dark_hi - cfg.dark_lo) * torch.rand(shape, generator=gen)
    flat = 1.0 + cfg.flat_sigma * torch.randn(shape, generator=gen)
    return dark.to(device=device, dtype=torch.float32), flat.to(device=device, dtype=torch.float32)


def control_matrix(cfg: WorkloadConfig, device="cpu", seed: int | None = None,
                   nact: int | None = None, nslopes: int | None = None) -> torch.Tensor:
    """Random control matrix, nact x nslopes float32 with entries N(0, 1/nslopes)."""
    gen = torch.Generator().manual_seed(cfg.matrix_seed if seed is None else seed)
    na = cfg.nact if nact is None else nact
    ns = cfg.nslopes if nslopes is None else nslopes
    m = torch.randn((na, ns), generator=gen, dtype=torch.float32) / math.sqrt(ns)
    return m.to(device)


def make_frames(cfg: WorkloadConfig, start: int, count: int, device="cpu",
                wfs_model: ShackHartmann | None = None, maps=None, noise_seed: int | None = None):
    """Frames ``start .. start+count-1`` -> (uint16 frames (count, n_wfs, H, W),
    true slopes (count, n_wfs, nv, 2))."""
    sh = wfs_model if wfs_model is not None else ShackHartmann(cfg, device=device)
    dark, flat = maps if maps is not None else calibration_maps(cfg, device=sh.device)
    gen = torch.Generator(device=sh.device)
    seed = cfg.noise_seed if noise_seed is None else noise_seed
    gen.manual_seed(int(seed) * 1_000_003 + int(start))
    idx = torch.arange(start, start + count)
    frames, slopes = [], []
    for w in range(cfg.n_wfs):
        s = sh.true_slopes(idx, wfs=w)
        frames.append(sh.render(s, dark[w], flat[w], gen))
        slopes.append(s)
    return torch.stack(frames, dim=1), torch.stack(slopes, dim=1)
