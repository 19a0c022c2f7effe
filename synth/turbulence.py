"""Seeded frozen-flow von Karman turbulence.

Each layer is one periodic FFT phase screen with the von Karman spectrum
``PSD(f) = 0.023 r0^(-5/3) (f^2 + 1/L0^2)^(-11/6)``, translated rigidly by its
wind vector (Taylor frozen flow) and sampled on the pupil grid with bilinear
interpolation.  Screens are drawn on the CPU from a seeded generator, so a
given seed gives the same screen whichever device later samples it.
"""
from __future__ import annotations

import math
from typing import Sequence

import torch


class PhaseScreenLayer:
    """One periodic n x n phase screen (radians at 500 nm) with sample pitch ``pitch_m``."""

    def __init__(self, n: int, pitch_m: float, r0_m: float, L0_m: float, seed: int,
                 device="cpu"):
        gen = torch.Generator().manual_seed(int(seed))
        f = torch.fft.fftfreq(n, d=pitch_m, dtype=torch.float64)
        f2 = f[None, :] ** 2 + f[:, None] ** 2
        psd = 0.023 * r0_m ** (-5.0 / 3.0) * (f2 + 1.0 / L0_m ** 2) ** (-11.0 / 6.0)
        psd[0, 0] = 0.0
        df = 1.0 / (n * pitch_m)
        re = torch.randn((n, n), generator=gen, dtype=torch.float64)
        im = torch.randn((n, n), generator=gen, dtype=torch.float64)
        coef = torch.complex(re, im) * torch.sqrt(psd) * df
        screen = torch.fft.ifft2(coef).real * (n * n)
        self.n = n
        self.pitch_m = pitch_m
        self.screen = screen.to(device=device, dtype=torch.float32)

    def sample(self, shift_px: torch.Tensor, npts: int) -> torch.Tensor:
        """Sample an npts x npts window displaced by ``shift_px`` (B x 2, (x, y) in
        screen pixels) with periodic wrap and bilinear interpolation -> B x npts x npts."""
        dev = self.screen.device
        shift = shift_px.to(device=dev, dtype=torch.float64)
        base = torch.floor(shift)
        frac = (shift - base).to(torch.float32)
        ix0 = base[:, 0].to(torch.int64)
        iy0 = base[:, 1].to(torch.int64)
        ar = torch.arange(npts + 1, device=dev, dtype=torch.int64)
        cols = (ix0[:, None] + ar[None, :]) % self.n        # B x (npts+1)
        rows = (iy0[:, None] + ar[None, :]) % self.n
        win = self.screen[rows[:, :, None], cols[:, None, :]]  # B x (npts+1) x (npts+1)
        fx = frac[:, 0].view(-1, 1, 1)
        fy = frac[:, 1].view(-1, 1, 1)
        a = win[:, :-1, :-1]
        b = win[:, :-1, 1:]
        c = win[:, 1:, :-1]
        d = win[:, 1:, 1:]
        return (1 - fy) * ((1 - fx) * a + fx * b) + fy * ((1 - fx) * c + fx * d)


class FrozenFlow:
    """Sum of translating layers, sampled on a (npts x npts) pupil grid of pitch ``pitch_m``.

    Layers share the turbulence strength equally (Cn^2 fraction 1/L each), so
    each layer's Fried parameter is ``r0 * (1/L)^(-3/5)``.
    """

    def __init__(self, npts: int, pitch_m: float, r0_m: float, L0_m: float,
                 wind_mps: Sequence[float], wind_dir_deg: Sequence[float],
                 seeds: Sequence[int], device="cpu", screen_n: int | None = None):
        nl = len(wind_mps)
        if not (len(wind_dir_deg) == nl == len(seeds)):
            raise ValueError("wind speeds, directions and seeds must have one entry per layer")
        if screen_n is None:
            screen_n = 256
            while screen_n < 2 * npts:
                screen_n *= 2
        r0_layer = r0_m * (1.0 / nl) ** (-3.0 / 5.0)
        self.npts = npts
        self.pitch_m = pitch_m
        self.layers = [PhaseScreenLayer(screen_n, pitch_m, r0_layer, L0_m, s, device)
                       for s in seeds]
        self.vel_px = torch.tensor(
            [[v * math.cos(math.radians(t)) / pitch_m, v * math.sin(math.radians(t)) / pitch_m]
             for v, t in zip(wind_mps, wind_dir_deg)], dtype=torch.float64)

    def phase(self, times_s: torch.Tensor) -> torch.Tensor:
        """Pupil phase at the given times -> B x npts x npts (float32)."""
        t = torch.as_tensor(times_s, dtype=torch.float64).reshape(-1)
        out = None
        for layer, v in zip(self.layers, self.vel_px):
            ph = layer.sample(t[:, None] * v[None, :], self.npts)
            out = ph if out is None else out + ph
        return out
