"""FP64 oracle of the per-frame pipeline (Sec. 2.1, Fig. 3 (a)-(d)) -- test infrastructure only.

Steps, in the paper's order:

(a) pixel calibration: background (dark) subtraction, flat-field, threshold;
(b) local wavefront gradient of each subaperture by centre of gravity;
    the x gradients of all subapertures come first, then the y gradients;
(c) wavefront reconstruction by a dense matrix-vector multiplication;
(d) a gain applied to the result -- generalised here to the leaky integrator
    ``a <- leak * a + g * d`` (``leak = 1`` on a zero state is the paper's plain gain).

Readings where the paper is silent (each listed in the design notes):

* flat field multiplies by ``1/flat``;
* threshold mode 0 zeroes pixels below ``thr``; mode 1 subtracts ``thr`` and
  clips at zero.  The keep/zero decision is an integer outcome of floating-point
  arithmetic, so it is taken on the FP32 value ``(raw - dark) * (1/flat)``
  evaluated with IEEE single rounding (as the device computes it); the kept
  values themselves are FP64;
* centroids are in pixels relative to the box centre ``(n-1)/2``, with no
  reference-slope subtraction; a subaperture whose flux is not positive gets
  zero slopes;
* the matrix is ``nact x nslopes`` (one row per actuator, columns in slope
  order) and ``d = M s``.

Parity pins: every function here is pinned by closed forms, invariants and
brute force in ``tests/test_oracle_pins.py``.
"""
from __future__ import annotations

import numpy as np


# -- (a) calibration ---------------------------------------------------------
def calibrate(raw, dark, flat, thr=0.0, thr_mode=0):
    """Calibrated pixels in FP64 (Fig. 3 (a)).

    raw: uint16 array; dark, flat: float32 arrays of the same shape;
    thr: scalar threshold (ADU after flat-fielding); thr_mode 0 or 1.
    """
    raw = np.asarray(raw)
    dark32 = np.asarray(dark, dtype=np.float32)
    flat32 = np.asarray(flat, dtype=np.float32)
    p = (raw.astype(np.float64) - dark32.astype(np.float64)) * (1.0 / flat32.astype(np.float64))
    # threshold decision in IEEE single precision, as the device takes it
    gain32 = np.float32(1.0) / flat32
    p32 = (raw.astype(np.float32) - dark32) * gain32
    t32 = np.float32(thr)
    if thr_mode == 0:
        return np.where(p32 < t32, 0.0, p)
    if thr_mode == 1:
        return np.where(p32 > t32, p - float(t32), 0.0)
    raise ValueError("thr_mode must be 0 or 1")


# -- (b) centre of gravity -----------------------------------------------------
def subap_blocks(pix, subaps, npx):
    """Pixels of each valid subaperture: (nv, npx(y), npx(x)) from an (H, W) image."""
    H, W = pix.shape
    r = np.asarray(subaps)[:, 0]
    c = np.asarray(subaps)[:, 1]
    out = np.empty((len(r), npx, npx), dtype=np.float64)
    for i in range(len(r)):
        out[i] = pix[r[i] * npx:(r[i] + 1) * npx, c[i] * npx:(c[i] + 1) * npx]
    return out


def centre_of_gravity(blocks):
    """Per-subap (cx, cy) in pixels about the box centre (Fig. 3 (b)); zero where flux <= 0."""
    nv, ny, nx = blocks.shape
    xs = np.arange(nx, dtype=np.float64) - (nx - 1) / 2.0
    ys = np.arange(ny, dtype=np.float64) - (ny - 1) / 2.0
    F = blocks.sum(axis=(1, 2))
    Sx = (blocks * xs[None, None, :]).sum(axis=(1, 2))
    Sy = (blocks * ys[None, :, None]).sum(axis=(1, 2))
    ok = F > 0
    safe = np.where(ok, F, 1.0)
    cx = np.where(ok, Sx / safe, 0.0)
    cy = np.where(ok, Sy / safe, 0.0)
    return cx, cy, F


def pack_slopes(cx, cy):
    """All x gradients, then all y gradients: (x, y)_i -> (s_i, s_{n/2+i}) (Fig. 3 caption)."""
    return np.concatenate([np.asarray(cx, np.float64), np.asarray(cy, np.float64)])


def slopes(raw, dark, flat, subaps, npx, thr=0.0, thr_mode=0):
    """Slope vector of one frame; ``raw`` is (H, W) or (n_wfs, H, W) with matching maps.

    With several WFS the per-WFS vectors (each x-block then y-block) are concatenated.
    """
    raw = np.asarray(raw)
    if raw.ndim == 2:
        raw = raw[None]
        dark = np.asarray(dark)[None] if np.asarray(dark).ndim == 2 else dark
        flat = np.asarray(flat)[None] if np.asarray(flat).ndim == 2 else flat
    parts = []
    for w in range(raw.shape[0]):
        p = calibrate(raw[w], np.asarray(dark)[w], np.asarray(flat)[w], thr, thr_mode)
        cx, cy, _ = centre_of_gravity(subap_blocks(p, subaps, npx))
        parts.append(pack_slopes(cx, cy))
    return np.concatenate(parts)


# -- (c) reconstruction ----------------------------------------------------------
def reconstruct(M, s):
    """d = M s with M (nact x nslopes) as stored, widened to FP64 (Fig. 3 (c))."""
    return np.asarray(M, dtype=np.float64) @ np.asarray(s, dtype=np.float64)


# -- (d) gain / leaky integrator ---------------------------------------------------
def integrate(a_prev, d, gain, leak):
    """a <- leak * a + gain * d (Sec. 2.1's final gain, with a leak)."""
    return float(leak) * np.asarray(a_prev, np.float64) + float(gain) * np.asarray(d, np.float64)


class Loop:
    """The whole per-frame pipeline with resident integrator state, in FP64."""

    def __init__(self, M, dark, flat, subaps, npx, gain=0.4, leak=0.99, thr=0.0, thr_mode=0):
        self.M = np.asarray(M, dtype=np.float64)
        self.dark = np.asarray(dark, dtype=np.float32)
        self.flat = np.asarray(flat, dtype=np.float32)
        self.subaps = np.asarray(subaps)
        self.npx = int(npx)
        self.gain, self.leak = float(gain), float(leak)
        self.thr, self.thr_mode = float(thr), int(thr_mode)
        self.a = np.zeros(self.M.shape[0], dtype=np.float64)

    def step(self, raw, slope_override=None):
        """Process one frame; returns (dm commands, slope vector)."""
        s = slopes(raw, self.dark, self.flat, self.subaps, self.npx, self.thr, self.thr_mode)
        s_used = s if slope_override is None else np.asarray(slope_override, np.float64)
        self.a = integrate(self.a, reconstruct(self.M, s_used), self.gain, self.leak)
        return self.a.copy(), s
