"""Seeded initial weights for the slope-predictor MLP (200 -> 64 -> 64 -> 2).

Every weight and bias of a layer with fan-in ``k`` is drawn uniformly from
``[-1/sqrt(k), 1/sqrt(k)]``.  These are inputs (the method's random draw), so
the device training run and the FP64 oracle start from identical values.
"""
from __future__ import annotations

import numpy as np

SIZES = (200, 64, 64, 2)
ORDER = ("W1", "b1", "W2", "b2", "W3", "b3")


def init_mlp_params(seed: int = 0) -> dict:
    rng = np.random.default_rng(seed)
    p = {}
    for li in range(3):
        fan_in, fan_out = SIZES[li], SIZES[li + 1]
        bound = 1.0 / np.sqrt(fan_in)
        p[f"W{li + 1}"] = rng.uniform(-bound, bound, size=(fan_out, fan_in)).astype(np.float32)
        p[f"b{li + 1}"] = rng.uniform(-bound, bound, size=(fan_out,)).astype(np.float32)
    return p


def flatten(params: dict) -> np.ndarray:
    """Concatenate parameters in the order W1, b1, W2, b2, W3, b3 (row-major) -> float32."""
    return np.concatenate([np.asarray(params[k], np.float32).reshape(-1) for k in ORDER])


def unflatten(vec) -> dict:
    vec = np.asarray(vec)
    out, off = {}, 0
    shapes = {"W1": (64, 200), "b1": (64,), "W2": (64, 64), "b2": (64,), "W3": (2, 64), "b3": (2,)}
    for k in ORDER:
        n = int(np.prod(shapes[k]))
        out[k] = vec[off:off + n].reshape(shapes[k])
        off += n
    return out
