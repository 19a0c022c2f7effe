"""FP64 oracle of the learned slope predictor -- test infrastructure only.

The paper has no learned component; this predictor is an addition whose
definition is fixed here and shared (as a definition, not as code) with the
device kernels:

* features of subaperture i at frame k: the 5x5 block of subapertures centred
  on i's grid position, for the 4 most recent slope vectors, both axes -- 200
  values; neighbours off the grid or off the pupil contribute 0.  Feature
  ``f = ((lag*2 + axis)*5 + (dr+2))*5 + (dc+2)``, ``lag`` 0 = newest frame,
  ``axis`` 0 = x, 1 = y, ``dr``/``dc`` the row/column offsets in -2..2;
  all features are divided by a fixed slope scale ``sigma``;
* network: ``z1 = X W1^T + b1``, ``h1 = GELU(z1)``, ``z2 = h1 W2^T + b2``,
  ``h2 = GELU(z2)``, ``y = h2 W3^T + b3`` with 200 -> 64 -> 64 -> 2 and the
  exact GELU ``z * Phi(z)``;
* the prediction of the next slopes is ``s_k + sigma * y`` (the network
  predicts the normalised one-frame change, so a zero network reproduces the
  plain one-frame-lag behaviour);
* loss: mean squared error over the batch and both outputs,
  ``L = sum((y - t)^2) / (2B)``, targets ``t = (s_{k+1} - s_k) / sigma``;
* Adam with bias correction.

Parity pins (tests/test_oracle_pins.py): GELU against scipy's erf (a library
routine); the analytic backward against central finite differences of the
forward; Adam's first step against its closed form (a step of lr * sign(g));
the gather against brute-force placement of marked values on the grid, and
the table-driven gather against the loop gather on both geometries.
"""
from __future__ import annotations

import math

import numpy as np

LAGS = 4
HALF = 2                     # 5x5 neighbourhood
NFEAT = LAGS * 2 * (2 * HALF + 1) ** 2   # 200
SIZES = (NFEAT, 64, 64, 2)


def gather_features(history, subaps, nsub, sigma=1.0):
    """X (nv x 200) from ``history`` (LAGS x 2nv slope vectors, history[0] newest)."""
    history = np.asarray(history, dtype=np.float64)
    subaps = np.asarray(subaps)
    nv = subaps.shape[0]
    grid_idx = -np.ones((nsub, nsub), dtype=np.int64)
    grid_idx[subaps[:, 0], subaps[:, 1]] = np.arange(nv)
    X = np.zeros((nv, NFEAT), dtype=np.float64)
    for i in range(nv):
        r, c = subaps[i]
        for lag in range(LAGS):
            for axis in range(2):
                for dr in range(-HALF, HALF + 1):
                    for dc in range(-HALF, HALF + 1):
                        rr, cc = r + dr, c + dc
                        if 0 <= rr < nsub and 0 <= cc < nsub and grid_idx[rr, cc] >= 0:
                            j = grid_idx[rr, cc]
                            f = ((lag * 2 + axis) * 5 + (dr + HALF)) * 5 + (dc + HALF)
                            X[i, f] = history[lag, axis * nv + j] / sigma
    return X


def neighbour_table(subaps, nsub):
    """(nv x 25) index of each subaperture's 5x5 neighbours, (dr, dc) row-major, -1 where
    the neighbour is off the grid or off the pupil -- the same placement rule as
    ``gather_features``, tabulated once so that long runs can gather by indexing."""
    subaps = np.asarray(subaps)
    nv = subaps.shape[0]
    grid_idx = -np.ones((nsub, nsub), dtype=np.int64)
    grid_idx[subaps[:, 0], subaps[:, 1]] = np.arange(nv)
    table = -np.ones((nv, (2 * HALF + 1) ** 2), dtype=np.int64)
    for dr in range(-HALF, HALF + 1):
        for dc in range(-HALF, HALF + 1):
            rr, cc = subaps[:, 0] + dr, subaps[:, 1] + dc
            inside = (rr >= 0) & (rr < nsub) & (cc >= 0) & (cc < nsub)
            nb = (dr + HALF) * (2 * HALF + 1) + (dc + HALF)
            table[inside, nb] = grid_idx[rr[inside], cc[inside]]
    return table


def gather_features_table(history, table, sigma=1.0):
    """``gather_features`` by indexing with a ``neighbour_table``: X (nv x 200) with
    ``X[i, (lag*2 + axis)*25 + nb] = history[lag, axis*nv + table[i, nb]] / sigma``
    (0 where the table holds -1)."""
    history = np.asarray(history, dtype=np.float64)
    nv = table.shape[0]
    X = np.zeros((nv, NFEAT), dtype=np.float64)
    ok = table >= 0
    j = np.where(ok, table, 0)
    for lag in range(LAGS):
        for axis in range(2):
            vals = history[lag, axis * nv + j] / sigma
            f0 = (lag * 2 + axis) * 25
            X[:, f0:f0 + 25] = np.where(ok, vals, 0.0)
    return X


def gelu(z):
    from math import erf
    z = np.asarray(z, dtype=np.float64)
    return 0.5 * z * (1.0 + np.vectorize(erf)(z / math.sqrt(2.0)))


def gelu_grad(z):
    from math import erf
    z = np.asarray(z, dtype=np.float64)
    cdf = 0.5 * (1.0 + np.vectorize(erf)(z / math.sqrt(2.0)))
    pdf = np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)
    return cdf + z * pdf


def forward(params, X):
    """Returns (y, cache).  params = dict W1 (64x200), b1, W2 (64x64), b2, W3 (2x64), b3."""
    X = np.asarray(X, np.float64)
    z1 = X @ params["W1"].T + params["b1"]
    h1 = gelu(z1)
    z2 = h1 @ params["W2"].T + params["b2"]
    h2 = gelu(z2)
    y = h2 @ params["W3"].T + params["b3"]
    return y, dict(X=X, z1=z1, h1=h1, z2=z2, h2=h2)


def mse_loss(y, t):
    y = np.asarray(y, np.float64)
    t = np.asarray(t, np.float64)
    B = y.shape[0]
    return float(np.sum((y - t) ** 2) / (2 * B)), (y - t) / B


def backward(params, cache, dy):
    """Gradients of the loss with respect to every parameter, given dL/dy."""
    g = {}
    dy = np.asarray(dy, np.float64)
    g["W3"] = dy.T @ cache["h2"]
    g["b3"] = dy.sum(axis=0)
    dz2 = (dy @ params["W3"]) * gelu_grad(cache["z2"])
    g["W2"] = dz2.T @ cache["h1"]
    g["b2"] = dz2.sum(axis=0)
    dz1 = (dz2 @ params["W2"]) * gelu_grad(cache["z1"])
    g["W1"] = dz1.T @ cache["X"]
    g["b1"] = dz1.sum(axis=0)
    return g


PARAM_ORDER = ("W1", "b1", "W2", "b2", "W3", "b3")


def adam_step(params, grads, m, v, step, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (step counts from 1).  Returns new (params, m, v)."""
    out_p, out_m, out_v = {}, {}, {}
    for k in PARAM_ORDER:
        mk = beta1 * m[k] + (1 - beta1) * grads[k]
        vk = beta2 * v[k] + (1 - beta2) * grads[k] ** 2
        mhat = mk / (1 - beta1 ** step)
        vhat = vk / (1 - beta2 ** step)
        out_p[k] = params[k] - lr * mhat / (np.sqrt(vhat) + eps)
        out_m[k], out_v[k] = mk, vk
    return out_p, out_m, out_v


def predict_next(params, history, subaps, nsub, sigma):
    """Predicted next slope vector: s_k + sigma * y, in the x-block/y-block order."""
    X = gather_features(history, subaps, nsub, sigma)
    y, _ = forward(params, X)
    nv = X.shape[0]
    s_k = np.asarray(history[0], np.float64)
    return s_k + sigma * np.concatenate([y[:, 0], y[:, 1]]) if nv else s_k
