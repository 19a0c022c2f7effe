"""The predictor network of oracle/mlp.py evaluated at the device kernels' rounding points.

The device kernels (forward, backward, fused inference) keep the network's FP64
definition except where they store values in BF16 for the tensor-core GEMMs:

* the features X (formed in FP32 as ``x * fl32(1/sigma)``),
* the weights W1 and W2,
* the first hidden activation h1 = GELU(z1),
* the back-propagated dz2 and dz1 that feed the dh1 and weight-gradient GEMMs.

Everything else (z1, z2, h2, y, dy, the bias gradients, W3 and its gradient) stays
in FP32 on the device and in FP64 here.  The functions below apply exactly those
roundings to FP64 values computed with the oracle's own layer functions, so that
the remaining device-vs-oracle difference is FP32 arithmetic (about 1e-6
relative) -- except where a value lies so close to a BF16 rounding midpoint that
the device's FP32 value may round to the other neighbour.  Such places are found
from an error bound on the device's FP32 value (``bf16_flip``); a test either
redraws its synthetic inputs until there are none (the result is then unique) or
allows exactly the effect of the other rounding.

Test infrastructure only; nothing here is used by the library.
"""
from __future__ import annotations

import math

import numpy as np

from oracle import mlp as L
from oracle import quant as Q

U32 = 2.0 ** -24          # FP32 unit roundoff
GELU2_MAX = 0.8           # largest |GELU''(z)| (0.798 at z = 0)


def bf16(x):
    """FP32 rounding then BF16 round-to-nearest-even, returned as FP64."""
    return Q.bf16_round(np.asarray(x, np.float64).astype(np.float32)).astype(np.float64)


def bf16_flip(v, delta):
    """(rounded, width): the BF16 rounding of v and, where a rounding midpoint lies
    within +-delta of v (a device value that far off may round to the other side),
    the signed step to the other candidate; 0 elsewhere.  Rounding is monotone, so
    the candidates are the roundings of v - delta and v + delta."""
    v = np.asarray(v, np.float64)
    r = bf16(v)
    lo, hi = bf16(v - delta), bf16(v + delta)
    return r, np.where(hi != r, hi - r, lo - r)


def stored_params(params):
    """Parameters as the kernels hold them: W1, W2 in BF16, the rest FP32, as FP64."""
    out = {k: np.asarray(v, np.float32).astype(np.float64) for k, v in params.items()}
    out["W1"] = bf16(params["W1"])
    out["W2"] = bf16(params["W2"])
    return out


def features_from_slopes(history, table, sigma):
    """Features as the device forms them from FP32 slope rows: bf16(x * fl32(1/sigma))
    with the product in FP32, gathered with the oracle's neighbour table."""
    inv = np.float32(1.0) / np.float32(sigma)
    raw = L.gather_features_table(np.asarray(history, np.float64).astype(np.float32), table, 1.0)
    return bf16(raw.astype(np.float32) * inv)


def fast_gelu(z):
    """GELU through scipy's erf (the oracle's GELU is pinned against that library
    routine); for long runs, where the oracle's element-wise erf takes minutes."""
    from scipy.special import erf
    z = np.asarray(z, np.float64)
    return 0.5 * z * (1.0 + erf(z / math.sqrt(2.0)))


def fast_gelu_grad(z):
    """GELU'(z) = Phi(z) + z phi(z) through scipy's erf (see fast_gelu)."""
    from scipy.special import erf
    z = np.asarray(z, np.float64)
    return 0.5 * (1.0 + erf(z / math.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)


def forward(P, Xb, gelu=L.gelu, gelu_grad=L.gelu_grad, want_allow=True):
    """Forward pass at the device's rounding points.  P: stored_params; Xb: BF16 features
    (FP64 array).  Returns (y, cache, allow): allow[s, o] is how far y[s, o] moves if
    every h1 entry of sample s that may round the other way does (first order, with
    the sample's own GELU slopes; 0 for a sample with no such entry; None unless
    want_allow)."""
    Xb = np.asarray(Xb, np.float64)
    z1 = Xb @ P["W1"].T + P["b1"]
    # device z1: FP32 tensor-core sum of 208 exact products; a generous error bound
    dz1 = 8 * U32 * (np.abs(Xb) @ np.abs(P["W1"]).T + np.abs(P["b1"]))
    g1 = gelu(z1)
    d1 = gelu_grad(z1)
    h1, width = bf16_flip(g1, np.abs(d1) * dz1 + 8 * U32 * np.abs(g1))
    z2 = h1 @ P["W2"].T + P["b2"]
    h2 = gelu(z2)
    y = h2 @ P["W3"].T + P["b3"]
    g2 = gelu_grad(z2)
    allow = None
    if want_allow:
        # dy[s, o] / dh1[s, j] = sum_n W3[o, n] gelu'(z2[s, n]) W2[n, j]
        sens = np.einsum("on,sn,nj->soj", P["W3"], g2, P["W2"])
        allow = 1.5 * np.einsum("sj,soj->so", np.abs(width), np.abs(sens))
    cache = dict(X=Xb, z1=z1, dz1=dz1, g1p=d1, h1=h1, flip_h1=width != 0, z2=z2, h2=h2, g2p=g2)
    return y, cache, allow


def backward(P, cache, dy, y_err=0.0):
    """Gradients at the device's rounding points (dz2 and dz1 rounded to BF16 where they
    enter a GEMM; the bias gradients sum the unrounded values).  y_err: bound on the
    device's error in dy (absolute).  Returns (grads, flagged): flagged[s] is True
    where a dz2 or dz1 entry of sample s may round the other way on the device."""
    dy = np.asarray(dy, np.float64)
    g = {"W3": dy.T @ cache["h2"], "b3": dy.sum(axis=0)}
    dh2 = dy @ P["W3"]
    g2p = cache["g2p"]
    # device dz2 = fl32(fl32(dy W3) * gelu'(z2)): errors from dy, the FMA pair, gelu'
    dz2_h2 = 8 * U32 * (np.abs(cache["h1"]) @ np.abs(P["W2"]).T + np.abs(P["b2"]))
    dz2 = dh2 * g2p
    d_dz2 = (np.abs(g2p) * (y_err * np.abs(P["W3"]).sum(axis=0) + 4 * U32 * np.abs(dy) @ np.abs(P["W3"]))
             + np.abs(dh2) * (GELU2_MAX * dz2_h2 + 8 * U32 * np.abs(g2p)) + 4 * U32 * np.abs(dz2))
    g["b2"] = dz2.sum(axis=0)
    dz2b, w2 = bf16_flip(dz2, d_dz2)
    g["W2"] = dz2b.T @ cache["h1"]
    dh1 = dz2b @ P["W2"]
    g1p = cache["g1p"]
    dz1 = dh1 * g1p
    d_dz1 = (np.abs(g1p) * 8 * U32 * (np.abs(dz2b) @ np.abs(P["W2"]))
             + np.abs(dh1) * (GELU2_MAX * cache["dz1"] + 8 * U32 * np.abs(g1p)) + 4 * U32 * np.abs(dz1))
    g["b1"] = dz1.sum(axis=0)
    dz1b, w1 = bf16_flip(dz1, d_dz1)
    g["W1"] = dz1b.T @ cache["X"]
    flagged = (w2 != 0).any(axis=1) | (w1 != 0).any(axis=1)
    return g, flagged


def unique_batch(P, X, T, rng, scale_x=0.7, scale_t=0.2, max_rounds=200):
    """Redraw rows of a synthetic batch until no BF16 rounding on the device path is
    ambiguous: rows with an h1 entry near a midpoint get new features, rows with a
    dz2 / dz1 entry near one new features and targets.  Returns (X, T, y, cache, grads, loss)
    for the final batch, whose device results are then unique up to FP32 rounding."""
    X = np.array(X, np.float32)
    T = np.array(T, np.float32)
    B = X.shape[0]
    for _ in range(max_rounds):
        y, cache, _ = forward(P, bf16(X))
        bad = cache["flip_h1"].any(axis=1)
        if bad.any():
            X[bad] = (scale_x * rng.standard_normal((int(bad.sum()), X.shape[1]))).astype(np.float32)
            continue
        loss, dy = L.mse_loss(y, T)
        # device y: FP32 (a 64-term FMA chain after GELU of FP32 z2), a few ulps of max |y|
        y_err = 8 * U32 * np.max(np.abs(y)) / B
        g, flagged = backward(P, cache, dy, y_err)
        if flagged.any():
            n = int(flagged.sum())
            X[flagged] = (scale_x * rng.standard_normal((n, X.shape[1]))).astype(np.float32)
            T[flagged] = (scale_t * rng.standard_normal((n, T.shape[1]))).astype(np.float32)
            continue
        return X, T, y, cache, g, loss
    raise RuntimeError("could not draw a batch without ambiguous BF16 roundings")


def max_rel(x, ref):
    """Largest element-wise deviation relative to the largest reference magnitude."""
    x = np.asarray(x, np.float64)
    ref = np.asarray(ref, np.float64)
    if ref.size == 0:
        return 0.0
    den = np.max(np.abs(ref))
    return float(np.max(np.abs(x - ref)) / (den if den > 0 else 1.0))
