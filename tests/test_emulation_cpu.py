"""CPU checks of the test-side emulation of the device's BF16 rounding points
(tests/mlp_emul.py), against the oracle and the format itself."""
import numpy as np

import mlp_emul as E
import synth
from oracle import mlp as L
from oracle import quant as Q
from synth.mlp_init import init_mlp_params


def test_bf16_flip_finds_midpoints_only():
    one = 1.0                                  # BF16 spacing at 1 is 2^-7
    mid = one + 2.0 ** -8                      # the midpoint between 1 and 1 + 2^-7
    r, w = E.bf16_flip(np.array([one, mid - 1e-6, mid + 1e-6, 1.5]), 4e-6)
    np.testing.assert_array_equal(r, [1.0, 1.0, 1.0 + 2.0 ** -7, 1.5])
    np.testing.assert_array_equal(w, [0.0, 2.0 ** -7, -(2.0 ** -7), 0.0])
    r, w = E.bf16_flip(np.array([mid - 1e-6, mid + 1e-6]), 1e-7)
    np.testing.assert_array_equal(w, [0.0, 0.0])


def test_fast_gelu_equals_oracle_gelu():
    z = np.linspace(-8, 8, 20001)
    np.testing.assert_allclose(E.fast_gelu(z), L.gelu(z), rtol=0, atol=1e-15)
    np.testing.assert_allclose(E.fast_gelu_grad(z), L.gelu_grad(z), rtol=0, atol=1e-15)


def test_emulated_forward_is_the_oracle_on_rounded_values():
    """With the roundings applied to the oracle's inputs by hand, the oracle's forward
    gives the emulation's outputs: the emulation adds roundings, nothing else."""
    params = init_mlp_params(3)
    P = E.stored_params(params)
    X = 0.7 * np.random.default_rng(1).standard_normal((40, 200))
    Xb = E.bf16(X)
    y, cache, _ = E.forward(P, Xb)
    h1 = Q.bf16_round(L.gelu(Xb @ P["W1"].T + P["b1"]).astype(np.float32)).astype(np.float64)
    np.testing.assert_array_equal(cache["h1"], h1)
    y2 = L.gelu(h1 @ P["W2"].T + P["b2"]) @ P["W3"].T + P["b3"]
    np.testing.assert_allclose(y, y2, rtol=1e-13, atol=1e-15)


def test_unique_batch_has_no_ambiguous_rounding():
    params = init_mlp_params(3)
    P = E.stored_params(params)
    rng = np.random.default_rng(2)
    X, T, y, cache, g, loss = E.unique_batch(P, 0.7 * rng.standard_normal((64, 200)),
                                             0.2 * rng.standard_normal((64, 2)), rng)
    assert not cache["flip_h1"].any()
    _, dy = L.mse_loss(y, T)
    _, flagged = E.backward(P, cache, dy, 8 * E.U32 * np.max(np.abs(y)) / 64)
    assert not flagged.any()


def test_features_from_slopes_round_the_fp32_product():
    cfg = synth.tiny_scao()
    hist = 0.3 * np.random.default_rng(4).standard_normal((4, cfg.nslopes))
    table = L.neighbour_table(cfg.subaps, cfg.nsub)
    X = E.features_from_slopes(hist, table, 0.3)
    raw = L.gather_features(hist.astype(np.float32), cfg.subaps, cfg.nsub, 1.0).astype(np.float32)
    want = Q.bf16_round(raw * (np.float32(1.0) / np.float32(0.3))).astype(np.float64)
    np.testing.assert_array_equal(X, want)
