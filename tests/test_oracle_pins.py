"""Pins of the FP64 oracle to facts outside itself: printed counts, closed forms,
invariants, library routines and brute force on tiny inputs.  CPU only."""
import math

import numpy as np
import pytest
import torch
from scipy.special import erf

import synth
from synth.geometry import valid_subaps, valid_actuators
from oracle import pipeline as P
from oracle import quant as Q
from oracle import mlp as L


# --------------------------------------------------------------------- geometry
def test_geometry_reproduces_paper_counts():
    # Sec. 3.1: 80x80 subaps, 0.25 D obscuration -> 4708 active subaps (9416 slopes)
    assert valid_subaps(80, 0.25).shape[0] == 4708
    # the paper's 81x81 circular DM has 5170 actuators; the circle rule gives 5169
    assert valid_actuators(81).shape[0] == 5169
    # tiny and ELT workloads
    assert valid_subaps(8, 0.0).shape[0] == 52
    assert valid_actuators(9).shape[0] == 69
    assert valid_subaps(74, 0.28).shape[0] == 3972
    assert valid_actuators(75).shape[0] == 4421


def test_subaps_row_major_order():
    sa = valid_subaps(74, 0.28)
    key = sa[:, 0] * 1000 + sa[:, 1]
    assert np.all(np.diff(key) > 0)


# --------------------------------------------------------------------- calibration
def test_calibrate_hand_values():
    raw = np.array([100, 105, 120, 99], np.uint16)
    dark = np.full(4, 100.0, np.float32)
    flat = np.array([1.0, 2.0, 0.5, 1.0], np.float32)
    # (raw - dark) / flat = [0, 2.5, 40, -1]
    np.testing.assert_array_equal(P.calibrate(raw, dark, flat, 0.0, 0), [0, 2.5, 40, 0])
    np.testing.assert_array_equal(P.calibrate(raw, dark, flat, 3.0, 0), [0, 0, 40, 0])
    np.testing.assert_array_equal(P.calibrate(raw, dark, flat, 3.0, 1), [0, 0, 37, 0])
    # exactly at threshold: mode 0 keeps (not below), mode 1 gives zero (not above)
    np.testing.assert_array_equal(P.calibrate(raw, dark, flat, 2.5, 0), [0, 2.5, 40, 0])
    np.testing.assert_array_equal(P.calibrate(raw, dark, flat, 2.5, 1), [0, 0, 37.5, 0])


def test_calibrate_inverts_detector_model():
    # raw = flat * signal + dark  ->  calibrated = signal
    sig = np.array([7.0, 0.0, 123.0, 40.0])
    flat = np.array([2.0, 1.0, 0.5, 1.25], np.float32)
    dark = np.array([10.0, 95.0, 100.5, 90.0], np.float32)
    raw = (flat * sig + dark).astype(np.uint16)
    np.testing.assert_allclose(P.calibrate(raw, dark, flat, -1e9, 0), sig, rtol=0, atol=1e-12)


# --------------------------------------------------------------------- centre of gravity
def _box_profile(n, mu, sigma):
    x = np.arange(n)
    k = 1.0 / (sigma * math.sqrt(2.0))
    return 0.5 * (erf((x + 0.5 - mu) * k) - erf((x - 0.5 - mu) * k))


def test_cog_single_pixel_is_its_offset():
    for (y0, x0) in [(0, 0), (3, 7), (9, 2), (5, 5)]:
        b = np.zeros((1, 10, 10))
        b[0, y0, x0] = 17.0
        cx, cy, F = P.centre_of_gravity(b)
        assert cx[0] == x0 - 4.5 and cy[0] == y0 - 4.5 and F[0] == 17.0


def test_cog_symmetric_spot_is_zero():
    p = _box_profile(10, 4.5, 1.2)
    b = (1000.0 * np.outer(p, p))[None]
    cx, cy, _ = P.centre_of_gravity(b)
    assert abs(cx[0]) < 1e-13 and abs(cy[0]) < 1e-13


@pytest.mark.parametrize("dx,dy", [(0.3, -0.2), (-0.45, 0.1), (0.0, 0.37), (0.5, -0.5)])
def test_cog_gaussian_spot_closed_form(dx, dy):
    n, sigma = 10, 1.2
    px = _box_profile(n, (n - 1) / 2 + dx, sigma)
    py = _box_profile(n, (n - 1) / 2 + dy, sigma)
    b = (1000.0 * np.outer(py, px))[None]           # rows = y, cols = x
    cx, cy, F = P.centre_of_gravity(b)
    xs = np.arange(n) - (n - 1) / 2
    # separable spot: the 2-D CoG equals the 1-D CoG of each marginal (truncated window)
    assert abs(cx[0] - (xs * px).sum() / px.sum()) < 1e-12
    assert abs(cy[0] - (xs * py).sum() / py.sum()) < 1e-12
    # and it recovers the true shift up to the window-truncation bias (< 1e-3 px here)
    assert abs(cx[0] - dx) < 1e-3 and abs(cy[0] - dy) < 1e-3
    assert abs(F[0] - 1000.0 * px.sum() * py.sum()) < 1e-9


def test_cog_zero_flux_gives_zero_slopes():
    b = np.zeros((2, 8, 8))
    b[1, 2, 3] = -5.0
    cx, cy, _ = P.centre_of_gravity(b)
    assert np.all(cx == 0) and np.all(cy == 0)


def test_tip_tilt_gives_uniform_slopes_in_x_then_y_order():
    # A pure tip/tilt moves every spot by the same offset: slopes are uniform,
    # all x first, then all y (Fig. 3 caption).
    cfg = synth.elt_scao()
    n = cfg.npx
    dx, dy = 0.31, -0.17
    spot = np.outer(_box_profile(n, (n - 1) / 2 + dy, 1.2), _box_profile(n, (n - 1) / 2 + dx, 1.2))
    block = np.round(1000.0 * spot + 100.0).astype(np.uint16)
    side = cfg.frame_side
    raw = np.full((side, side), 100, np.uint16)
    sa = cfg.subaps
    for r, c in sa:
        raw[r * n:(r + 1) * n, c * n:(c + 1) * n] = block
    s = P.slopes(raw, np.full((side, side), 100.0, np.float32), np.ones((side, side), np.float32),
                 sa, n)
    nv = sa.shape[0]
    assert s.shape == (2 * nv,)
    assert np.all(s[:nv] == s[0]) and np.all(s[nv:] == s[nv])
    # counts are rounded to integers (1000 e- spot), which biases the CoG by a few 1e-3 px
    assert abs(s[0] - dx) < 1e-2 and abs(s[nv] - dy) < 1e-2


def test_generator_tip_tilt_phase_gives_uniform_gradients():
    cfg = synth.tiny_scao()
    sh = synth.ShackHartmann(cfg)
    S = synth.wfs.SAMPLES_PER_SUBAP
    npts = S * cfg.nsub + 1
    yy, xx = np.meshgrid(np.arange(npts), np.arange(npts), indexing="ij")
    phase = torch.from_numpy(0.7 * xx - 0.2 * yy).float()[None]
    g = sh._gradients(phase)[0].numpy()
    np.testing.assert_allclose(g[:, 0], 0.7 * S, rtol=1e-5)
    np.testing.assert_allclose(g[:, 1], -0.2 * S, rtol=1e-5)


# --------------------------------------------------------------------- reconstruction
def test_mvm_tiny_brute_force():
    rng = np.random.default_rng(3)
    for (m, k) in [(1, 1), (2, 3), (3, 17), (69, 104)]:
        M = rng.integers(-9, 10, size=(m, k))
        s = rng.integers(-9, 10, size=k)
        expect = [sum(int(M[i, j]) * int(s[j]) for j in range(k)) for i in range(m)]
        np.testing.assert_array_equal(P.reconstruct(M, s), np.array(expect, np.float64))


def test_mvm_linearity_zero_identity_permutation():
    rng = np.random.default_rng(0)
    M = rng.standard_normal((40, 31))
    s1, s2 = rng.standard_normal(31), rng.standard_normal(31)
    np.testing.assert_allclose(P.reconstruct(M, 2.5 * s1 - 0.5 * s2),
                               2.5 * P.reconstruct(M, s1) - 0.5 * P.reconstruct(M, s2), atol=1e-12)
    assert np.all(P.reconstruct(M, np.zeros(31)) == 0)
    np.testing.assert_array_equal(P.reconstruct(np.eye(31), s1), s1)
    perm = rng.permutation(31)
    np.testing.assert_array_equal(P.reconstruct(np.eye(31)[perm], s1), s1[perm])


# --------------------------------------------------------------------- integrator
def test_integrator_closed_forms():
    g, leak = 0.4, 0.99
    d = np.array([1.0, -2.0, 0.5])
    a = np.zeros(3)
    for k in range(1, 301):
        a = P.integrate(a, d, g, leak)
        np.testing.assert_allclose(a, g * d * (1 - leak ** k) / (1 - leak), rtol=1e-12)
    a0 = np.array([3.0, -1.0, 0.0])
    a = a0.copy()
    for k in range(1, 51):
        a = P.integrate(a, np.zeros(3), g, leak)
    np.testing.assert_allclose(a, leak ** 50 * a0, rtol=1e-12)
    # leak = 1 on a zero state is the paper's plain gain factor
    np.testing.assert_array_equal(P.integrate(np.zeros(3), d, g, 1.0), g * d)


def test_loop_first_frame_is_gain_times_mvm():
    cfg = synth.tiny_scao()
    frames, _ = synth.make_frames(cfg, 0, 2)
    dark, flat = synth.calibration_maps(cfg)
    M = synth.control_matrix(cfg).numpy()
    loop = P.Loop(M, dark[0].numpy(), flat[0].numpy(), cfg.subaps, cfg.npx, 0.4, 0.99)
    a1, s1 = loop.step(frames[0, 0].numpy())
    np.testing.assert_allclose(a1, 0.4 * (M.astype(np.float64) @ s1), rtol=1e-12)
    a2, s2 = loop.step(frames[1, 0].numpy())
    np.testing.assert_allclose(a2, 0.99 * a1 + 0.4 * (M.astype(np.float64) @ s2), rtol=1e-12)


# --------------------------------------------------------------------- quantisers
def _bf16_brute(x):
    """Nearest bfloat16 by explicit search over the two truncation neighbours."""
    out = np.empty_like(x)
    for i, v in enumerate(x):
        u = np.float32(v).view(np.uint32)
        lo = np.uint32(u & 0xFFFF0000)
        hi = np.uint32(lo + 0x10000)
        flo, fhi = lo.view(np.float32), hi.view(np.float32)
        dlo, dhi = abs(float(v) - float(flo)), abs(float(fhi) - float(v))
        if dlo < dhi or (dlo == dhi and ((int(lo) >> 16) & 1) == 0):
            out[i] = flo
        else:
            out[i] = fhi
    return out


def test_bf16_round_matches_library_and_brute_force():
    rng = np.random.default_rng(1)
    x = np.concatenate([rng.standard_normal(4000).astype(np.float32) * 0.01,
                        np.array([0.0, -0.0, 1.0, 1.00390625, 1.01171875, 65504.0, -3.3e-5],
                                 np.float32)])
    mine = Q.bf16_round(x)
    lib = torch.from_numpy(x).to(torch.bfloat16).to(torch.float32).numpy()
    np.testing.assert_array_equal(mine, lib)
    np.testing.assert_array_equal(mine, _bf16_brute(x))
    # 1 + 2^-8 is a tie between 1 and 1 + 2^-7: even mantissa -> 1
    assert Q.bf16_round(np.float32(1.00390625)) == 1.0


def test_e4m3_format_and_known_roundings():
    v = Q.e4m3_values()
    assert len(v) == 127 and v[0] == 0 and v[-1] == 448.0
    assert v[1] == 2.0 ** -9 and v[8] == 2.0 ** -6
    assert np.all(np.diff(v) > 0)
    cases = {0.1: 0.1015625, 17.0: 16.0, 19.0: 20.0, 500.0: 448.0, -500.0: -448.0,
             2.0 ** -10: 0.0, 3 * 2.0 ** -10: 2.0 ** -8, 448.0: 448.0, 1.0: 1.0, -0.3: -0.3125}
    for x, want in cases.items():
        assert Q.e4m3_round(x) == want, (x, Q.e4m3_round(x), want)


def test_e4m3_round_matches_library():
    rng = np.random.default_rng(2)
    x = np.concatenate([rng.uniform(-440, 440, 3000), rng.standard_normal(3000) * 0.05,
                        Q.e4m3_values(), -Q.e4m3_values(),
                        (Q.e4m3_values()[1:] + Q.e4m3_values()[:-1]) / 2]).astype(np.float32)
    lib = torch.from_numpy(x).to(torch.float8_e4m3fn).to(torch.float64).numpy()
    np.testing.assert_array_equal(Q.e4m3_round(x), lib)


def test_fp8_row_scale_invariants():
    rng = np.random.default_rng(4)
    M = (rng.standard_normal((50, 300)) / math.sqrt(300)).astype(np.float32)
    M[7] = 0.0
    q, sc = Q.fp8_row_quantise(M)
    assert sc[7] == 1.0 and np.all(q[7] == 0)
    rows = [r for r in range(50) if r != 7]
    amax_idx = np.argmax(np.abs(M[rows]), axis=1)
    assert np.all(np.abs(q[rows, amax_idx]) == 448.0)
    assert np.all(np.abs(q) <= 448.0)
    deq = Q.stored_matrix(M, "fp8")
    np.testing.assert_allclose(np.max(np.abs(deq[rows]), 1), np.max(np.abs(M[rows]), 1), rtol=1e-6)
    # every code is a representable E4M3 value
    assert np.all(np.isin(np.abs(q), Q.e4m3_values()))


def test_f16_format_and_known_roundings():
    v = Q.f16_values()
    assert len(v) == 0x7C00 and v[0] == 0.0 and v[-1] == 65504.0
    assert v[1] == 2.0 ** -24 and v[0x400] == 2.0 ** -14 and v[0x3C00] == 1.0
    assert np.all(np.diff(v) > 0)
    # 1 + 2^-11 is a tie between 1 and 1 + 2^-10: even code -> 1; 1 + 3*2^-11 -> 1 + 2^-9
    cases = {1.0 + 2.0 ** -11: 1.0, 1.0 + 3 * 2.0 ** -11: 1.0 + 2.0 ** -9, 65519.0: 65504.0,
             65520.0: np.inf, -1e6: -np.inf, 2.0 ** -25: 0.0, 3 * 2.0 ** -25: 2.0 ** -23,
             0.1: 0.0999755859375}
    for x, want in cases.items():
        assert Q.f16_round(x) == want, (x, Q.f16_round(x), want)


def test_f16_round_matches_libraries():
    rng = np.random.default_rng(5)
    v = Q.f16_values()
    x = np.concatenate([rng.standard_normal(4000) * 0.011, rng.uniform(-6e4, 6e4, 2000),
                        rng.standard_normal(2000) * 1e-6, v[::97], -v[::89],
                        (v[1::61] + v[:-1:61]) / 2]).astype(np.float32)
    mine = Q.f16_round(x)
    np.testing.assert_array_equal(mine, x.astype(np.float16).astype(np.float64))
    np.testing.assert_array_equal(mine, torch.from_numpy(x).half().double().numpy())


def test_int8_row_quantise_invariants_and_ties():
    rng = np.random.default_rng(6)
    M = (rng.standard_normal((40, 500)) / math.sqrt(500)).astype(np.float32)
    M[3] = 0.0
    q, sc = Q.int8_row_quantise(M)
    assert sc[3] == 1.0 and np.all(q[3] == 0)
    rows = [r for r in range(40) if r != 3]
    amax_idx = np.argmax(np.abs(M[rows]), axis=1)
    assert np.all(np.abs(q[rows, amax_idx]) == 127.0)
    assert np.all(q == np.round(q)) and np.all(np.abs(q) <= 127.0)
    deq = Q.stored_matrix(M, "int8")
    # each entry within half a step of its row's grid
    assert np.all(np.abs(deq - M) <= 0.5 * sc[:, None].astype(np.float64) * (1 + 1e-6))
    # a row whose maximum is 127 has scale 1, so the codes are the entries rounded
    # half to even: 2.5 -> 2, 3.5 -> 4, -2.5 -> -2, 0.5 -> 0, 126.5 -> 126
    row = np.array([[127.0, 2.5, 3.5, -2.5, 0.5, 126.5, -127.0, 1.49]], np.float32)
    q1, s1 = Q.int8_row_quantise(row)
    assert s1[0] == 1.0
    np.testing.assert_array_equal(q1[0], [127, 2, 4, -2, 0, 126, -127, 1])


def test_reduced_precision_errors_are_ordered():
    """Relative RMS error of M s for the stored formats on an ELT-shaped block:
    FP16 < BF16 < INT8 < FP8, with FP16 and BF16 inside 2e-3 and INT8 inside 2e-2."""
    rng = np.random.default_rng(7)
    M = (rng.standard_normal((256, 8000)) / math.sqrt(8000)).astype(np.float32)
    s = rng.standard_normal(8000) * 0.3
    d = M.astype(np.float64) @ s
    err = {k: np.sqrt(np.mean((Q.stored_matrix(M, k) @ s - d) ** 2) / np.mean(d ** 2))
           for k in ("f16", "bf16", "int8", "fp8")}
    assert err["f16"] < err["bf16"] < err["int8"] < err["fp8"], err
    assert err["f16"] <= 2e-3 and err["bf16"] <= 2e-3 and err["int8"] <= 2e-2, err


# --------------------------------------------------------------------- predictor MLP
def test_gelu_matches_library_erf():
    z = np.linspace(-6, 6, 101)
    np.testing.assert_allclose(L.gelu(z), 0.5 * z * (1 + erf(z / math.sqrt(2))), rtol=0, atol=1e-15)
    tz = torch.from_numpy(z)
    np.testing.assert_allclose(L.gelu(z), torch.nn.functional.gelu(tz).numpy(), atol=1e-14)
    assert L.gelu(0.0) == 0.0


def _small_params(seed):
    from synth.mlp_init import init_mlp_params
    return {k: v.astype(np.float64) for k, v in init_mlp_params(seed).items()}


def test_mlp_backward_matches_finite_differences():
    rng = np.random.default_rng(5)
    p = _small_params(1)
    X = rng.standard_normal((7, 200))
    t = rng.standard_normal((7, 2))

    def loss(params):
        y, _ = L.forward(params, X)
        return L.mse_loss(y, t)[0]

    y, cache = L.forward(p, X)
    _, dy = L.mse_loss(y, t)
    g = L.backward(p, cache, dy)
    h = 1e-6
    for k in L.PARAM_ORDER:
        flat = p[k].reshape(-1)
        idx = rng.choice(flat.size, size=min(12, flat.size), replace=False)
        for i in idx:
            pp = {kk: vv.copy() for kk, vv in p.items()}
            pm = {kk: vv.copy() for kk, vv in p.items()}
            pp[k].reshape(-1)[i] += h
            pm[k].reshape(-1)[i] -= h
            fd = (loss(pp) - loss(pm)) / (2 * h)
            assert abs(fd - g[k].reshape(-1)[i]) < 1e-7 + 1e-5 * abs(fd), (k, i)


def test_mlp_forward_backward_match_autograd():
    rng = np.random.default_rng(6)
    p = _small_params(2)
    X = rng.standard_normal((33, 200))
    t = rng.standard_normal((33, 2))
    y, cache = L.forward(p, X)
    loss, dy = L.mse_loss(y, t)
    g = L.backward(p, cache, dy)
    tp = {k: torch.tensor(v, requires_grad=True) for k, v in p.items()}
    F = torch.nn.functional
    tx = torch.from_numpy(X)
    h1 = F.gelu(F.linear(tx, tp["W1"], tp["b1"]))
    h2 = F.gelu(F.linear(h1, tp["W2"], tp["b2"]))
    ty = F.linear(h2, tp["W3"], tp["b3"])
    tl = ((ty - torch.from_numpy(t)) ** 2).sum() / (2 * 33)
    tl.backward()
    np.testing.assert_allclose(y, ty.detach().numpy(), rtol=1e-12, atol=1e-13)
    assert abs(loss - tl.item()) < 1e-12
    for k in L.PARAM_ORDER:
        np.testing.assert_allclose(g[k], tp[k].grad.numpy(), rtol=1e-10, atol=1e-13)


def test_zero_network_outputs_bias_and_predicts_last_slopes():
    p = {k: np.zeros_like(v) for k, v in _small_params(0).items()}
    p["b3"] = np.array([0.0, 0.0])
    cfg = synth.tiny_scao()
    hist = np.random.default_rng(0).standard_normal((4, cfg.nslopes))
    np.testing.assert_array_equal(L.predict_next(p, hist, cfg.subaps, cfg.nsub, 0.3), hist[0])


def test_adam_closed_form_constant_gradient():
    p = {k: np.ones((3,)) for k in L.PARAM_ORDER}
    g = {k: np.array([0.5, -2.0, 1e-3]) for k in L.PARAM_ORDER}
    m = {k: np.zeros(3) for k in L.PARAM_ORDER}
    v = {k: np.zeros(3) for k in L.PARAM_ORDER}
    lr, eps = 1e-3, 1e-8
    for step in range(1, 6):
        p, m, v = L.adam_step(p, g, m, v, step, lr=lr, eps=eps)
        # bias-corrected moments of a constant gradient are g and g^2: each step is
        # lr * g / (|g| + eps)
        want = 1.0 - step * lr * g["W1"] / (np.abs(g["W1"]) + eps)
        np.testing.assert_allclose(p["W1"], want, rtol=1e-12)


def test_gather_places_each_neighbour():
    cfg = synth.tiny_scao()
    sa = cfg.subaps
    nv = sa.shape[0]
    hist = np.zeros((4, 2 * nv))
    for lag in range(4):
        for axis in range(2):
            hist[lag, axis * nv:(axis + 1) * nv] = 1 + 10000 * lag + 1000 * axis + np.arange(nv)
    X = L.gather_features(hist, sa, cfg.nsub, 1.0)
    pos = {tuple(rc): i for i, rc in enumerate(sa)}
    for i, (r, c) in enumerate(sa):
        for f in range(200):
            dc = f % 5 - 2
            dr = (f // 5) % 5 - 2
            axis = (f // 25) % 2
            lag = f // 50
            j = pos.get((r + dr, c + dc))
            want = 0.0 if j is None else 1 + 10000 * lag + 1000 * axis + j
            assert X[i, f] == want


@pytest.mark.parametrize("name", ["tiny", "elt"])
def test_table_gather_equals_loop_gather(name):
    """The indexed gather used for long runs places every value where the loop gather
    does (the loop gather is itself pinned above by brute-force placement)."""
    cfg = synth.CONFIGS[name]()
    sa = cfg.subaps
    nv = sa.shape[0]
    hist = np.random.default_rng(3).standard_normal((4, 2 * nv))
    table = L.neighbour_table(sa, cfg.nsub)
    assert table.shape == (nv, 25)
    assert np.all(table[:, 12] == np.arange(nv))          # the centre is the subaperture itself
    np.testing.assert_array_equal(L.gather_features_table(hist, table, 0.3),
                                  L.gather_features(hist, sa, cfg.nsub, 0.3))
