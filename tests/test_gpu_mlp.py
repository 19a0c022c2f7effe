"""Predictor kernels (BF16 tensor-core MLP) against the FP64 oracle.

The kernels store X, W1, W2, h1 and the back-propagated dz2 / dz1 in BF16 for the
tensor-core GEMMs and keep everything else in FP32.  The comparison applies those
same roundings to the oracle's FP64 layer functions (``tests/mlp_emul.py``), so
what remains is FP32 arithmetic.  Explicit batches are redrawn, row by row, until
no value that the device rounds to BF16 lies within its FP32 error of a rounding
midpoint: the device result is then unique, and

* forward outputs agree element by element within 1e-5 of the largest output;
* every gradient element within 1e-5 of its tensor's largest element;
* the first Adam step on every entry, within the FP32 rounding of the new weight
  plus the step's sensitivity to that gradient error, lr eps dg / (|g| + eps)^2.

Where the inputs cannot be redrawn (slope histories shared by neighbouring
samples), a sample whose h1 may round the other way is allowed exactly that
rounding's effect (first order through W3, GELU'(z2) and W2).  DM commands of the
predictor path agree within 1e-5 relative RMS, the FP32 path's bound: the device
forms features from its FP32 slopes and the oracle from FP64 ones, so a feature
within an FP32 ulp of a BF16 midpoint can round the other way (2^-8 relative), but
such features are rare and their effect on the commands stays far below 1e-5
(2e-6 measured over 1,000 ELT frames).
"""
import numpy as np
import pytest
import torch

import mlp_emul as E
import synth
from helpers import make_pair, rel_rms
from oracle import mlp as L
from synth.mlp_init import init_mlp_params, flatten, unflatten

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda:0")
FWD_TOL = 1e-5      # forward: FP32 arithmetic only, relative to max |y|
GRAD_TOL = 1e-5     # gradients: per tensor, relative to its max |g|
DM_PRED_TOL = 1e-5  # DM commands with the predictor, relative RMS


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__ as g
    g.build()


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def _case(seed_p, seed_x, B):
    """A batch whose device results are unique, with its emulated forward and backward."""
    params = init_mlp_params(seed_p)
    P = E.stored_params(params)
    rng = np.random.default_rng(seed_x)
    X = 0.7 * rng.standard_normal((B, 200))
    T = 0.2 * rng.standard_normal((B, 2))
    X, T, y, cache, g, loss = E.unique_batch(P, X, T, rng)
    return params, X, T, y, g, loss


@pytest.mark.parametrize("B", [1, 64, 300])
def test_forward_matches_oracle(B):
    from paper_1805_07254_gb300 import Mlp
    params, X, _, y_ref, _, _ = _case(1, 2, B)
    m = Mlp(params=flatten(params))
    dY = torch.empty((B, 2), device=DEV)
    m.forward(_dev(X), dY)
    torch.cuda.synchronize()
    err = E.max_rel(dY.cpu().numpy(), y_ref)
    assert err <= FWD_TOL, err


@pytest.mark.parametrize("B", [64, 300])
def test_gradient_matches_oracle(B):
    from paper_1805_07254_gb300 import Mlp
    params, X, T, _, g_ref, loss = _case(3, 4, B)
    m = Mlp(params=flatten(params))
    dG = torch.empty(17154, device=DEV)
    dL = torch.empty(1, device=DEV)
    m.gradient(_dev(X), _dev(T), dG, dL)
    torch.cuda.synchronize()
    g = unflatten(dG.cpu().numpy())
    errs = {k: E.max_rel(g[k], g_ref[k]) for k in L.PARAM_ORDER}
    assert max(errs.values()) <= GRAD_TOL, errs
    assert abs(dL.item() - loss) <= 1e-5 * loss


def test_first_adam_step_matches_oracle():
    from paper_1805_07254_gb300 import Mlp
    B, lr, eps = 256, 1e-3, 1e-8
    params, X, T, _, g, _ = _case(5, 6, B)
    m = Mlp(params=flatten(params))
    m.train_step(_dev(X), _dev(T), lr)
    torch.cuda.synchronize()
    new = m.get_params()
    zeros = {k: np.zeros_like(v) for k, v in g.items()}
    master = {k: np.asarray(v, np.float32).astype(np.float64) for k, v in params.items()}
    p_ref, _, _ = L.adam_step(master, g, zeros, zeros, 1, lr=lr, eps=eps)
    old = flatten(params).astype(np.float64)
    step_gpu = new - old
    step_ref = flatten(p_ref) - old
    gf = flatten(g)
    # the gradient error the gradient test allows, per tensor
    dg = np.concatenate([np.full(np.size(g[k]), GRAD_TOL * np.max(np.abs(g[k]))) for k in L.PARAM_ORDER])
    ulp = np.spacing(np.abs(new).astype(np.float32)).astype(np.float64)
    tol = 2 * ulp + 1e-6 * lr + lr * eps * dg / (np.abs(gf) + eps) ** 2
    bad = np.abs(step_gpu - step_ref) > tol
    assert not bad.any(), (int(bad.sum()), np.flatnonzero(bad)[:10])
    # and the bound is tight (within 1e-3 lr) on almost every entry
    assert np.mean(tol <= 1e-3 * lr) > 0.99, np.mean(tol <= 1e-3 * lr)


def test_sequence_training_equals_explicit_batch():
    """rtc_mlp_train_seq gathers features from a slope sequence on the device; one
    step must equal rtc_mlp_train_step on the batch the oracle gathers."""
    from paper_1805_07254_gb300 import Mlp
    cfg = synth.tiny_scao()
    sa = cfg.subaps
    nv = sa.shape[0]
    rng = np.random.default_rng(7)
    S = (0.3 * rng.standard_normal((20, 2 * nv))).astype(np.float32)
    samples = np.stack([rng.integers(0, nv, 130), rng.integers(3, 19, 130)], axis=1).astype(np.int32)
    X = np.stack([L.gather_features(S[k::-1][:4], sa, cfg.nsub, 1.0)[i] for i, k in samples]).astype(np.float32)
    T = np.stack([(S[k + 1] - S[k])[[i, nv + i]] for i, k in samples]).astype(np.float32)
    params = flatten(init_mlp_params(8))
    a, b = Mlp(params=params), Mlp(params=params)
    b.set_geometry(sa, cfg.nsub)
    la, lb = torch.empty(1, device=DEV), torch.empty(1, device=DEV)
    a.train_step(_dev(X), _dev(T), 1e-3, la)
    b.train_seq(_dev(S), _dev(samples), 1.0, 1e-3, lb)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(a.get_params(), b.get_params())
    assert la.item() == lb.item()


def test_training_lowers_the_loss():
    from paper_1805_07254_gb300 import Mlp
    rng = np.random.default_rng(9)
    B = 1024
    w = rng.standard_normal((200, 2)) / 20
    X = (0.7 * rng.standard_normal((B, 200))).astype(np.float32)
    T = np.tanh(X.astype(np.float64) @ w).astype(np.float32)
    m = Mlp(params=flatten(init_mlp_params(10)))
    dX, dT, dL = _dev(X), _dev(T), torch.empty(1, device=DEV)
    losses = []
    for step in range(300):
        m.train_step(dX, dT, 3e-3, dL)
        if step in (0, 299):
            torch.cuda.synchronize()
            losses.append(dL.item())
    assert losses[1] < 0.2 * losses[0], losses


def test_predict_seq_matches_oracle():
    from paper_1805_07254_gb300 import Mlp
    cfg = synth.tiny_scao()
    sa = cfg.subaps
    nv = sa.shape[0]
    rng = np.random.default_rng(11)
    S = (0.3 * rng.standard_normal((12, 2 * nv))).astype(np.float32)
    params = init_mlp_params(12)
    m = Mlp(params=flatten(params))
    m.set_geometry(sa, cfg.nsub)
    sigma = 0.3
    dout = torch.zeros((12, 2 * nv), device=DEV)
    m.predict_seq(_dev(S), sigma, dout)
    torch.cuda.synchronize()
    out = dout.cpu().numpy()
    P = E.stored_params(params)
    table = L.neighbour_table(sa, cfg.nsub)
    for k in range(3, 11):
        Xb = E.features_from_slopes(S[k::-1][:4], table, sigma)
        y, _, allow = E.forward(P, Xb)
        ref = S[k].astype(np.float64) + sigma * np.concatenate([y[:, 0], y[:, 1]])
        # FP32 arithmetic, the other rounding of an ambiguous h1, the FP32 result's ulp
        tol = (FWD_TOL * sigma * np.max(np.abs(y)) + sigma * np.concatenate([allow[:, 0], allow[:, 1]])
               + np.spacing(np.abs(ref).astype(np.float32)))
        worst = float(np.max(np.abs(out[k + 1] - ref) / tol))
        assert worst <= 1.0, (k, worst)
    assert np.all(out[:4] == 0)


def test_handle_predictor_path_matches_oracle():
    cfg = synth.tiny_scao()
    frames, _ = synth.make_frames(cfg, 0, 12)
    frames = frames.numpy()
    r, oracle, *_ = make_pair(cfg)
    params = init_mlp_params(13)
    sigma = 0.3
    r.load_predictor(flatten(params), sigma)
    r.set_predictor(True)
    P = E.stored_params(params)
    table = L.neighbour_table(cfg.subaps, cfg.nsub)
    hist = np.zeros((4, cfg.nslopes))
    from oracle import pipeline as PL
    worst = 0.0
    for k in range(frames.shape[0]):      # the 4-row history ring wraps twice
        dm, s = r.process_frame(frames[k], want_slopes=True)
        s_ref = PL.slopes(frames[k], oracle.dark, oracle.flat, cfg.subaps, cfg.npx)
        hist = np.concatenate([s_ref[None], hist[:3]])
        y, _, _ = E.forward(P, E.features_from_slopes(hist, table, sigma))
        s_pred = s_ref + sigma * np.concatenate([y[:, 0], y[:, 1]])
        a_ref, _ = oracle.step(frames[k], slope_override=s_pred)
        assert np.max(np.abs(s - s_ref)) <= 1e-5
        worst = max(worst, rel_rms(dm, a_ref))
    assert worst <= DM_PRED_TOL, worst
    # switched off: the plain path again, from a fresh state
    r.set_predictor(False)
    r.reset()
    oracle.a[:] = 0
    dm = r.process_frame(frames[0])
    a_ref, _ = oracle.step(frames[0])
    assert rel_rms(dm, a_ref) <= 1e-5


@pytest.mark.parametrize("cfg_name", ["tiny", "elt"])
def test_fused_prediction_equals_standalone_kernels(cfg_name):
    """The prediction inside the fused frame kernel is the stand-alone predictor's, bit
    for bit: a handle with the predictor on gives the DM commands of a plain handle
    that reconstructs from rtc_mlp_predict_seq's predictions of the slopes the first
    handle measured."""
    from paper_1805_07254_gb300 import Mlp
    cfg = synth.CONFIGS[cfg_name]()
    n = 7
    frames, _ = synth.make_frames(cfg, 0, n)
    r1, *_ = make_pair(cfg, store="bf16")
    r2, *_ = make_pair(cfg, store="bf16")
    params = flatten(init_mlp_params(21))
    sigma = 0.25
    r1.load_predictor(params, sigma)
    r1.set_predictor(True)
    nv, nslopes = cfg.subaps.shape[0], cfg.nslopes
    st = torch.cuda.current_stream()
    d_frames = frames.to(DEV)
    dm1 = torch.zeros((n, cfg.nact), device=DEV)
    s1 = torch.zeros((n, nslopes), device=DEV)
    for k in range(n):
        r1.process_frame_async(d_frames[k], dm1[k], s1[k], stream=st)
    # the measured slopes the fused path reported, after 3 empty history rows
    S = torch.zeros((n + 4, nslopes), device=DEV)
    S[3:3 + n] = s1
    m = Mlp(params=params)
    m.set_geometry(cfg.subaps, cfg.nsub)
    P = torch.zeros_like(S)
    m.predict_seq(S, sigma, P, stream=st)
    kpad = r2.info()["kpad"]
    dm2 = torch.zeros((n, cfg.nact), device=DEV)
    for k in range(n):
        sp = torch.zeros(kpad, device=DEV)
        sp[:nslopes] = P[k + 4]
        r2.reconstruct_async(sp, dm2[k], stream=st)
        torch.cuda.synchronize()
    torch.cuda.synchronize()
    assert nv * 2 == nslopes
    assert torch.count_nonzero(s1) > 0
    assert torch.equal(dm1, dm2)
