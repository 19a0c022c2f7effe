"""Long ELT runs against the FP64 oracle, frame by frame.

Short runs cannot show what builds up over many frames: integrator drift with a
leak of 0.99 (a command keeps a trace of the last few hundred frames), the
predictor's 4-row history ring wrapping, the matrix slices and partial vectors
re-used frame after frame.  These runs take 1,000 ELT frames (740x740 pixels,
3972 subapertures, 4421 x 7944 matrix) through the library's per-frame call and
compare every frame's slopes (1e-5 px) and DM commands with the oracle:

* FP32 matrix: 1e-5 relative RMS, the same bound as a single frame;
* BF16 matrix with the learned predictor: also 1e-5 relative RMS.  The oracle
  applies the device's BF16 roundings (tests/mlp_emul.py) and runs on the stored
  BF16 matrix; what remains is that the device forms features from its FP32 slopes
  and the oracle from FP64 ones, so a rare feature rounds to the other BF16
  neighbour (2^-8 relative), far too rarely to reach 1e-5 in the commands.

The six-WFS stress sizing (4421 x 47664 FP8 matrix + row scales) is checked on
every actuator of two frames.
"""
import numpy as np
import pytest
import torch

import mlp_emul as E
import synth
from helpers import make_pair, rel_rms
from oracle import mlp as L
from oracle import pipeline as P
from oracle import quant as Q
from synth.mlp_init import init_mlp_params, flatten

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda:0")
N_FRAMES = 1000
CHUNK = 100


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__ as g
    g.build()


def _chunks(cfg, n, chunk=CHUNK):
    """Frames 0 .. n-1 in chunks, rendered on the CPU by one wavefront-sensor model."""
    sh = synth.wfs.ShackHartmann(cfg)
    maps = synth.calibration_maps(cfg)
    for k0 in range(0, n, chunk):
        frames, _ = synth.make_frames(cfg, k0, min(chunk, n - k0), wfs_model=sh, maps=maps)
        yield k0, frames


def _run_device(r, frames, nslopes, nact):
    """One chunk through rtc_process_frame_async on the current stream; returns the
    chunk's DM commands and measured slopes (host arrays)."""
    st = torch.cuda.current_stream()
    d_frames = frames.to(DEV)
    dm = torch.empty((frames.shape[0], nact), device=DEV)
    s = torch.empty((frames.shape[0], nslopes), device=DEV)
    for k in range(frames.shape[0]):
        r.process_frame_async(d_frames[k], dm[k], s[k], stream=st)
    r.synchronize(st)
    return dm.cpu().numpy(), s.cpu().numpy()


def test_elt_fp32_1000_frames_frame_by_frame():
    cfg = synth.elt_scao()
    r, oracle, *_ = make_pair(cfg)
    worst_s = worst_a = 0.0
    for k0, frames in _chunks(cfg, N_FRAMES):
        dm, s = _run_device(r, frames, cfg.nslopes, cfg.nact)
        for k in range(frames.shape[0]):
            a_ref, s_ref = oracle.step(frames[k].numpy())
            worst_s = max(worst_s, float(np.max(np.abs(s[k] - s_ref))))
            worst_a = max(worst_a, rel_rms(dm[k], a_ref))
            assert worst_s <= 1e-5 and worst_a <= 1e-5, (k0 + k, worst_s, worst_a)
    # the integrator has built up over the run: the state is far from one frame's step
    assert np.sqrt(np.mean(oracle.a ** 2)) > 2 * cfg.gain * np.sqrt(np.mean((oracle.M @ s_ref) ** 2))
    print(f"\n1000 ELT frames FP32: slopes {worst_s:.2e} px, DM {worst_a:.2e} rel RMS")


def test_elt_bf16_predictor_1000_frames_frame_by_frame():
    cfg = synth.elt_scao()
    r, oracle, *_ = make_pair(cfg, store="bf16")
    params = init_mlp_params(13)
    sigma = 0.3
    r.load_predictor(flatten(params), sigma)
    r.set_predictor(True)
    Pm = E.stored_params(params)
    table = L.neighbour_table(cfg.subaps, cfg.nsub)
    hist = np.zeros((4, cfg.nslopes))
    worst_s = worst_a = 0.0
    for k0, frames in _chunks(cfg, N_FRAMES):
        dm, s = _run_device(r, frames, cfg.nslopes, cfg.nact)
        for k in range(frames.shape[0]):
            raw = frames[k].numpy()
            s_ref = P.slopes(raw, oracle.dark, oracle.flat, cfg.subaps, cfg.npx)
            hist = np.concatenate([s_ref[None], hist[:3]])
            y, _, _ = E.forward(Pm, E.features_from_slopes(hist, table, sigma), gelu=E.fast_gelu,
                                gelu_grad=E.fast_gelu_grad, want_allow=False)
            s_pred = s_ref + sigma * np.concatenate([y[:, 0], y[:, 1]])
            a_ref, _ = oracle.step(raw, slope_override=s_pred)
            worst_s = max(worst_s, float(np.max(np.abs(s[k] - s_ref))))
            worst_a = max(worst_a, rel_rms(dm[k], a_ref))
            assert worst_s <= 1e-5 and worst_a <= 1e-5, (k0 + k, worst_s, worst_a)
    print(f"\n1000 ELT frames BF16 + predictor: slopes {worst_s:.2e} px, DM {worst_a:.2e} rel RMS")


def test_stress_six_wfs_fp8_every_actuator():
    """Stress sizing: 6 WFS stacked into one 4421 x 47664 FP8 matrix + row scales;
    slopes and every DM command of two frames against the oracle on the stored
    matrix, then the integrator step between them."""
    cfg = synth.elt_scao_6wfs()
    frames, _ = synth.make_frames(cfg, 0, 2)
    from paper_1805_07254_gb300 import Rtc
    dark, flat = synth.calibration_maps(cfg)
    dark, flat = dark.numpy(), flat.numpy()
    M = synth.control_matrix(cfg).numpy()
    r = Rtc(cfg.nsub, cfg.npx, cfg.nact, n_wfs=cfg.n_wfs, obs=cfg.obs, gain=cfg.gain, leak=cfg.leak)
    r.load_calib(dark, flat)
    r.load_cmat(M, store="fp8")
    oracle = P.Loop(Q.stored_matrix(M, "fp8"), dark, flat, cfg.subaps, cfg.npx, cfg.gain, cfg.leak)
    del M
    for k in range(2):
        raw = frames[k].numpy()
        dm, s = r.process_frame(raw, want_slopes=True)
        a_ref, s_ref = oracle.step(raw)
        assert np.max(np.abs(s - s_ref)) <= 1e-5
        assert rel_rms(dm, a_ref) <= 1e-5, (k, rel_rms(dm, a_ref))
        assert E.max_rel(dm, a_ref) <= 1e-4, (k, E.max_rel(dm, a_ref))
    r.close()
