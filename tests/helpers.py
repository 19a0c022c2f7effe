"""Shared set-up for the GPU parity tests: one workload -> (device controller, oracle loop)."""
from __future__ import annotations

import numpy as np

import synth
from oracle import pipeline as P
from oracle import quant as Q


def rel_rms(x, ref):
    x = np.asarray(x, np.float64)
    ref = np.asarray(ref, np.float64)
    den = np.sqrt(np.mean(ref ** 2))
    return float(np.sqrt(np.mean((x - ref) ** 2)) / (den if den > 0 else 1.0))


def make_pair(cfg, store="f32", thr_mode=0, thr=0.0, subaps=None, M=None, device=0):
    """Device controller and FP64 oracle loop set up from the same seeded inputs."""
    from paper_1805_07254_gb300 import Rtc
    dark, flat = synth.calibration_maps(cfg)
    dark, flat = dark.numpy(), flat.numpy()
    sa = cfg.subaps if subaps is None else np.asarray(subaps, np.int32)
    if M is None:
        M = synth.control_matrix(cfg, nslopes=2 * sa.shape[0] * cfg.n_wfs).numpy()
    r = Rtc(cfg.nsub, cfg.npx, cfg.nact, n_wfs=cfg.n_wfs, obs=cfg.obs, gain=cfg.gain,
            leak=cfg.leak, thr_mode=thr_mode, thr=thr, device=device)
    if subaps is not None:
        r.load_subaps(sa)
    r.load_calib(dark, flat)
    r.load_cmat(M, store=store)
    Ms = Q.stored_matrix(M, store)
    oracle = P.Loop(Ms, dark, flat, sa, cfg.npx, cfg.gain, cfg.leak, thr, thr_mode)
    return r, oracle, M, dark, flat, sa
