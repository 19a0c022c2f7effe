"""Training and evaluation of the learned slope predictor on pipeline slopes.

Slopes come from the pipeline itself: seeded frozen-flow frames are rendered on
the GPU and centroided by the library's pixel-stage kernel.  Training runs the
library's own forward/backward/Adam kernels (rtc_mlp_train_seq) on random
(subaperture, frame) samples; evaluation runs rtc_mlp_predict_seq on held-out
frames from new seeds.

The yardstick for the predictor is the plain integrator's one-frame servo lag:
  integrator residual = RMS(s_{k+1} - s_k)       (commands built from s_k act on k+1)
  predictor residual  = RMS(s_{k+1} - s_hat_{k+1})
over the same held-out frames.  The predictor is kept only if its residual is
lower.
"""
from __future__ import annotations

import math
import time
from dataclasses import dataclass

import numpy as np
import torch

import synth
from .rtc import Mlp, Rtc


@dataclass
class PredictorResult:
    params: np.ndarray
    sigma: float
    steps: int
    train_frames: int
    test_frames: int
    residual_predictor: float
    residual_integrator: float
    train_seconds: float
    final_loss: float

    @property
    def gain(self) -> float:
        """Integrator residual over predictor residual (> 1 means the predictor helps)."""
        return self.residual_integrator / self.residual_predictor

    @property
    def keep(self) -> bool:
        return self.residual_predictor < self.residual_integrator


def pipeline_slopes(cfg, n_frames: int, screen_seeds, noise_seed: int, device="cuda:0",
                    chunk: int = 64, start: int = 0) -> torch.Tensor:
    """Slope vectors [n_frames][2 n_valid] of frames start.. rendered on `device` and
    centroided by the library (rtc_centroid_async)."""
    dev = torch.device(device)
    sh = synth.ShackHartmann(cfg, device=dev, screen_seeds=screen_seeds)
    dark, flat = synth.calibration_maps(cfg, device=dev)
    r = Rtc(cfg.nsub, cfg.npx, cfg.nact, obs=cfg.obs, device=dev.index or 0)
    r.load_calib(dark.cpu().numpy(), flat.cpu().numpy())
    S = torch.empty((n_frames, cfg.nslopes), dtype=torch.float32, device=dev)
    st = torch.cuda.current_stream(dev)
    for c0 in range(0, n_frames, chunk):
        n = min(chunk, n_frames - c0)
        frames, _ = synth.make_frames(cfg, start + c0, n, device=dev, wfs_model=sh,
                                      maps=(dark, flat), noise_seed=noise_seed)
        frames = frames.contiguous()
        for j in range(n):
            r.centroid_async(frames[j], S[c0 + j], stream=st)
    r.synchronize(st)
    r.close()
    return S


def residuals(S: torch.Tensor, S_hat: torch.Tensor, k0: int = 4) -> tuple[float, float]:
    """(predictor, integrator) residual RMS over frames k0+1 .. end."""
    nxt = S[k0 + 1:]
    pred = torch.sqrt(torch.mean((nxt - S_hat[k0 + 1:]) ** 2)).item()
    lag = torch.sqrt(torch.mean((nxt - S[k0:-1]) ** 2)).item()
    return pred, lag


def train_on(S: torch.Tensor, cfg, steps: int | None = None, batch: int = 4096, lr: float = 1e-3,
             seed: int = 0, log_every: int = 0):
    """Train a network on the slope sequence S [frames][2 n_valid] (device) with the
    library's training kernel: random (subaperture, frame) samples, target the next
    frame's slope change over sigma = RMS(S).  One epoch of samples unless `steps`
    is given.  Returns (Mlp, sigma, steps, final loss, seconds)."""
    dev = S.device
    n_frames = S.shape[0]
    sigma = float(torch.sqrt(torch.mean(S ** 2)).item())
    from synth.mlp_init import init_mlp_params, flatten
    m = Mlp(device=dev.index or 0, params=flatten(init_mlp_params(seed)))
    m.set_geometry(cfg.subaps, cfg.nsub)
    nv = cfg.n_valid
    if steps is None:
        steps = max(1, (n_frames - 5) * nv // batch)
    gen = torch.Generator(device=dev)
    gen.manual_seed(9000 + seed)
    d_loss = torch.zeros(1, device=dev)
    samples = torch.empty((batch, 2), dtype=torch.int32, device=dev)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for step in range(steps):
        samples[:, 0] = torch.randint(0, nv, (batch,), generator=gen, device=dev, dtype=torch.int32)
        samples[:, 1] = torch.randint(3, n_frames - 1, (batch,), generator=gen, device=dev,
                                      dtype=torch.int32)
        m.train_seq(S, samples, sigma, lr, d_loss)
        if log_every and step % log_every == 0:
            print(f"step {step} loss {d_loss.item():.5f}", flush=True)
    torch.cuda.synchronize(dev)
    return m, sigma, steps, d_loss.item(), time.perf_counter() - t0


def train_predictor(cfg=None, train_frames: int = 200_000, test_frames: int = 20_000,
                    steps: int | None = None, batch: int = 4096, lr: float = 1e-3, seed: int = 0,
                    device="cuda:0", log_every: int = 0) -> PredictorResult:
    """Train on `train_frames` pipeline frames (one epoch of samples unless `steps`
    is given) and evaluate on `test_frames` held-out frames with new seeds."""
    cfg = cfg or synth.elt_scao()
    dev = torch.device(device)
    nl = len(cfg.screen_seeds)
    train_seeds = tuple(1000 + 10 * seed + i for i in range(nl))
    test_seeds = tuple(5000 + 10 * seed + i for i in range(nl))
    S = pipeline_slopes(cfg, train_frames, train_seeds, noise_seed=7000 + seed, device=dev)
    m, sigma, steps, final_loss, train_s = train_on(S, cfg, steps, batch, lr, seed, log_every)
    del S
    T = pipeline_slopes(cfg, test_frames, test_seeds, noise_seed=8000 + seed, device=dev)
    T_hat = torch.zeros_like(T)
    m.predict_seq(T, sigma, T_hat)
    torch.cuda.synchronize(dev)
    res_p, res_i = residuals(T, T_hat)
    params = m.get_params()
    m.close()
    return PredictorResult(params=params, sigma=sigma, steps=steps, train_frames=train_frames,
                           test_frames=test_frames, residual_predictor=res_p,
                           residual_integrator=res_i, train_seconds=train_s, final_loss=final_loss)


def main(argv=None):
    import argparse
    import json
    ap = argparse.ArgumentParser(description="Train the slope predictor on pipeline slopes "
                                 "and compare it with the integrator on held-out frames.")
    ap.add_argument("--config", default="elt", choices=sorted(synth.CONFIGS))
    ap.add_argument("--train-frames", type=int, default=200_000)
    ap.add_argument("--test-frames", type=int, default=20_000)
    ap.add_argument("--steps", type=int, default=None)
    ap.add_argument("--batch", type=int, default=4096)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--save", default=None, help="write the trained parameters (.npy)")
    a = ap.parse_args(argv)
    res = train_predictor(synth.CONFIGS[a.config](), a.train_frames, a.test_frames, a.steps,
                          a.batch, a.lr, a.seed)
    if a.save:
        np.save(a.save, res.params)
    print(json.dumps({"config": a.config, "train_frames": res.train_frames, "test_frames": res.test_frames,
                      "steps": res.steps, "batch": a.batch, "lr": a.lr, "sigma_px": res.sigma,
                      "final_loss": res.final_loss, "train_seconds": round(res.train_seconds, 2),
                      "residual_rms_predictor_px": res.residual_predictor,
                      "residual_rms_integrator_px": res.residual_integrator,
                      "gain": res.gain, "keep_predictor": res.keep}))


if __name__ == "__main__":
    main()
