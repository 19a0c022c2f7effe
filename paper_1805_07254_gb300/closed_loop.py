"""Physical closed loop: the controller drives a deformable mirror that corrects
the turbulence its WFS sees.

The paper's RTC computes DM commands from slopes through a control matrix and a
gain (Sec. 2.1, Fig. 3 (c)-(d)); its experiments use a random matrix, and so does
the benchmark here.  This module closes the loop physically:

* the mirror is a Fried-geometry DM whose surface is the bilinear interpolation
  of its commands, and the WFS sees turbulence minus mirror (``synth.dm``);
* the control matrix is the regularised least-squares reconstructor of the
  DM-to-WFS interaction matrix;
* every frame, the true residual slopes ``s_turb(k) - D a(k-1)`` (the commands of
  the previous frame are on the mirror: a one-frame servo lag) are rendered into
  a detector frame with photon and read noise, and the controller turns that
  frame into new commands.

The controller is a callable (frame -> commands); with the library it is one
``rtc_process_frame_async`` per frame on the simulation's CUDA stream, so frames,
slopes, commands and mirror never leave the device.  The scores are the RMS of
the true residual slopes the WFS sees and the RMS of the residual wavefront over
the pupil (piston removed), against the turbulence alone.  ``evaluate`` compares
the plain integrator with the integrator fed by the learned slope predictor,
trained on the residual slopes of closed-loop runs with other turbulence;
``evaluate_pol`` compares it with pseudo-open-loop predictive control, the
predictor forecasting the turbulence's own slopes (``PolController``).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
import torch

import synth
from synth.dm import FriedDM, reconstructor
from synth.wfs import SAMPLES_PER_SUBAP
from .rtc import Rtc

NM_PER_RAD = 500.0 / (2.0 * math.pi)       # the screens are phase in radians at 500 nm


@dataclass
class LoopScore:
    frames: int                  # frames scored (after the burn-in)
    slope_rms_px: float          # true residual slopes seen by the WFS
    phase_rms_rad: float         # residual wavefront over the pupil, piston removed
    open_slope_rms_px: float     # the turbulence's own slopes
    open_phase_rms_rad: float    # the turbulence's own wavefront, piston removed

    @property
    def phase_rms_nm(self) -> float:
        return self.phase_rms_rad * NM_PER_RAD

    @property
    def open_phase_rms_nm(self) -> float:
        return self.open_phase_rms_rad * NM_PER_RAD


class ClosedLoopSim:
    """Turbulence, WFS and DM of one workload on one device."""

    def __init__(self, cfg, device="cuda:0", screen_seeds=None, noise_seed: int | None = None,
                 alpha_rel: float = 1e-3):
        if cfg.n_wfs != 1:
            raise ValueError("the closed loop drives one WFS")
        self.cfg = cfg
        self.device = torch.device(device)
        self.sh = synth.ShackHartmann(cfg, device=self.device, screen_seeds=screen_seeds)
        self.dm = FriedDM(cfg, self.sh.plate_scale, SAMPLES_PER_SUBAP)
        D = self.dm.interaction()
        self.R = reconstructor(D, alpha_rel).astype(np.float32)          # control matrix
        self.D = torch.from_numpy(D.astype(np.float32)).to(self.device)
        dark, flat = synth.calibration_maps(cfg, device=self.device)
        self.dark, self.flat = dark, flat
        self.noise_seed = cfg.noise_seed if noise_seed is None else noise_seed
        # the pupil on the WFS sampling grid: the union of the valid subapertures
        S = SAMPLES_PER_SUBAP
        npts = S * cfg.nsub + 1
        m = torch.zeros((npts, npts), dtype=torch.bool)
        for r, c in cfg.subaps:
            m[S * r:S * (r + 1) + 1, S * c:S * (c + 1) + 1] = True
        self.mask = m.to(self.device)
        self.npup = int(m.sum())

    def _phase_sq(self, ph: torch.Tensor) -> torch.Tensor:
        """Sum of squares of a wavefront over the pupil after removing its mean."""
        v = ph[self.mask]
        v = v - v.mean()
        return torch.sum(v.double() ** 2)

    def run(self, step, n_frames: int, start: int = 0, burn_in: int = 50, chunk: int = 32,
            trace: list | None = None) -> LoopScore:
        """Close the loop for frames start .. start+n_frames-1 with `step` (uint16 frame
        (H, W) on the device -> new commands (nact,) on the device, applied from the
        next frame on).  Scores frames after the first `burn_in`; `trace` receives each
        scored frame's residual wavefront RMS (radians) when given."""
        cfg, sh, dev = self.cfg, self.sh, self.device
        nv = cfg.n_valid
        gen = torch.Generator(device=dev)
        gen.manual_seed(int(self.noise_seed) * 1_000_003 + int(start))
        a = torch.zeros(self.dm.nact, device=dev)
        zero = torch.zeros((), dtype=torch.float64, device=dev)
        res_s, res_p, open_s, open_p = zero.clone(), zero.clone(), zero.clone(), zero.clone()
        scored = 0
        for c0 in range(start, start + n_frames, chunk):
            n = min(chunk, start + n_frames - c0)
            idx = torch.arange(c0, c0 + n)
            s_turb = sh.true_slopes(idx)                                     # n x nv x 2
            ph_turb = sh.flow.phase(idx.double() / cfg.frame_rate_hz)        # n x npts x npts
            for j in range(n):
                s_dm = self.D @ a
                s_res = s_turb[j] - torch.stack([s_dm[:nv], s_dm[nv:]], dim=-1)
                if c0 + j - start >= burn_in:
                    res_s += torch.sum(s_res.double() ** 2)
                    open_s += torch.sum(s_turb[j].double() ** 2)
                    sq = self._phase_sq(ph_turb[j] - self.dm.phase(a)[0])
                    res_p += sq
                    if trace is not None:
                        trace.append(sq)
                    open_p += self._phase_sq(ph_turb[j])
                    scored += 1
                frame = sh.render(s_res[None], self.dark[0], self.flat[0], gen)[0]
                a = step(frame)
        ns = max(scored, 1)
        if trace is not None:
            trace[:] = [math.sqrt(v.item() / self.npup) for v in trace]
        return LoopScore(frames=scored,
                         slope_rms_px=math.sqrt(res_s.item() / (ns * 2 * nv)),
                         phase_rms_rad=math.sqrt(res_p.item() / (ns * self.npup)),
                         open_slope_rms_px=math.sqrt(open_s.item() / (ns * 2 * nv)),
                         open_phase_rms_rad=math.sqrt(open_p.item() / (ns * self.npup)))

    # -- the library as the controller ----------------------------------------------
    def controller(self, store: str = "f32") -> Rtc:
        """A library handle with this loop's calibration maps and reconstructor."""
        cfg = self.cfg
        r = Rtc(cfg.nsub, cfg.npx, cfg.nact, obs=cfg.obs, gain=cfg.gain, leak=cfg.leak,
                device=self.device.index or 0)
        r.load_calib(self.dark.cpu().numpy(), self.flat.cpu().numpy())
        r.load_cmat(self.R, store=store)
        return r


def library_step(r: Rtc, device, slopes: torch.Tensor | None = None):
    """frame -> commands through the library on the current CUDA stream.  With
    `slopes` ([frames][nslopes], device) the measured slopes of each frame are kept
    (the stage path: centroid, then reconstruct; the same bits as the fused path)."""
    st = torch.cuda.current_stream(device)
    d_dm = torch.zeros(r.cfg.nact, device=device)
    k = [0]

    def step(frame):
        if slopes is None:
            r.process_frame_async(frame, d_dm, stream=st)
        else:
            row = slopes[k[0]]
            r.centroid_async(frame, row, stream=st)
            r.reconstruct_async(row, d_dm, stream=st)
        k[0] += 1
        return d_dm
    return step


class PolController:
    """Pseudo-open-loop (POL) predictive control with the library's kernels.

    The measured slopes s(k) = s_turb(k) - D a(k-1) plus the mirror's own slopes
    give the POL slopes p(k) = s(k) + D a(k-1), an estimate of the turbulence alone
    that does not depend on the control law.  The learned predictor, trained on POL
    sequences, forecasts p(k+1) from p(k) .. p(k-3); the integrator is then fed the
    residual the new commands will meet, e(k) = p_hat(k+1) - D a(k-1), so that
    a(k) = leak a(k-1) + g R e(k).  With the prediction replaced by p(k) itself this
    is exactly the plain integrator (e = s).  Per frame: rtc_centroid_async (slopes),
    rtc_mvm_integrate_noalloc with D (the POL slopes, p = s + D a), rtc_mlp_predict_seq
    (the forecast) and rtc_reconstruct_async (integrator)."""

    def __init__(self, r: Rtc, D: torch.Tensor, params, sigma: float, cfg, device, predict: bool = True):
        from .rtc import Mlp
        self.r, self.dev, self.cfg, self.sigma = r, device, cfg, float(sigma)
        self.ns, self.na = D.shape
        self.kpad_a = (self.na + 15) // 16 * 16
        self.D = torch.zeros((self.ns, self.kpad_a), device=device)
        self.D[:, :self.na] = D
        self.a_pad = torch.zeros(self.kpad_a, device=device)       # a(k-1), zero padded
        self.s = torch.zeros(self.ns, device=device)
        self.pol = torch.zeros(self.ns, device=device)
        self.hist = torch.zeros((5, self.ns), device=device)        # p(k-3) .. p(k), spare row
        self.out = torch.zeros((5, self.ns), device=device)
        self.e = torch.zeros(self.ns, device=device)
        self.d_dm = torch.zeros(cfg.nact, device=device)
        self.m = None
        if predict:
            self.m = Mlp(device=device.index or 0, params=params)
            self.m.set_geometry(cfg.subaps, cfg.nsub)
        self.k = 0

    def close(self):
        if self.m is not None:
            self.m.close()

    def step(self, frame):
        from .rtc import mvm_integrate_noalloc
        st = torch.cuda.current_stream(self.dev)
        self.r.centroid_async(frame, self.s, stream=st)
        # p = s + D a(k-1): the allocation-free MVM with leak 1 and gain 1 on p := s
        self.pol.copy_(self.s)
        mvm_integrate_noalloc(self.D, "f32", None, self.ns, self.kpad_a, self.a_pad, self.pol, None,
                              1.0, 1.0, 1, stream=st)
        self.hist[:4] = self.hist[1:].clone()
        self.hist[3] = self.pol
        if self.m is not None and self.k >= 3:
            self.m.predict_seq(self.hist, self.sigma, self.out, stream=st)
            p_hat = self.out[4]
        else:
            p_hat = self.pol
        # e = p_hat - D a(k-1) = p_hat - (p - s)
        torch.add(p_hat - self.pol, self.s, out=self.e)
        self.r.reconstruct_async(self.e, self.d_dm, stream=st)
        self.a_pad[:self.na] = self.d_dm
        self.k += 1
        return self.d_dm


def evaluate_pol(cfg=None, train_frames: int = 20_000, test_frames: int = 5_000, seed: int = 0,
                 steps: int | None = None, gains=(0.4, 0.7, 1.0), device="cuda:0",
                 alpha_rel: float = 1e-3) -> dict:
    """Integrator against POL predictive control in the closed loop.  The predictor
    is trained on the POL slopes of an integrator loop through turbulence with other
    seeds; every law is scored on the same held-out turbulence and noise."""
    from .predictor import train_on
    cfg = cfg or synth.elt_scao()
    dev = torch.device(device)
    nl = len(cfg.screen_seeds)
    train_seeds = tuple(2000 + 10 * seed + i for i in range(nl))
    test_seeds = tuple(6000 + 10 * seed + i for i in range(nl))

    sim = ClosedLoopSim(cfg, dev, train_seeds, noise_seed=7100 + seed, alpha_rel=alpha_rel)
    r = sim.controller()
    ctl = PolController(r, sim.D, None, 1.0, cfg, dev, predict=False)
    P = torch.zeros((train_frames, cfg.nslopes), device=dev)

    def record(frame):
        out = ctl.step(frame)
        P[ctl.k - 1] = ctl.pol
        return out
    sim.run(record, train_frames)
    r.close()
    m, sigma, n_steps, loss, train_s = train_on(P, cfg, steps, seed=seed)
    params = m.get_params()
    m.close()
    del P

    test = ClosedLoopSim(cfg, dev, test_seeds, noise_seed=8100 + seed, alpha_rel=alpha_rel)
    out = {"config": cfg.name, "alpha_rel": alpha_rel, "train_frames": train_frames,
           "test_frames": test_frames, "training_steps": n_steps, "final_loss": loss,
           "train_seconds": round(train_s, 2), "sigma_px": sigma, "laws": {}}
    for g in gains:
        for predict in (False, True):
            r = test.controller()
            r.set_gain(g, cfg.leak)
            ctl = PolController(r, test.D, params, sigma, cfg, dev, predict=predict)
            sc = test.run(ctl.step, test_frames)
            ctl.close()
            r.close()
            out["laws"][f"{'pol_predictor' if predict else 'integrator'}_g{g}"] = {
                "phase_nm": sc.phase_rms_nm, "slope_rms_px": sc.slope_rms_px, "frames": sc.frames}
            out["open_loop_phase_nm"] = sc.open_phase_rms_nm
    torch.cuda.synchronize(dev)
    best_i = min((v["phase_nm"], k) for k, v in out["laws"].items() if k.startswith("integrator"))
    best_p = min((v["phase_nm"], k) for k, v in out["laws"].items() if k.startswith("pol_predictor"))
    out["best_integrator"] = {"law": best_i[1], "phase_nm": best_i[0]}
    out["best_pol_predictor"] = {"law": best_p[1], "phase_nm": best_p[0]}
    out["keep_predictor"] = bool(best_p[0] < best_i[0])
    return out


def evaluate(cfg=None, train_frames: int = 20_000, test_frames: int = 5_000, seed: int = 0,
             store: str = "f32", steps: int | None = None, device="cuda:0",
             alpha_rel: float = 1e-3) -> dict:
    """Integrator against integrator + predictor in the closed loop.  The predictor
    is trained on the measured residual slopes of an integrator closed loop through
    turbulence with other seeds; both are then scored on the same held-out
    turbulence and noise."""
    from .predictor import train_on
    cfg = cfg or synth.elt_scao()
    dev = torch.device(device)
    nl = len(cfg.screen_seeds)
    train_seeds = tuple(2000 + 10 * seed + i for i in range(nl))
    test_seeds = tuple(6000 + 10 * seed + i for i in range(nl))

    sim = ClosedLoopSim(cfg, dev, train_seeds, noise_seed=7100 + seed, alpha_rel=alpha_rel)
    r = sim.controller(store)
    S = torch.zeros((train_frames, cfg.nslopes), device=dev)
    train_score = sim.run(library_step(r, dev, slopes=S), train_frames)
    r.close()
    m, sigma, n_steps, loss, train_s = train_on(S, cfg, steps, seed=seed)
    params = m.get_params()
    m.close()
    del S

    test = ClosedLoopSim(cfg, dev, test_seeds, noise_seed=8100 + seed, alpha_rel=alpha_rel)
    r = test.controller(store)
    integ = test.run(library_step(r, dev), test_frames)
    r.close()
    r = test.controller(store)
    r.load_predictor(params, sigma)
    r.set_predictor(True)
    pred = test.run(library_step(r, dev), test_frames)
    r.close()
    torch.cuda.synchronize(dev)
    keep = pred.phase_rms_rad < integ.phase_rms_rad
    return {"config": cfg.name, "store": store, "alpha_rel": alpha_rel, "train_frames": train_frames, "test_frames": test_frames,
            "scored_frames": integ.frames, "training_steps": n_steps, "final_loss": loss,
            "train_seconds": round(train_s, 2), "sigma_px": sigma,
            "train_loop_residual_phase_nm": train_score.phase_rms_nm,
            "open_loop_phase_nm": integ.open_phase_rms_nm,
            "open_loop_slope_rms_px": integ.open_slope_rms_px,
            "integrator_phase_nm": integ.phase_rms_nm, "integrator_slope_rms_px": integ.slope_rms_px,
            "predictor_phase_nm": pred.phase_rms_nm, "predictor_slope_rms_px": pred.slope_rms_px,
            "keep_predictor": bool(keep)}


def main(argv=None):
    import argparse
    import json
    ap = argparse.ArgumentParser(description="Close the loop on a Fried-geometry DM with the "
                                 "least-squares reconstructor; integrator vs integrator + predictor.")
    ap.add_argument("--config", default="elt", choices=["tiny", "elt"])
    ap.add_argument("--train-frames", type=int, default=20_000)
    ap.add_argument("--test-frames", type=int, default=5_000)
    ap.add_argument("--steps", type=int, default=None)
    ap.add_argument("--store", default="f32", choices=["f32", "bf16", "f16", "fp8", "int8"])
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--alpha", type=float, default=1e-3, help="reconstructor regularisation, "
                    "relative to the mean diagonal of D^T D")
    ap.add_argument("--pol", action="store_true", help="pseudo-open-loop predictive control "
                    "against the integrator, at gains 0.4, 0.7 and 1.0")
    a = ap.parse_args(argv)
    if a.pol:
        print(json.dumps(evaluate_pol(synth.CONFIGS[a.config](), a.train_frames, a.test_frames, a.seed,
                                      a.steps, alpha_rel=a.alpha)))
        return
    print(json.dumps(evaluate(synth.CONFIGS[a.config](), a.train_frames, a.test_frames, a.seed,
                              a.store, a.steps, alpha_rel=a.alpha)))


if __name__ == "__main__":
    main()
