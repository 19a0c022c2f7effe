"""The physical closed loop driven by the library on the GPU: parity with the FP64
oracle frame by frame, correction at ELT scale, and the predictor comparison."""
import math

import numpy as np
import pytest
import torch

import synth
from helpers import rel_rms
from oracle import pipeline as P
from oracle import quant as Q

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__ as g
    g.build()


@pytest.mark.parametrize("store", ["f32", "bf16", "int8"])
def test_closed_loop_commands_match_the_oracle_frame_by_frame(store):
    """The library closes the loop on the tiny system; the oracle, stepped on the very
    same frames with the matrix as stored, gives the same commands."""
    tol = 1e-5
    from paper_1805_07254_gb300.closed_loop import ClosedLoopSim, library_step
    cfg = synth.tiny_scao()
    dev = torch.device("cuda:0")
    sim = ClosedLoopSim(cfg, dev)
    r = sim.controller(store)
    lib = library_step(r, dev)
    oracle = P.Loop(Q.stored_matrix(sim.R, store), sim.dark.cpu().numpy(), sim.flat.cpu().numpy(),
                    cfg.subaps, cfg.npx, cfg.gain, cfg.leak)
    errs = []

    def step(frame):
        a = lib(frame)
        a_ref, _ = oracle.step(frame.cpu().numpy())
        errs.append(rel_rms(a.cpu().numpy(), a_ref))
        return a

    sc = sim.run(step, 120, burn_in=20)
    r.close()
    assert max(errs) <= tol, max(errs)
    assert sc.phase_rms_rad < 0.5 * sc.open_phase_rms_rad


def test_elt_closed_loop_corrects_the_turbulence():
    from paper_1805_07254_gb300.closed_loop import ClosedLoopSim, library_step
    cfg = synth.elt_scao()
    dev = torch.device("cuda:0")
    sim = ClosedLoopSim(cfg, dev)
    r = sim.controller("f32")
    sc = sim.run(library_step(r, dev), 300, burn_in=100)
    r.close()
    print(f"ELT closed loop: residual {sc.phase_rms_nm:.1f} nm (open {sc.open_phase_rms_nm:.1f} nm), "
          f"slopes {sc.slope_rms_px:.4f} px (open {sc.open_slope_rms_px:.4f} px)")
    assert sc.frames == 200
    assert sc.phase_rms_rad < 0.3 * sc.open_phase_rms_rad
    assert sc.slope_rms_px < 0.5 * sc.open_slope_rms_px


def test_predictor_comparison_runs_and_reports():
    """The integrator-vs-predictor evaluation end to end on the tiny system (short
    training); both loops score the same held-out turbulence and noise."""
    from paper_1805_07254_gb300.closed_loop import evaluate
    res = evaluate(synth.tiny_scao(), train_frames=3000, test_frames=600, steps=300)
    print(res)
    for k in ("integrator_phase_nm", "predictor_phase_nm", "open_loop_phase_nm",
              "integrator_slope_rms_px", "predictor_slope_rms_px"):
        assert math.isfinite(res[k]) and res[k] > 0
    assert res["integrator_phase_nm"] < res["open_loop_phase_nm"]
    assert res["keep_predictor"] == (res["predictor_phase_nm"] < res["integrator_phase_nm"])


def test_pol_controller_without_prediction_is_the_integrator():
    """The pseudo-open-loop controller with the forecast replaced by the present POL
    slopes feeds the integrator e = s, so it gives the plain integrator's commands bit
    for bit; its POL slopes p = s + D a(k-1), computed by the allocation-free MVM,
    match the same product in FP64."""
    from paper_1805_07254_gb300.closed_loop import ClosedLoopSim, PolController, library_step
    cfg = synth.tiny_scao()
    dev = torch.device("cuda:0")
    sim = ClosedLoopSim(cfg, dev)
    r1, r2 = sim.controller(), sim.controller()
    ctl = PolController(r2, sim.D, None, 1.0, cfg, dev, predict=False)
    lib = library_step(r1, dev)
    D64 = sim.D.double().cpu().numpy()
    worst = [0.0]

    def step(frame):
        a_prev = ctl.a_pad[:cfg.nact].double().cpu().numpy()
        a1 = lib(frame).clone()
        a2 = ctl.step(frame)
        assert torch.equal(a1, a2)
        ref = ctl.s.double().cpu().numpy() + D64 @ a_prev
        worst[0] = max(worst[0], rel_rms(ctl.pol.cpu().numpy(), ref))
        return a2

    sim.run(step, 80, burn_in=10)
    r1.close()
    r2.close()
    assert worst[0] <= 1e-5, worst[0]


def test_pol_predictive_control_runs_and_reports():
    """The POL evaluation end to end on the tiny system (short training): every law
    scores the same held-out turbulence and noise, and the switch follows the scores."""
    from paper_1805_07254_gb300.closed_loop import evaluate_pol
    res = evaluate_pol(synth.tiny_scao(), train_frames=3000, test_frames=600, steps=300, gains=(0.4, 1.0))
    print(res)
    assert set(res["laws"]) == {"integrator_g0.4", "pol_predictor_g0.4", "integrator_g1.0", "pol_predictor_g1.0"}
    for v in res["laws"].values():
        assert math.isfinite(v["phase_nm"]) and 0 < v["phase_nm"] < res["open_loop_phase_nm"]
    assert res["keep_predictor"] == (res["best_pol_predictor"]["phase_nm"] < res["best_integrator"]["phase_nm"])
