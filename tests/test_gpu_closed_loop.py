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
