"""The physical closed loop on the CPU: the Fried-geometry DM model against the WFS
model, the least-squares reconstructor, and the loop closed by the FP64 oracle."""
import numpy as np
import pytest
import torch

import synth
from oracle import pipeline as P
from synth.dm import FriedDM, reconstructor
from synth.geometry import subap_index_grid
from synth.wfs import SAMPLES_PER_SUBAP


def _mid():
    return synth.tiny_scao().with_(name="mid_20x20", nsub=20, npx=8, obs=0.2, dm_side=21, diameter_m=8.0)


def _dm(cfg):
    sh = synth.ShackHartmann(cfg)
    return sh, FriedDM(cfg, sh.plate_scale, SAMPLES_PER_SUBAP)


@pytest.mark.parametrize("make", [synth.tiny_scao, _mid])
def test_interaction_matches_the_wfs_on_the_mirror_surface(make):
    """D a equals the WFS gradient operator applied to the interpolated mirror surface
    (two independent computations of the same slopes)."""
    cfg = make()
    sh, dm = _dm(cfg)
    D = dm.interaction()
    a = np.random.default_rng(3).standard_normal((4, dm.nact))
    g = sh._gradients(dm.phase(torch.from_numpy(a).float())) * sh.plate_scale
    s = torch.cat([g[..., 0], g[..., 1]], dim=1).double().numpy()
    np.testing.assert_allclose(s, a @ D.T, atol=1e-5 * np.abs(s).max())


def test_poke_gives_the_four_corner_slopes():
    """A unit command at an interior actuator: the four subapertures around it see
    +-plate/2 in x and y with the signs of their corner, all others nothing."""
    cfg = synth.tiny_scao()
    sh, dm = _dm(cfg)
    D = dm.interaction()
    h = 0.5 * sh.plate_scale
    col = D[:, dm.index[4, 4]]
    grid = subap_index_grid(cfg.nsub, cfg.subaps)
    nv = cfg.n_valid
    expect = {(3, 3): (h, h), (3, 4): (-h, h), (4, 3): (h, -h), (4, 4): (-h, -h)}
    want = np.zeros(2 * nv)
    for (r, c), (sx, sy) in expect.items():
        want[grid[r, c]] = sx
        want[nv + grid[r, c]] = sy
    np.testing.assert_allclose(col, want, rtol=0, atol=1e-15)


@pytest.mark.parametrize("make", [synth.tiny_scao, _mid])
def test_reconstructor_reproduces_the_slopes_of_mirror_shapes(make):
    cfg = make()
    _, dm = _dm(cfg)
    D = dm.interaction()
    R = reconstructor(D)
    assert R.shape == (dm.nact, cfg.nslopes)
    a = np.random.default_rng(5).standard_normal(dm.nact)
    s = D @ a
    assert np.linalg.norm(D @ (R @ s) - s) <= 1e-2 * np.linalg.norm(s)
    # regularisation: a shape the WFS cannot see (piston on a pupil without
    # partial subapertures) is not commanded
    if cfg.obs == 0.0:
        inner = np.array([all(dm.index[r + dr, c + dc] >= 0 for dr in (0, 1) for dc in (0, 1))
                          for r, c in cfg.subaps])
        if inner.all():
            assert np.abs(R @ (D @ np.ones(dm.nact))).max() < 1e-9


def test_closed_loop_with_the_oracle_corrects_the_turbulence():
    """Tiny system, 300 frames: the FP64 oracle as the controller with the
    reconstructor as its matrix takes the residual wavefront and slopes well below
    the turbulence's own."""
    from paper_1805_07254_gb300.closed_loop import ClosedLoopSim
    cfg = synth.tiny_scao()
    sim = ClosedLoopSim(cfg, "cpu")
    loop = P.Loop(sim.R, sim.dark.numpy(), sim.flat.numpy(), cfg.subaps, cfg.npx, cfg.gain, cfg.leak)

    def step(frame):
        a, _ = loop.step(frame.numpy())
        return torch.from_numpy(a).float()

    sc = sim.run(step, 300, burn_in=50)
    assert sc.frames == 250
    assert sc.slope_rms_px < 0.5 * sc.open_slope_rms_px
    assert sc.phase_rms_rad < 0.5 * sc.open_phase_rms_rad
