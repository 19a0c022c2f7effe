"""The trained predictor against the plain integrator on held-out frames.

Training uses the library's own forward/backward/Adam kernels on slopes that the
pipeline's centroid kernel produced from seeded frozen-flow frames; the held-out
frames use new turbulence and noise seeds.  The predictor must lower the residual
slope RMS below the integrator's one-frame-lag residual, else it would be
switched off."""
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__ as g
    g.build()


def test_trained_predictor_beats_the_integrator_on_held_out_frames():
    from paper_1805_07254_gb300.predictor import train_predictor
    res = train_predictor(synth.tiny_scao(), train_frames=6000, test_frames=1500, steps=2500,
                          batch=1024, lr=2e-3, seed=0)
    print(f"residual RMS: predictor {res.residual_predictor:.5f} px, integrator "
          f"{res.residual_integrator:.5f} px, gain {res.gain:.3f}")
    assert res.keep, (res.residual_predictor, res.residual_integrator)
    assert res.gain > 1.05
