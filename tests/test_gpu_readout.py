"""Asymmetric subaperture allocation (rtc_set_readout, Sec. 2.3.3 / Fig. 6 (d)):
the re-cut matrix gives the oracle's DM commands, the on-device re-layout equals
a fresh load under the same cut, the loop equals the per-frame path under it, and
the cut lowers last-pixel -> DM latency of a banded readout."""
import numpy as np
import pytest
import torch

import synth
from helpers import make_pair, rel_rms

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__ as g
    g.build()


def _run(r, frames):
    return [r.process_frame(f).copy() for f in frames]


def test_cut_matches_oracle_and_shrinks_the_last_slices():
    cfg = synth.elt_scao()
    frames, _ = synth.make_frames(cfg, 0, 3)
    frames = frames.numpy()
    r, oracle, *_ = make_pair(cfg, store="f32")
    equal = r.info()["slices"]
    r.set_readout(74, 10.0)
    inf = r.info()
    assert 1 <= inf["slices"] <= equal
    for f in frames:
        a_ref, _ = oracle.step(f)
        assert rel_rms(r.process_frame(f), a_ref) <= 1e-5


@pytest.mark.parametrize("store", ["f32", "bf16", "f16", "fp8", "int8"])
def test_relayout_equals_fresh_load(store):
    """The device re-layout of a resident matrix gives the same bits as loading
    the matrix under the new cut, and restoring equal slices gives a fresh
    handle's bits."""
    cfg = synth.elt_scao()
    frames, _ = synth.make_frames(cfg, 0, 3)
    frames = frames.numpy()
    r1, _, M, *_ = make_pair(cfg, store=store)
    r2, *_ = make_pair(cfg, store=store, M=M)
    r3, *_ = make_pair(cfg, store=store, M=M)
    r1.set_readout(74, 10.0)                       # re-cut the resident matrix
    r2.set_readout(74, 10.0)
    r2.load_cmat(M, store=store)                   # loaded under the cut
    assert r1.info()["slices"] == r2.info()["slices"]
    for a, b in zip(_run(r1, frames), _run(r2, frames)):
        np.testing.assert_array_equal(a, b)
    r1.set_readout(0)
    r1.reset()
    for a, b in zip(_run(r1, frames), _run(r3, frames)):
        np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("name", ["elt", "six"])
def test_loop_under_the_cut_equals_per_frame_path(name):
    cfg = {"elt": synth.elt_scao, "six": synth.elt_scao_6wfs}[name]()
    frames, _ = synth.make_frames(cfg, 0, 3)
    frames = frames.numpy()
    store = "f32" if name == "elt" else "fp8"
    r1, _, M, *_ = make_pair(cfg, store=store)
    r2, *_ = make_pair(cfg, store=store, M=M)
    for r in (r1, r2):
        r.set_readout(74, 10.0)
    got = {}
    r1.run_loop(6, frames=frames, sink=lambda k, dm: got.__setitem__(k, dm), bands=74, band_interval_us=3.0)
    for k, ref in enumerate(_run(r2, [frames[k % 3] for k in range(6)])):
        np.testing.assert_array_equal(got[k], ref)


def test_set_readout_rejects_bad_arguments():
    from paper_1805_07254_gb300.rtc import RtcError, RTC_EINVAL
    cfg = synth.tiny_scao()
    r, oracle, *_ = make_pair(cfg)
    for bands, dt in ((-1, 0.0), (cfg.frame_side + 1, 0.0), (4, -1.0), (4, float("inf"))):
        with pytest.raises(RtcError) as e:
            r.set_readout(bands, dt)
        assert e.value.code == RTC_EINVAL
    frames, _ = synth.make_frames(cfg, 0, 1)
    r.set_readout(cfg.frame_side, 1.0)             # a band per pixel row
    a_ref, _ = oracle.step(frames.numpy()[0])
    assert rel_rms(r.process_frame(frames.numpy()[0]), a_ref) <= 1e-5


def test_cut_lowers_last_pixel_latency():
    """A 1 kHz rolling readout of 74 bands, 10 us apart: last pixel -> DM with equal
    slices and with the asymmetric cut, against the whole frame at once."""
    cfg = synth.elt_scao()
    frames, _ = synth.make_frames(cfg, 0, 2)
    frames = frames.numpy()
    r, *_ = make_pair(cfg, store="f32")
    whole, _, _ = r.run_loop(300, rate_hz=1000.0, frames=frames)
    equal, _, _ = r.run_loop(300, rate_hz=1000.0, frames=frames, bands=74, band_interval_us=10.0)
    r.set_readout(74, 10.0)
    asym, _, _ = r.run_loop(300, rate_hz=1000.0, frames=frames, bands=74, band_interval_us=10.0)
    for name, st in (("whole", whole), ("banded, equal", equal), ("banded, cut", asym)):
        print(f"{name}: dev p50 {st['dev_p50_us']:.2f} p99 {st['dev_p99_us']:.2f} us, "
              f"e2e p50 {st['e2e_p50_us']:.2f} p99 {st['e2e_p99_us']:.2f} us")
    assert asym["dev_p50_us"] < equal["dev_p50_us"] < whole["dev_p50_us"]
