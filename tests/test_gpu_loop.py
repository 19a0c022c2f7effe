"""The persistent real-time loop (rtc_run_loop) against the per-frame path and the
FP64 oracle; pacing, early stop, and the bounded frame wait."""
import time

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


def _per_frame_reference(r, frames, n):
    """DM commands of frames[k % len(frames)], k < n, through the fused per-frame kernel."""
    dev = torch.device("cuda:0")
    st = torch.cuda.current_stream()
    d_dm = torch.empty(r.cfg.nact, device=dev)
    out = []
    for k in range(n):
        r.process_frame_async(torch.from_numpy(frames[k % len(frames)]).to(dev), d_dm, stream=st)
        r.synchronize(st)
        out.append(d_dm.cpu().numpy().copy())
    return out


@pytest.mark.parametrize("store", ["f32", "bf16", "f16", "fp8", "int8"])
def test_loop_equals_per_frame_path(store):
    cfg = synth.elt_scao()
    frames, _ = synth.make_frames(cfg, 0, 4)
    frames = frames.numpy()
    n = 12
    r1, *_ = make_pair(cfg, store=store)
    r2, *_ = make_pair(cfg, store=store)
    got = {}
    stats, e2e, dev = r1.run_loop(n, frames=frames, sink=lambda k, dm: got.__setitem__(k, dm))
    assert stats["frames"] == n and len(got) == n
    ref = _per_frame_reference(r2, frames, n)
    for k in range(n):
        np.testing.assert_array_equal(got[k], ref[k])
    np.testing.assert_array_equal(r1.get_dm(), ref[-1])
    assert np.all(e2e > 0) and np.all(dev > 0) and np.all(dev <= e2e)


def test_loop_with_predictor_equals_per_frame_path():
    """BF16 matrix + learned predictor: the loop kernel's frames are the per-frame
    kernel's, bit for bit, and both leave the same history behind."""
    from synth.mlp_init import flatten, init_mlp_params
    cfg = synth.elt_scao()
    frames, _ = synth.make_frames(cfg, 0, 4)
    frames = frames.numpy()
    n = 10
    params = flatten(init_mlp_params(5))
    r1, *_ = make_pair(cfg, store="bf16")
    r2, *_ = make_pair(cfg, store="bf16")
    for r in (r1, r2):
        r.load_predictor(params, 0.3)
        r.set_predictor(True)
    got = {}
    stats, _, _ = r1.run_loop(n, frames=frames, sink=lambda k, dm: got.__setitem__(k, dm))
    assert stats["frames"] == n
    ref = _per_frame_reference(r2, frames, n)
    for k in range(n):
        np.testing.assert_array_equal(got[k], ref[k])
    # the history carries over from the loop into the per-frame path
    ref2 = _per_frame_reference(r2, frames[::-1].copy(), 3)
    got2 = _per_frame_reference(r1, frames[::-1].copy(), 3)
    for a, b in zip(got2, ref2):
        np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("name,store,bands,interval_us", [
    ("elt", "f32", 74, 2.0),          # one band per row of subapertures
    ("elt", "fp8", 7, 0.0),           # bands that cut through subaperture rows
    ("elt", "bf16", 740, 0.0),        # one band per pixel row
    ("six", "fp8", 37, 1.0),          # six WFS read out side by side
    ("tiny", "f32", 3, 5.0),
])
def test_banded_loop_equals_per_frame_path(name, store, bands, interval_us):
    """Frames published band by band (a rolling readout): each block starts on its
    own rows, and the DM commands are the per-frame kernel's, bit for bit."""
    cfg = {"elt": synth.elt_scao, "six": synth.elt_scao_6wfs, "tiny": synth.tiny_scao}[name]()
    frames, _ = synth.make_frames(cfg, 0, 3)
    frames = frames.numpy()
    n = 9
    r1, *_ = make_pair(cfg, store=store)
    r2, *_ = make_pair(cfg, store=store)
    got = {}
    stats, e2e, dev = r1.run_loop(n, frames=frames, sink=lambda k, dm: got.__setitem__(k, dm),
                                  bands=bands, band_interval_us=interval_us)
    assert stats["frames"] == n
    ref = _per_frame_reference(r2, frames, n)
    for k in range(n):
        np.testing.assert_array_equal(got[k], ref[k])
    assert np.all(dev > 0) and np.all(dev <= e2e)


def test_banded_loop_with_scattered_subapertures():
    """A subaperture map with holes and isolated subapertures (runs of one box,
    runs broken by gaps) through the banded ingest, against the oracle."""
    cfg = synth.tiny_scao()
    rng = np.random.default_rng(7)
    sa = cfg.subaps[np.sort(rng.choice(cfg.subaps.shape[0], 23, replace=False))]
    frames, _ = synth.make_frames(cfg, 0, 4)
    frames = frames.numpy()
    r, oracle, *_ = make_pair(cfg, subaps=sa)
    got = {}
    r.run_loop(8, frames=frames, sink=lambda k, dm: got.__setitem__(k, dm), bands=5)
    for k in range(8):
        a_ref, _ = oracle.step(frames[k % len(frames)])
        assert rel_rms(got[k], a_ref) <= 1e-5, k


def test_banded_loop_with_predictor_equals_per_frame_path():
    from synth.mlp_init import flatten, init_mlp_params
    cfg = synth.elt_scao()
    frames, _ = synth.make_frames(cfg, 0, 3)
    frames = frames.numpy()
    params = flatten(init_mlp_params(9))
    r1, *_ = make_pair(cfg, store="bf16")
    r2, *_ = make_pair(cfg, store="bf16")
    for r in (r1, r2):
        r.load_predictor(params, 0.3)
        r.set_predictor(True)
    got = {}
    r1.run_loop(6, frames=frames, sink=lambda k, dm: got.__setitem__(k, dm), bands=74, band_interval_us=2.0)
    ref = _per_frame_reference(r2, frames, 6)
    for k in range(6):
        np.testing.assert_array_equal(got[k], ref[k])


def test_bands_overlap_processing_with_readout():
    """With a slow rolling readout (74 bands, 10 us apart) most of the frame is
    processed before its last rows arrive: last pixel -> DM is well below the
    latency of the same frame published whole."""
    cfg = synth.elt_scao()
    frames, _ = synth.make_frames(cfg, 0, 2)
    frames = frames.numpy()
    r, *_ = make_pair(cfg, store="f32")
    whole, _, _ = r.run_loop(200, rate_hz=1000.0, frames=frames)
    banded, _, _ = r.run_loop(200, rate_hz=1000.0, frames=frames, bands=74, band_interval_us=10.0)
    print(f"dev p50 whole {whole['dev_p50_us']:.2f} us, banded {banded['dev_p50_us']:.2f} us; "
          f"e2e p50 whole {whole['e2e_p50_us']:.2f} us, banded {banded['e2e_p50_us']:.2f} us")
    assert banded["dev_p50_us"] < 0.8 * whole["dev_p50_us"]


def test_loop_rejects_bad_bands():
    from paper_1805_07254_gb300.rtc import RtcError, RTC_EINVAL
    cfg = synth.tiny_scao()
    frames, _ = synth.make_frames(cfg, 0, 1)
    r, *_ = make_pair(cfg)
    for bands, dt in ((-1, 0.0), (cfg.frame_side + 1, 0.0), (4, -1.0), (4, float("nan"))):
        with pytest.raises(RtcError) as e:
            r.run_loop(2, frames=frames.numpy(), bands=bands, band_interval_us=dt)
        assert e.value.code == RTC_EINVAL
    stats, _, _ = r.run_loop(2, frames=frames.numpy(), bands=cfg.frame_side)
    assert stats["frames"] == 2


def test_release_inside_a_callback_is_queued():
    """Releasing other handles, a network and a server from inside the loop's
    callbacks (as a garbage collector may do) is queued until the loop ends
    instead of waiting for the device that runs the loop."""
    from paper_1805_07254_gb300 import Mlp, Server
    cfg = synth.tiny_scao()
    frames, _ = synth.make_frames(cfg, 0, 4)
    frames = frames.numpy()
    r, oracle, *_ = make_pair(cfg)
    others = [make_pair(cfg)[0] for _ in range(2)]
    net, srv = Mlp(), Server(max_slots=2)

    def sink(k, dm):
        if k == 3:
            others.pop().close()
            net.close()
            srv.close()

    def source(k):
        if k == 5:
            others.pop().close()
        return frames[k % 4]

    got = {}
    t0 = time.time()
    stats, _, _ = r.run_loop(12, source=source, sink=lambda k, dm: (sink(k, dm), got.__setitem__(k, dm)))
    assert stats["frames"] == 12 and time.time() - t0 < 1.5
    for k in range(12):
        a_ref, _ = oracle.step(frames[k % 4])
        assert rel_rms(got[k], a_ref) <= 1e-5


def test_loop_tiny_against_oracle():
    cfg = synth.tiny_scao()
    frames, _ = synth.make_frames(cfg, 0, 8)
    frames = frames.numpy()
    n = 64
    r, oracle, *_ = make_pair(cfg)
    got = {}
    r.run_loop(n, frames=frames, sink=lambda k, dm: got.__setitem__(k, dm))
    for k in range(n):
        a_ref, _ = oracle.step(frames[k % len(frames)])
        assert rel_rms(got[k], a_ref) <= 1e-5, k


def test_loop_source_callback_stop_and_continue():
    cfg = synth.tiny_scao()
    frames, _ = synth.make_frames(cfg, 0, 7)
    frames = frames.numpy()
    r, oracle, *_ = make_pair(cfg)

    def source(k):
        return frames[k] if k < 5 else None          # the source ends after 5 frames

    got = {}
    stats, e2e, dev = r.run_loop(20, source=source, sink=lambda k, dm: got.__setitem__(k, dm))
    assert stats["frames"] == 5 and len(e2e) == 5
    for k in range(5):
        a_ref, _ = oracle.step(frames[k])
        assert rel_rms(got[k], a_ref) <= 1e-5
    # the integrator carries on in the per-frame path
    dm = r.process_frame(frames[5])
    a_ref, _ = oracle.step(frames[5])
    assert rel_rms(dm, a_ref) <= 1e-5


def test_loop_paced_rate_and_stats():
    cfg = synth.tiny_scao()
    frames, _ = synth.make_frames(cfg, 0, 2)
    r, *_ = make_pair(cfg)
    stats, e2e, dev = r.run_loop(200, rate_hz=2000.0, frames=frames.numpy())
    assert stats["frames"] == 200
    assert 1600.0 <= stats["frames_per_s"] <= 2100.0, stats["frames_per_s"]
    for pre in ("e2e", "dev"):
        assert 0 < stats[f"{pre}_p50_us"] <= stats[f"{pre}_p99_us"] <= stats[f"{pre}_p999_us"]
        assert stats[f"{pre}_rms_jitter_us"] >= 0
    assert abs(stats["e2e_p50_us"] - np.median(e2e) / 1e3) < 1.0


def test_loop_frame_wait_times_out_and_context_survives():
    """A frame that never comes: the kernel's bounded wait (2 s) expires, the call
    returns RTC_ETIMEDOUT, and the handle keeps working."""
    from paper_1805_07254_gb300.rtc import RtcError, RTC_ETIMEDOUT
    cfg = synth.tiny_scao()
    frames, _ = synth.make_frames(cfg, 0, 3)
    frames = frames.numpy()
    r, oracle, *_ = make_pair(cfg)

    def slow_source(k):
        if k == 2:
            time.sleep(3.0)                          # longer than the device's frame wait
        return frames[k % 3]

    t0 = time.time()
    with pytest.raises(RtcError) as e:
        r.run_loop(4, source=slow_source)
    assert e.value.code == RTC_ETIMEDOUT
    assert time.time() - t0 < 15
    r.reset()
    oracle.a[:] = 0
    dm = r.process_frame(frames[0])
    a_ref, _ = oracle.step(frames[0])
    assert rel_rms(dm, a_ref) <= 1e-5
