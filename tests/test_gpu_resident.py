"""Resident per-frame calls (rtc_resident_start / rtc_process_frame / rtc_resident_stop):
the persistent kernel driven one frame per call from the caller's thread, against the
per-frame launch path and the FP64 oracle; what is refused while resident; an idle
period longer than the kernel's bounded frame wait; and hand-over of the integrator and
predictor history in both directions."""
import time

import numpy as np
import pytest
import torch

import synth
from helpers import make_pair, rel_rms
from paper_1805_07254_gb300.rtc import RTC_ESTATE, RtcError

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__ as g
    g.build()


def _pinned(frames):
    return [torch.from_numpy(np.ascontiguousarray(f)).pin_memory() for f in frames]


def _launch_path(r, pin, n, nact):
    """DM commands of n frames through rtc_process_frame with pinned buffers, one
    kernel launch per frame."""
    dm = torch.empty(nact).pin_memory()
    out = []
    for k in range(n):
        r.process_frame(pin[k % len(pin)], dm_out=dm)
        out.append(dm.numpy().copy())
    return out


@pytest.mark.parametrize("store", ["f32", "bf16", "fp8"])
def test_resident_frames_equal_the_launch_path(store):
    cfg = synth.elt_scao()
    frames, _ = synth.make_frames(cfg, 0, 4)
    pin = _pinned(frames.numpy())
    n = 12
    r1, oracle, *_ = make_pair(cfg, store=store)
    r2, *_ = make_pair(cfg, store=store)
    ref = _launch_path(r2, pin, n, cfg.nact)
    dm = torch.empty(cfg.nact).pin_memory()
    r1.resident_start()
    try:
        for k in range(n):
            r1.process_frame(pin[k % 4], dm_out=dm)
            np.testing.assert_array_equal(dm.numpy(), ref[k])
    finally:
        r1.resident_stop()
    # the integrator state left behind is the launch path's
    np.testing.assert_array_equal(r1.get_dm(), ref[-1])
    if store == "f32":
        for k in range(n):
            a_ref, _ = oracle.step(frames[k % 4].numpy())
        assert rel_rms(ref[-1], a_ref) <= 1e-5


def test_resident_with_predictor_hands_history_both_ways():
    """BF16 + learned predictor: launch-path frames, then resident frames, then launch
    frames again give exactly the all-launch sequence (history ring and integrator
    carried across each switch)."""
    from synth.mlp_init import flatten, init_mlp_params
    cfg = synth.elt_scao()
    frames, _ = synth.make_frames(cfg, 0, 4)
    pin = _pinned(frames.numpy())
    params = flatten(init_mlp_params(3))
    r1, *_ = make_pair(cfg, store="bf16")
    r2, *_ = make_pair(cfg, store="bf16")
    for r in (r1, r2):
        r.load_predictor(params, 0.3)
        r.set_predictor(True)
    n = 14
    ref = _launch_path(r2, pin, n, cfg.nact)
    dm = torch.empty(cfg.nact).pin_memory()
    got = []
    for k in range(n):
        if k == 3:
            r1.resident_start()
        if k == 10:
            r1.resident_stop()
        r1.process_frame(pin[k % 4], dm_out=dm)
        got.append(dm.numpy().copy())
    for k in range(n):
        np.testing.assert_array_equal(got[k], ref[k], err_msg=f"frame {k}")


def test_calls_refused_while_resident_and_allowed_after():
    cfg = synth.tiny_scao()
    frames, _ = synth.make_frames(cfg, 0, 2)
    pin = _pinned(frames.numpy())
    r, *_ = make_pair(cfg)
    dev = torch.device("cuda:0")
    d_frame = torch.from_numpy(frames[0].numpy()).to(dev)
    d_dm = torch.empty(cfg.nact, device=dev)
    r.resident_start()
    try:
        with pytest.raises(RtcError) as e:
            r.resident_start()
        assert e.value.code == RTC_ESTATE
        for call in (lambda: r.process_frame_async(d_frame, d_dm),
                     lambda: r.centroid_async(d_frame),
                     lambda: r.set_gain(0.3, 0.99),
                     lambda: r.reset(),
                     lambda: r.get_dm(),
                     lambda: r.process_frame(frames[0].numpy()),            # pageable frame
                     lambda: r.process_frame(pin[0], want_slopes=True),     # slopes are not served
                     lambda: r.run_loop(2, frames=frames.numpy())):
            with pytest.raises(RtcError) as e:
                call()
            assert e.value.code == RTC_ESTATE
        dm = torch.empty(cfg.nact).pin_memory()
        r.process_frame(pin[0], dm_out=dm)
    finally:
        r.resident_stop()
    r.resident_stop()                     # a second stop is a no-op
    r.process_frame_async(d_frame, d_dm)  # allowed again
    r.synchronize()


def test_idle_longer_than_the_frame_wait_is_transparent():
    """The resident kernel's frame wait is bounded (2 s); a caller idle for longer
    finds it ended, and the next call relaunches it with the state carried over."""
    cfg = synth.tiny_scao()
    frames, _ = synth.make_frames(cfg, 0, 3)
    pin = _pinned(frames.numpy())
    r1, *_ = make_pair(cfg)
    r2, *_ = make_pair(cfg)
    ref = _launch_path(r2, pin, 3, cfg.nact)
    dm = torch.empty(cfg.nact).pin_memory()
    r1.resident_start()
    try:
        r1.process_frame(pin[0], dm_out=dm)
        np.testing.assert_array_equal(dm.numpy(), ref[0])
        time.sleep(2.6)
        for k in (1, 2):
            r1.process_frame(pin[k], dm_out=dm)
            np.testing.assert_array_equal(dm.numpy(), ref[k])
    finally:
        r1.resident_stop()


def test_destroy_stops_a_resident_handle():
    cfg = synth.tiny_scao()
    frames, _ = synth.make_frames(cfg, 0, 1)
    pin = _pinned(frames.numpy())
    r, *_ = make_pair(cfg)
    r.resident_start()
    dm = torch.empty(cfg.nact).pin_memory()
    r.process_frame(pin[0], dm_out=dm)
    r.close()
    # the device is free for other work afterwards
    r2, *_ = make_pair(cfg)
    r2.process_frame(pin[0], dm_out=dm)
    r2.close()


def test_six_wfs_and_asymmetric_cut_resident_equal_the_launch_path():
    """Several WFS in one frame, and a handle re-cut for a banded readout (its frames
    still handed over whole): the resident frames are the launch path's bit for bit."""
    cfg = synth.elt_scao_6wfs()
    frames, _ = synth.make_frames(cfg, 0, 2)
    pin = _pinned(frames.numpy())
    r1, *_ = make_pair(cfg, store="fp8")
    r2, *_ = make_pair(cfg, store="fp8")
    ref = _launch_path(r2, pin, 3, cfg.nact)
    dm = torch.empty(cfg.nact).pin_memory()
    r1.resident_start()
    try:
        for k in range(3):
            r1.process_frame(pin[k % 2], dm_out=dm)
            np.testing.assert_array_equal(dm.numpy(), ref[k])
    finally:
        r1.resident_stop()
    r1.close()
    r2.close()

    cfg = synth.elt_scao()
    frames, _ = synth.make_frames(cfg, 0, 2)
    pin = _pinned(frames.numpy())
    r1, *_ = make_pair(cfg)
    r2, *_ = make_pair(cfg)
    for r in (r1, r2):
        r.set_readout(74, 10.0)
    ref = _launch_path(r2, pin, 3, cfg.nact)
    r1.resident_start()
    try:
        for k in range(3):
            r1.process_frame(pin[k % 2], dm_out=dm)
            np.testing.assert_array_equal(dm.numpy(), ref[k])
    finally:
        r1.resident_stop()


def test_server_refuses_a_resident_handle_and_stop_after_an_idle_expiry():
    from paper_1805_07254_gb300 import Server
    cfg = synth.tiny_scao()
    frames, _ = synth.make_frames(cfg, 0, 2)
    pin = _pinned(frames.numpy())
    r, *_ = make_pair(cfg)
    srv = Server(max_slots=2)
    r.resident_start()
    try:
        with pytest.raises(RtcError) as e:
            srv.submit(r, frames.numpy())
        assert e.value.code == RTC_ESTATE
        # a pinned frame with a pageable DM buffer is refused too
        with pytest.raises(RtcError) as e:
            r.process_frame(pin[0], dm_out=np.empty(cfg.nact, np.float32))
        assert e.value.code == RTC_ESTATE
        time.sleep(2.6)                   # the kernel's frame wait expires meanwhile
    finally:
        r.resident_stop()                 # stopping an already ended kernel is fine
    dm = torch.empty(cfg.nact).pin_memory()
    r.process_frame(pin[0], dm_out=dm)    # the launch path works again
    srv.close()
    r.close()
