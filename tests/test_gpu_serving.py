"""Serving several controllers on one GPU with continuous batching: results are the
same alone and in the mix, admission is gated by slots and memory, work overlaps."""
import time

import numpy as np
import pytest

import synth
from helpers import make_pair, rel_rms

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__ as g
    g.build()


def _jobs():
    tiny = synth.tiny_scao()
    elt = synth.elt_scao()
    ft, _ = synth.make_frames(tiny, 0, 60)
    fe, _ = synth.make_frames(elt, 0, 12)
    r1, o1, *_ = make_pair(tiny)
    r2, *_ = make_pair(elt, store="f32")
    r3, *_ = make_pair(elt.with_(matrix_seed=8), store="bf16")
    return [(r1, ft.numpy(), o1), (r2, fe.numpy(), None), (r3, fe.numpy(), None)]


def test_each_result_is_the_same_alone_and_in_the_mix():
    from paper_1805_07254_gb300 import Server
    jobs = _jobs()
    srv = Server(max_slots=3)
    alone = []
    for r, frames, _ in jobs:
        r.reset()
        alone.append(srv.wait(srv.submit(r, frames)))
    for r, _, _ in jobs:
        r.reset()
    slots = [srv.submit(r, frames) for r, frames, _ in jobs]     # admitted while others run
    assert srv.info()["active_slots"] >= 2
    mixed = [srv.wait(s) for s in slots]
    for a, m in zip(alone, mixed):
        np.testing.assert_array_equal(a, m)
    # and the tiny job is the pipeline: DM commands against the FP64 oracle
    r1, ft, o1 = jobs[0]
    for k in range(ft.shape[0]):
        a_ref, _ = o1.step(ft[k])
        assert rel_rms(mixed[0][k], a_ref) <= 1e-5
    assert srv.info() == {"active_slots": 0, "mem_in_use": 0}


def test_admission_waits_for_slots_and_memory():
    from paper_1805_07254_gb300 import Server
    from paper_1805_07254_gb300.rtc import RtcError, RTC_EBUSY
    jobs = _jobs()
    (_, _, _), (r2, fe, _), (r3, _, _) = jobs
    # budget for one ELT job only
    srv = Server(max_slots=4, mem_budget=200 * 1024 * 1024)
    s2 = srv.submit(r2, fe)
    with pytest.raises(RtcError) as e:
        srv.submit(r3, fe)
    assert e.value.code == RTC_EBUSY
    srv.wait(s2)
    srv.wait(srv.submit(r3, fe))
    # one slot only
    srv1 = Server(max_slots=1)
    s = srv1.submit(r2, fe)
    with pytest.raises(RtcError) as e:
        srv1.submit(r3, fe)
    assert e.value.code == RTC_EBUSY
    srv1.wait(s)


def test_jobs_overlap_on_the_device():
    from paper_1805_07254_gb300 import Server
    elt = synth.elt_scao()
    fe, _ = synth.make_frames(elt, 0, 8)
    frames = np.concatenate([fe.numpy()] * 25)             # 200 frames per job
    ra, *_ = make_pair(elt, store="f32")
    rb, *_ = make_pair(elt.with_(matrix_seed=9), store="f32")
    srv = Server(max_slots=2)
    srv.wait(srv.submit(ra, frames[:8]))                    # warm-up
    t0 = time.perf_counter()
    srv.wait(srv.submit(ra, frames))
    srv.wait(srv.submit(rb, frames))
    serial = time.perf_counter() - t0
    t0 = time.perf_counter()
    sa, sb = srv.submit(ra, frames), srv.submit(rb, frames)
    srv.wait(sa)
    srv.wait(sb)
    both = time.perf_counter() - t0
    print(f"two jobs back to back {serial * 1e3:.1f} ms, together {both * 1e3:.1f} ms")
    assert both < 0.9 * serial


def test_handle_calls_are_refused_while_its_job_is_in_a_slot():
    """The job's kernels use the handle's device state: until the job is done the
    handle's own calls return RTC_ESTATE (rtc_destroy included), then it works again."""
    from paper_1805_07254_gb300 import Server
    from paper_1805_07254_gb300.rtc import RtcError, RTC_ESTATE
    cfg = synth.elt_scao()
    frames, _ = synth.make_frames(cfg, 0, 4)
    frames = np.tile(frames.numpy(), (80, 1, 1, 1))          # 320 ELT frames, ~15 ms of work
    r, oracle, M, *_ = make_pair(cfg)
    srv = Server(max_slots=2)
    slot = srv.submit(r, frames)
    if srv.poll(slot)[0]:
        pytest.skip("the job finished before the checks")
    for call in (lambda: r.load_cmat(M), lambda: r.set_readout(74, 10.0), lambda: r.reset(),
                 lambda: r.process_frame(frames[0]), lambda: r.close()):
        with pytest.raises(RtcError) as e:
            call()
        assert e.value.code == RTC_ESTATE
    assert not srv.poll(slot)[0], "the job must still have been running for the checks to count"
    dm = srv.wait(slot)
    assert dm.shape == (frames.shape[0], cfg.nact)
    r.reset()
    oracle.a[:] = 0
    a_ref, _ = oracle.step(frames[0])
    assert rel_rms(r.process_frame(frames[0]), a_ref) <= 1e-5
    r.close()
    srv.close()
